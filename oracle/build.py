"""Compile the C oracle into oracle/liboracle.so with gcc.

TEST INFRASTRUCTURE ONLY.  Plain IEEE double arithmetic: no fast-math and no
FMA contraction, so the oracle gives the same bits on x86-64 and AArch64.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pic_oracle.c")
HDR = os.path.join(HERE, "pic_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")


def build(force=False):
    """Build the oracle library if it is missing or older than its sources."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if t >= os.path.getmtime(SRC) and t >= os.path.getmtime(HDR):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
