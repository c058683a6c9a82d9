"""Build libpic.so (the CUDA library behind include/pic.h) in-tree for sm_103a."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpic.so")
SOURCES = ["pic_capi.cu", "pic_noalloc.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _newest_source():
    names = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    names.append(os.path.join(os.path.dirname(HERE), "include", "pic.h"))
    return max(os.path.getmtime(n) for n in names)


def build(force=False, verbose=False):
    """Compile the library unless it is newer than every source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_source():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC, "-O3", "-std=c++17", ARCH, "-lineinfo", "-shared", "-Xcompiler", "-fPIC",
           "-o", tmp] + [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd, stdout=sys.stdout if verbose else subprocess.DEVNULL)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
