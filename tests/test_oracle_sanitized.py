"""The oracle under the address and undefined-behaviour sanitizers: every path
(periodic and open x, window, both laser modes, both solvers, absorbing
layers, all diagnostics) runs once in a small case (oracle/selfcheck.c) and
must finish with no out-of-bounds access, leak or undefined operation."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "selfcheck")
    src = [os.path.join(ROOT, "oracle", f) for f in ("selfcheck.c", "pic_oracle.c")]
    flags = ["-std=c11", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
             "-fno-omit-frame-pointer", "-ffp-contract=off"]
    build = subprocess.run([gcc, *flags, *src, "-lm", "-o", exe], capture_output=True, text=True)
    if build.returncode != 0 and "asan" in build.stderr.lower():
        pytest.skip("sanitizer runtime not installed")
    assert build.returncode == 0, build.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "0 failure(s)" in run.stdout
