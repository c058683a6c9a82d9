"""The C-ABI library builds, loads and exports every entry point of include/pic.h.

No compute call is made, so this runs without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(pic_\w+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1204_0838_gb300 import build
    return build.build()


def test_header_declares_the_paper_api():
    names = _declared()
    for n in ["pic_create", "pic_add_species", "pic_add_laser", "pic_step", "pic_diag",
              "pic_destroy", "pic_batch_create", "pic_batch_step", "pic_batch_diag",
              "pic_batch_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pic_\w+)", out))
    assert set(_declared()) <= exported


def test_library_is_built_for_sm_103a(libpath):
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", libpath],
                         capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_version_string_needs_no_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.pic_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.pic_version()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1204_0838_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"(from|import)\s+oracle|liboracle|pic_oracle", src), fn
