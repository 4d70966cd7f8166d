"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lc.h declares; the Python binding names the same functions.  No
GPU needed: nothing here launches a kernel."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_2412_10770_gb300 import build as lcbuild
from paper_2412_10770_gb300 import lc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lc_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def libpath():
    return lcbuild.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    decl = declared_symbols()
    assert decl, "no declarations found"
    missing = [s for s in sorted(decl) if not hasattr(lib, s)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_the_abi():
    decl = declared_symbols()
    assert set(lc.EXPORTS) <= decl
    for name in lc.EXPORTS:
        assert callable(getattr(lc, name, None)) or name in ("lc_strerror",)


def test_strerror_and_version_without_gpu(libpath):
    lib = lc.load(libpath)
    assert lib.lc_version() >= 10000
    assert lib.lc_strerror(lc.LC_ERR_UNSORTED) == b"keys are not sorted"
    assert lib.lc_strerror(12345) == b"unknown status"


def test_invalid_arguments_are_rejected_before_any_device_work(libpath):
    lib = lc.load(libpath)
    h = ctypes.c_void_p()
    prm = lc._Params(1 << 31, 16)
    assert lib.lc_compress(ctypes.c_void_p(16), 10, 8, ctypes.byref(prm), None, ctypes.byref(h)) == lc.LC_ERR_INVALID_ARG
    prm = lc._Params(1, 7)
    assert lib.lc_compress(ctypes.c_void_p(16), 10, 8, ctypes.byref(prm), None, ctypes.byref(h)) == lc.LC_ERR_INVALID_ARG
    prm = lc._Params(1, 16)
    assert lib.lc_compress(ctypes.c_void_p(16), 10, 3, ctypes.byref(prm), None, ctypes.byref(h)) == lc.LC_ERR_INVALID_ARG
    assert lib.lc_compress(None, 10, 8, ctypes.byref(prm), None, ctypes.byref(h)) == lc.LC_ERR_INVALID_ARG
    assert lib.lc_decode(None, 0, 0, None, None) == lc.LC_ERR_INVALID_ARG
    assert lib.lc_ratio(None) < 0
    assert lib.lc_free_async(None, None) == lc.LC_ERR_INVALID_ARG
    assert lib.lc_selftest_wait(0, None) == lc.LC_ERR_INVALID_ARG
    assert lib.lc_selftest_wait((1 << 20) + 1, None) == lc.LC_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(lc, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lc.load(str(tmp_path / "nope.so"))
