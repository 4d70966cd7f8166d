"""Plain CPU oracle of the learned compressor (arXiv 2412.10770).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product path (the
CUDA library in ``paper_2412_10770_gb300``) never imports it, and the two share
no code.  The definitions it follows (Def. 1, Def. 2 / Eq. (1), the residual
encoding of Sec. II-A and Fig. 2) and the "LCF1" byte format it writes are
documented in ``lc_oracle.h``.

The C source is compiled with gcc into ``oracle/_build/liblcoracle.so`` by
:func:`build` (called lazily on first use).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lc_oracle.c")
_SRC_FOR = os.path.join(_HERE, "for_bp128.c")
_HDR = os.path.join(_HERE, "lc_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liblcoracle.so")

ERRORS = {
    -1: "invalid argument",
    -2: "keys not sorted",
    -3: "index out of range",
    -4: "out of memory",
    -5: "corrupt blob",
    -9: "internal error",
}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + __int128, no intrinsics)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)) or max(
        os.path.getmtime(_SRC), os.path.getmtime(_SRC_FOR), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall",
                               "-Wextra", "-o", tmp, _SRC, _SRC_FOR])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def bind(path: str) -> ctypes.CDLL:
    """Load an oracle shared library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    u64, p = ctypes.c_uint64, ctypes.c_void_p
    pp = ctypes.POINTER(ctypes.c_void_p)
    pu64 = ctypes.POINTER(ctypes.c_uint64)
    lib.lco_compress.argtypes = [p, u64, ctypes.c_int, u64, ctypes.c_int, pp, pu64]
    lib.lco_compress_lists.argtypes = [p, p, u64, ctypes.c_int, p, p, pp, pu64]
    lib.lco_compress_jump.argtypes = [p, u64, ctypes.c_int, u64, ctypes.c_int, pp, pu64]
    lib.lco_compress_jump.restype = ctypes.c_int
    lib.lco_info.argtypes = [p, u64, pu64, ctypes.POINTER(ctypes.c_int), pu64, pu64, pu64]
    lib.lco_decode.argtypes = [p, u64, p]
    lib.lco_access.argtypes = [p, u64, p, u64, p]
    lib.lco_lower_bound.argtypes = [p, u64, p, u64, p]
    lib.lco_predict.argtypes = [p, u64, p, u64, p]
    lib.lco_predict.restype = ctypes.c_int
    lib.lco_free.argtypes = [p]
    lib.lco_for_compress.argtypes = [p, u64, ctypes.c_int, pp, pu64]
    lib.lco_for_decode.argtypes = [p, u64, p]
    lib.lco_for_compress.restype = ctypes.c_int
    lib.lco_for_decode.restype = ctypes.c_int
    for f in ("lco_compress", "lco_compress_lists", "lco_info", "lco_decode",
              "lco_access", "lco_lower_bound"):
        getattr(lib, f).restype = ctypes.c_int
    lib.lco_free.restype = None
    return lib


def _L():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def _check(rc: int) -> None:
    if rc != 0:
        raise OracleError(rc)


def _keys_array(keys) -> np.ndarray:
    a = np.ascontiguousarray(keys)
    if a.dtype not in (np.uint32, np.uint64):
        raise TypeError("keys must be uint32 or uint64")
    return a


def _take_blob(ptr: ctypes.c_void_p, length: int) -> bytes:
    try:
        return ctypes.string_at(ptr.value, length) if length else b""
    finally:
        _L().lco_free(ptr)


def compress(keys, eps: int, chunk_log2: int = 16) -> bytes:
    """K^c of one sorted column (uint32 or uint64 keys)."""
    a = _keys_array(keys)
    blob, n = ctypes.c_void_p(), ctypes.c_uint64()
    _check(_L().lco_compress(a.ctypes.data, a.size, a.itemsize, int(eps), int(chunk_log2),
                             ctypes.byref(blob), ctypes.byref(n)))
    return _take_blob(blob, n.value)


def compress_jump(keys, eps: int, chunk_log2: int = 16) -> bytes:
    """K^c of one sorted column with the jump fit (fewest segments among greedy
    prefixes, see lc_oracle.h)."""
    a = _keys_array(keys)
    blob, n = ctypes.c_void_p(), ctypes.c_uint64()
    _check(_L().lco_compress_jump(a.ctypes.data, a.size, a.itemsize, int(eps), int(chunk_log2),
                                  ctypes.byref(blob), ctypes.byref(n)))
    return _take_blob(blob, n.value)


def compress_lists(keys, list_begin, eps, chunk_log2) -> bytes:
    """K^c of many sorted lists stored back to back (list mode)."""
    a = _keys_array(keys)
    lb = np.ascontiguousarray(list_begin, dtype=np.uint64)
    nl = lb.size - 1
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.uint64), (nl,)))
    g = np.ascontiguousarray(np.broadcast_to(np.asarray(chunk_log2, dtype=np.uint8), (nl,)))
    blob, n = ctypes.c_void_p(), ctypes.c_uint64()
    _check(_L().lco_compress_lists(a.ctypes.data, lb.ctypes.data, nl, a.itemsize, e.ctypes.data,
                                   g.ctypes.data, ctypes.byref(blob), ctypes.byref(n)))
    return _take_blob(blob, n.value)


def info(blob: bytes) -> dict:
    n, c, l, w = (ctypes.c_uint64() for _ in range(4))
    kb = ctypes.c_int()
    _check(_L().lco_info(blob, len(blob), ctypes.byref(n), ctypes.byref(kb), ctypes.byref(c),
                         ctypes.byref(l), ctypes.byref(w)))
    return {"n": n.value, "key_bytes": kb.value, "chunks": c.value, "segments": l.value,
            "words": w.value}


def _dtype(kb: int):
    return np.uint32 if kb == 4 else np.uint64


def decode(blob: bytes) -> np.ndarray:
    """Dec(K^c): every key."""
    inf = info(blob)
    out = np.empty(inf["n"], dtype=_dtype(inf["key_bytes"]))
    _check(_L().lco_decode(blob, len(blob), out.ctypes.data))
    return out


def access(blob: bytes, idx) -> np.ndarray:
    """K[i] for every i in idx."""
    inf = info(blob)
    ix = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(ix.size, dtype=_dtype(inf["key_bytes"]))
    _check(_L().lco_access(blob, len(blob), ix.ctypes.data, ix.size, out.ctypes.data))
    return out


def predict(blob: bytes, idx) -> np.ndarray:
    """floor(f(i)) for every i in idx: the model alone, without residuals."""
    inf = info(blob)
    ix = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(ix.size, dtype=_dtype(inf["key_bytes"]))
    _check(_L().lco_predict(blob, len(blob), ix.ctypes.data, ix.size, out.ctypes.data))
    return out


def quantile_index(n: int, k: int, q: int) -> int:
    """Index of the k-th q-quantile (Sec. III-C): floor(n k / q), the last key
    for k = q (exact integer arithmetic)."""
    return min(n * k // q, n - 1)


def lower_bound(blob: bytes, values) -> np.ndarray:
    """First i with K[i] >= v for every v in values (N if none)."""
    inf = info(blob)
    v = np.ascontiguousarray(values, dtype=_dtype(inf["key_bytes"]))
    out = np.empty(v.size, dtype=np.uint64)
    _check(_L().lco_lower_bound(blob, len(blob), v.ctypes.data, v.size, out.ctypes.data))
    return out


def for_compress(keys) -> bytes:
    """The FOR1 blob of the frame-of-reference delta bit-packing baseline
    (blocks of 128 keys; see for_bp128.c)."""
    a = _keys_array(keys)
    blob, n = ctypes.c_void_p(), ctypes.c_uint64()
    _check(_L().lco_for_compress(a.ctypes.data, a.size, a.itemsize, ctypes.byref(blob), ctypes.byref(n)))
    return _take_blob(blob, n.value)


def for_decode(blob: bytes) -> np.ndarray:
    """Every key of a FOR1 blob."""
    if len(blob) < 32:
        raise OracleError(-5)
    kb = int.from_bytes(blob[4:8], "little")
    n = int.from_bytes(blob[8:16], "little")
    out = np.empty(n, dtype=_dtype(kb) if kb in (4, 8) else np.uint64)
    _check(_L().lco_for_decode(blob, len(blob), out.ctypes.data))
    return out
