"""Thin Python binding of the C ABI in ``include/lc.h`` (ctypes).

Every function has the name of the C entry point it calls and only marshals
arguments: torch tensors become device pointers, the current torch CUDA stream
becomes the ``stream`` argument.  Every step of the compressor runs in the CUDA
kernels of ``liblc.so``; there is no CPU path.  If the library is not built the
first call raises (build it with ``paper_2412_10770_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

LC_OK = 0
LC_ERR_INVALID_ARG = -1
LC_ERR_UNSORTED = -2
LC_ERR_OUT_OF_RANGE = -3
LC_ERR_NOMEM = -4
LC_ERR_CORRUPT = -5
LC_ERR_CUDA = -6
LC_ERR_TIMEOUT = -7
LC_ERR_BUSY = -8
LC_ERR_INTERNAL = -9
LC_ERR_UNSUPPORTED = -10
LC_ERR_STALE = -11

EXPORTS = ("lc_compress", "lc_compress_batch", "lc_decode", "lc_decode_ranges", "lc_decode_ranges_noalloc",
           "lc_decode_batch",
           "lc_access", "lc_lower_bound", "lc_access1", "lc_lower_bound1", "lc_ratio", "lc_size",
           "lc_info", "lc_serialize", "lc_deserialize", "lc_status", "lc_selftest_wait", "lc_free", "lc_free_async",
           "lc_strerror",
           "lc_version", "lc_launch_count", "lc_graph_decode", "lc_graph_launch", "lc_graph_free", "lc_server_create", "lc_server_submit",
           "lc_server_poll", "lc_server_wait", "lc_server_stats", "lc_server_destroy", "lc_serve_sync",
           "lc_timing_enable", "lc_timing_read",
           "lc_for_compress", "lc_for_decode", "lc_for_size", "lc_for_serialize", "lc_for_free",
           "lc_quantile", "lc_decode_approx", "lc_intersect", "lc_union", "lc_chunk_bytes", "lc_compress_jump",
           "lc_pool_usage", "lc_compress_host", "lc_decode_host", "lc_decode_ranges_host", "lc_access_host",
           "lc_lower_bound_host", "lc_batch_create", "lc_batch_launch", "lc_batch_column", "lc_batch_free",
           "lc_set_query_plan")

LC_OP_ACCESS, LC_OP_LOWER_BOUND, LC_OP_DECODE = 1, 2, 3
LC_QUERIES_AUTO, LC_QUERIES_DIRECT, LC_QUERIES_PARTITIONED, LC_QUERIES_DECODED = 0, 1, 2, 3


class LcError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        msg = _lib_or_none().lc_strerror(code).decode() if _lib_or_none() else str(code)
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_uint64), ("chunk_log2", ctypes.c_uint32), ("span_log2", ctypes.c_uint32)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("chunks", ctypes.c_uint64), ("segments", ctypes.c_uint64),
                ("words", ctypes.c_uint64), ("lists", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("eps", ctypes.c_uint64), ("key_bytes", ctypes.c_uint32), ("chunk_log2", ctypes.c_uint32)]


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


class _Request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint32), ("column", ctypes.c_uint32), ("count", ctypes.c_uint64),
                ("begin", ctypes.c_uint64), ("input", ctypes.c_void_p), ("output", ctypes.c_void_p),
                ("user", ctypes.c_uint64)]


class _Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("user", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("batch_size", ctypes.c_uint32), ("latency_us", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("peak_hbm_bytes", ctypes.c_uint64), ("peak_inflight", ctypes.c_uint32), ("slots", ctypes.c_uint32),
                ("launch_us_max", ctypes.c_double), ("launch_us_total", ctypes.c_double),
                ("staging_regrows", ctypes.c_uint64)]


_lib = None


def _lib_or_none():
    return _lib


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblc.so (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(paper_2412_10770_gb300.build.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    p, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    pu64 = ctypes.POINTER(ctypes.c_uint64)
    sig = {
        "lc_compress": ([p, u64, i32, ctypes.POINTER(_Params), p, pp], i32),
        "lc_compress_batch": ([p, p, u64, i32, p, p, ctypes.c_uint32, p, pp], i32),
        "lc_decode": ([p, u64, u64, p, p], i32),
        "lc_decode_ranges": ([p, p, p, p, u64, p, u64, p], i32),
        "lc_decode_ranges_noalloc": ([p, p, p, p, u64, p, u64, p], i32),
        "lc_decode_batch": ([p, p, p], i32),
        "lc_access": ([p, p, u64, p, p], i32),
        "lc_lower_bound": ([p, p, u64, p, p], i32),
        "lc_set_query_plan": ([i32], i32),
        "lc_access1": ([p, u64, pu64], i32),
        "lc_lower_bound1": ([p, u64, pu64], i32),
        "lc_ratio": ([p], ctypes.c_double),
        "lc_size": ([p, pu64], i32),
        "lc_info": ([p, ctypes.POINTER(_Info)], i32),
        "lc_serialize": ([p, p, u64, pu64], i32),
        "lc_deserialize": ([p, u64, p, pp], i32),
        "lc_status": ([p, p], i32),
        "lc_free": ([p], None),
        "lc_free_async": ([p, p], i32),
        "lc_selftest_wait": ([ctypes.c_uint32, p], i32),
        "lc_strerror": ([i32], ctypes.c_char_p),
        "lc_version": ([], i32),
        "lc_launch_count": ([], u64),
        "lc_pool_usage": ([i32, pu64, pu64], i32),
        "lc_compress_host": ([p, u64, i32, ctypes.POINTER(_Params), p, pp], i32),
        "lc_decode_host": ([p, u64, u64, p, p], i32),
        "lc_decode_ranges_host": ([p, p, p, p, u64, p, u64, p], i32),
        "lc_access_host": ([p, p, u64, p, p], i32),
        "lc_lower_bound_host": ([p, p, u64, p, p], i32),
        "lc_batch_create": ([p, p, u64, i32, p, p, ctypes.c_uint32, p, p, pp], i32),
        "lc_batch_launch": ([p, p], i32),
        "lc_batch_column": ([p], p),
        "lc_batch_free": ([p], None),
        "lc_graph_decode": ([p, u64, u64, p, p, pp], i32),
        "lc_graph_launch": ([p, p], i32),
        "lc_graph_free": ([p], None),
        "lc_server_create": ([p, ctypes.c_int, u64, ctypes.c_int, pp], i32),
        "lc_server_submit": ([p, ctypes.POINTER(_Request), pu64], i32),
        "lc_server_poll": ([p, ctypes.POINTER(_Completion), ctypes.c_int, ctypes.POINTER(ctypes.c_int)], i32),
        "lc_server_wait": ([p, ctypes.POINTER(_Completion), ctypes.c_int, ctypes.POINTER(ctypes.c_int), u64], i32),
        "lc_server_stats": ([p, ctypes.POINTER(_ServerStats)], i32),
        "lc_server_destroy": ([p], i32),
        "lc_serve_sync": ([p, ctypes.c_int, ctypes.POINTER(_Request), p, ctypes.POINTER(_Completion)], i32),
        "lc_timing_enable": ([ctypes.c_int], i32),
        "lc_timing_read": ([ctypes.POINTER(_KernelTime), ctypes.c_int, ctypes.POINTER(ctypes.c_int)], i32),
        "lc_for_compress": ([p, u64, i32, p, pp], i32),
        "lc_for_decode": ([p, p, p], i32),
        "lc_for_size": ([p, pu64], i32),
        "lc_for_serialize": ([p, p, u64, pu64], i32),
        "lc_for_free": ([p], None),
        "lc_quantile": ([p, p, u64, u64, i32, p, p], i32),
        "lc_decode_approx": ([p, u64, u64, p, p], i32),
        "lc_intersect": ([p, ctypes.c_int64, p, ctypes.c_int64, p, u64, pu64, p], i32),
        "lc_union": ([p, ctypes.c_int64, p, ctypes.c_int64, p, u64, pu64, p], i32),
        "lc_chunk_bytes": ([p, p, u64], i32),
        "lc_compress_jump": ([p, u64, i32, ctypes.POINTER(_Params), p, pp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int, where: str) -> None:
    if rc != LC_OK:
        raise LcError(rc, where)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _key_bytes(t: torch.Tensor) -> int:
    if t.element_size() not in (4, 8) or t.is_floating_point():
        raise TypeError("keys must be 32- or 64-bit integers")
    return t.element_size()


def _dev(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _out_keys(col: "Column", out: torch.Tensor, need: int, name: str = "out") -> torch.Tensor:
    """An output buffer of the column's key width holding at least `need` keys."""
    _dev(out, name)
    if out.element_size() != col.key_bytes or out.is_floating_point():
        raise TypeError(f"{name} must hold {8 * col.key_bytes}-bit integer keys")
    if out.numel() < need:
        raise ValueError(f"{name} holds {out.numel()} keys, {need} needed")
    return out


def _ranges_args(begin: torch.Tensor, count: torch.Tensor, out_off: torch.Tensor) -> int:
    """begin, count and out_off: CUDA, contiguous, 64-bit integers, one entry per range."""
    for t, nm in ((begin, "begin"), (count, "count"), (out_off, "out_off")):
        _dev(t, nm)
        if t.element_size() != 8 or t.is_floating_point():
            raise TypeError(f"{nm} must hold 64-bit integers")
    if not (begin.numel() == count.numel() == out_off.numel()):
        raise ValueError("begin, count and out_off must have one entry per range")
    return begin.numel()


def key_dtype(key_bytes: int) -> torch.dtype:
    return torch.uint32 if key_bytes == 4 else torch.uint64


class Column:
    """An lc_column handle (owns its device memory; freed with lc_free)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)
        info = lc_info(self)
        self.n = info["n"]
        self.key_bytes = info["key_bytes"]
        self.info = info

    @property
    def dtype(self) -> torch.dtype:
        return key_dtype(self.key_bytes)

    def free(self) -> None:
        if self.handle and self.handle.value and _lib is not None:
            _lib.lc_free(self.handle)
        self.handle = ctypes.c_void_p(0)

    def free_async(self, stream=None) -> None:
        """lc_free_async: release in the order of `stream` without waiting."""
        if self.handle and self.handle.value and _lib is not None:
            h, self.handle = self.handle, ctypes.c_void_p(0)
            _check(_lib.lc_free_async(h, _stream(stream)), "lc_free_async")
        self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # convenience methods
    def decode(self, begin: int = 0, count: int | None = None, out=None, stream=None):
        return lc_decode(self, begin, count, out, stream)

    def access(self, idx, out=None, stream=None):
        return lc_access(self, idx, out, stream)

    def lower_bound(self, values, out=None, stream=None):
        return lc_lower_bound(self, values, out, stream)

    def serialize(self) -> bytes:
        return lc_serialize(self)

    def ratio(self) -> float:
        return lc_ratio(self)


def lc_compress(keys: torch.Tensor, eps: int = 0, chunk_log2: int = 16, stream=None, span_log2: int = 0) -> Column:
    lib = load()
    _dev(keys, "keys")
    kb = _key_bytes(keys)
    h = ctypes.c_void_p()
    prm = _Params(int(eps), int(chunk_log2), int(span_log2))
    _check(lib.lc_compress(keys.data_ptr(), keys.numel(), kb, ctypes.byref(prm), _stream(stream),
                           ctypes.byref(h)), "lc_compress")
    return Column(h.value)


def lc_compress_jump(keys: torch.Tensor, eps: int = 0, chunk_log2: int = 16, stream=None) -> Column:
    """lc_compress with the jump fit (fewest segments; never more than the greedy's)."""
    lib = load()
    _dev(keys, "keys")
    kb = _key_bytes(keys)
    h = ctypes.c_void_p()
    prm = _Params(int(eps), int(chunk_log2))
    _check(lib.lc_compress_jump(keys.data_ptr(), keys.numel(), kb, ctypes.byref(prm), _stream(stream),
                                ctypes.byref(h)), "lc_compress_jump")
    return Column(h.value)


def lc_compress_batch(ids: torch.Tensor, list_begin, eps=0, chunk_log2=16, stream=None, span_log2: int = 0) -> Column:
    lib = load()
    _dev(ids, "ids")
    kb = _key_bytes(ids)
    lb = np.ascontiguousarray(list_begin, dtype=np.uint64)
    nl = lb.size - 1
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.uint64), (nl,)))
    g = np.ascontiguousarray(np.broadcast_to(np.asarray(chunk_log2, dtype=np.uint8), (nl,)))
    h = ctypes.c_void_p()
    _check(lib.lc_compress_batch(ids.data_ptr(), lb.ctypes.data, nl, kb, e.ctypes.data, g.ctypes.data,
                                 int(span_log2), _stream(stream), ctypes.byref(h)), "lc_compress_batch")
    return Column(h.value)


class _BorrowedColumn(Column):
    """A column owned by someone else (a Batch): free() and free_async() do nothing."""

    def __init__(self, handle: int):
        super().__init__(handle)

    def free(self) -> None:
        self.handle = ctypes.c_void_p(0)

    def free_async(self, stream=None) -> None:
        self.handle = ctypes.c_void_p(0)


class Batch:
    """lc_batch_*: a batched compress of posting lists plus a decode of every
    list, recorded once into a CUDA graph and replayed by launch()."""

    def __init__(self, ids: torch.Tensor, list_begin, out: torch.Tensor, eps=0, chunk_log2=16, stream=None,
                 span_log2: int = 0):
        lib = load()
        _dev(ids, "ids")
        kb = _key_bytes(ids)
        _dev(out, "out")
        if out.element_size() != kb or out.numel() < ids.numel():
            raise ValueError("out must hold every id")
        lb = np.ascontiguousarray(list_begin, dtype=np.uint64)
        nl = lb.size - 1
        e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.uint64), (nl,)))
        g = np.ascontiguousarray(np.broadcast_to(np.asarray(chunk_log2, dtype=np.uint8), (nl,)))
        h = ctypes.c_void_p()
        _check(lib.lc_batch_create(ids.data_ptr(), lb.ctypes.data, nl, kb, e.ctypes.data, g.ctypes.data,
                                   int(span_log2), out.data_ptr(), _stream(stream), ctypes.byref(h)),
               "lc_batch_create")
        self.handle = h
        self._keep = (ids, out)
        self.column = _BorrowedColumn(lib.lc_batch_column(h))  # owned by the batch

    def launch(self, stream=None) -> None:
        _check(load().lc_batch_launch(self.handle, _stream(stream)), "lc_batch_launch")

    def free(self) -> None:
        if self.handle and self.handle.value and _lib is not None:
            self.column.free()
            _lib.lc_batch_free(self.handle)
        self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def lc_batch_create(ids: torch.Tensor, list_begin, out: torch.Tensor, eps=0, chunk_log2=16, stream=None,
                    span_log2: int = 0) -> Batch:
    return Batch(ids, list_begin, out, eps, chunk_log2, stream, span_log2)


def lc_batch_launch(batch: Batch, stream=None) -> None:
    batch.launch(stream)


def lc_batch_column(batch: Batch) -> Column:
    return batch.column


def lc_batch_free(batch: Batch) -> None:
    batch.free()


def lc_decode(col: Column, begin: int = 0, count: int | None = None, out=None, stream=None) -> torch.Tensor:
    lib = load()
    if count is None:
        count = col.n - begin
    if out is None:
        out = torch.empty(count, dtype=col.dtype, device="cuda")
    _out_keys(col, out, int(count))
    _check(lib.lc_decode(col.handle, int(begin), int(count), out.data_ptr(), _stream(stream)), "lc_decode")
    return out


def lc_decode_ranges(col: Column, begin: torch.Tensor, count: torch.Tensor, out_off: torch.Tensor, out: torch.Tensor,
                     stream=None) -> torch.Tensor:
    """Range r = keys [begin[r], begin[r] + count[r]) into out at out_off[r];
    a range past N or past the end of out is skipped and recorded in the
    column's status word (lc_status)."""
    lib = load()
    m = _ranges_args(begin, count, out_off)
    _out_keys(col, out, 0)
    _check(lib.lc_decode_ranges(col.handle, begin.data_ptr(), count.data_ptr(), out_off.data_ptr(), m,
                                out.data_ptr(), out.numel(), _stream(stream)), "lc_decode_ranges")
    return out


LC_NOALLOC_MAX_RANGES = 32768


def lc_decode_ranges_noalloc(col: Column, begin: torch.Tensor, count: torch.Tensor, out_off: torch.Tensor,
                             out: torch.Tensor, stream=None) -> torch.Tensor:
    """lc_decode_ranges without any device allocation (at most
    LC_NOALLOC_MAX_RANGES ranges; see include/lc.h)."""
    lib = load()
    m = _ranges_args(begin, count, out_off)
    _out_keys(col, out, 0)
    _check(lib.lc_decode_ranges_noalloc(col.handle, begin.data_ptr(), count.data_ptr(), out_off.data_ptr(), m,
                                        out.data_ptr(), out.numel(), _stream(stream)), "lc_decode_ranges_noalloc")
    return out


def lc_decode_batch(col: Column, out=None, stream=None) -> torch.Tensor:
    lib = load()
    if out is None:
        out = torch.empty(col.n, dtype=col.dtype, device="cuda")
    _out_keys(col, out, col.n)
    _check(lib.lc_decode_batch(col.handle, out.data_ptr(), _stream(stream)), "lc_decode_batch")
    return out


def lc_access(col: Column, idx: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    lib = load()
    _dev(idx, "idx")
    if idx.element_size() != 8:
        raise TypeError("idx must hold 64-bit indices")
    if out is None:
        out = torch.empty(idx.numel(), dtype=col.dtype, device="cuda")
    _out_keys(col, out, idx.numel())
    _check(lib.lc_access(col.handle, idx.data_ptr(), idx.numel(), out.data_ptr(), _stream(stream)), "lc_access")
    return out


def lc_lower_bound(col: Column, values: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    lib = load()
    _dev(values, "values")
    if values.element_size() != col.key_bytes:
        raise TypeError("values must have the column's key width")
    if out is None:
        out = torch.empty(values.numel(), dtype=torch.uint64, device="cuda")
    _dev(out, "out")
    if out.element_size() != 8 or out.numel() < values.numel():
        raise ValueError("out must hold one 64-bit position per value")
    _check(lib.lc_lower_bound(col.handle, values.data_ptr(), values.numel(), out.data_ptr(), _stream(stream)),
           "lc_lower_bound")
    return out


def lc_set_query_plan(plan: int) -> int:
    """How lc_access / lc_lower_bound run a batch (LC_QUERIES_AUTO, _DIRECT,
    _PARTITIONED or _DECODED; process-wide); returns the previous setting."""
    rc = load().lc_set_query_plan(int(plan))
    if rc < 0:
        _check(rc, "lc_set_query_plan")
    return rc


def lc_access1(col: Column, i: int) -> int:
    v = ctypes.c_uint64()
    _check(load().lc_access1(col.handle, int(i), ctypes.byref(v)), "lc_access1")
    return v.value


def lc_lower_bound1(col: Column, x: int) -> int:
    v = ctypes.c_uint64()
    _check(load().lc_lower_bound1(col.handle, int(x), ctypes.byref(v)), "lc_lower_bound1")
    return v.value


def _host(t: torch.Tensor, name: str) -> torch.Tensor:
    if t.is_cuda:
        raise ValueError(f"{name} must be in host memory (page-locked for asynchronous copies)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def lc_compress_host(keys: torch.Tensor, eps: int = 0, chunk_log2: int = 16, stream=None) -> Column:
    """lc_compress from keys in host memory (the library copies them in)."""
    lib = load()
    _host(keys, "keys")
    kb = _key_bytes(keys)
    h = ctypes.c_void_p()
    prm = _Params(int(eps), int(chunk_log2))
    _check(lib.lc_compress_host(keys.data_ptr(), keys.numel(), kb, ctypes.byref(prm), _stream(stream),
                                ctypes.byref(h)), "lc_compress_host")
    return Column(h.value)


def lc_decode_host(col: Column, out: torch.Tensor, begin: int = 0, count: int | None = None, stream=None):
    lib = load()
    if count is None:
        count = col.n - begin
    _host(out, "out")
    if out.element_size() != col.key_bytes or out.numel() < count:
        raise ValueError("out must hold count keys of the column's width")
    _check(lib.lc_decode_host(col.handle, int(begin), int(count), out.data_ptr(), _stream(stream)), "lc_decode_host")
    return out


def lc_decode_ranges_host(col: Column, begin: torch.Tensor, count: torch.Tensor, out_off: torch.Tensor,
                          out: torch.Tensor, stream=None) -> torch.Tensor:
    lib = load()
    for t, nm in ((begin, "begin"), (count, "count"), (out_off, "out_off"), (out, "out")):
        _host(t, nm)
    if not (begin.numel() == count.numel() == out_off.numel()) or begin.element_size() != 8:
        raise ValueError("begin, count and out_off: one 64-bit entry per range")
    if out.element_size() != col.key_bytes:
        raise TypeError("out must hold keys of the column's width")
    _check(lib.lc_decode_ranges_host(col.handle, begin.data_ptr(), count.data_ptr(), out_off.data_ptr(),
                                     begin.numel(), out.data_ptr(), out.numel(), _stream(stream)),
           "lc_decode_ranges_host")
    return out


def lc_access_host(col: Column, idx: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    lib = load()
    _host(idx, "idx")
    _host(out, "out")
    if idx.element_size() != 8 or out.element_size() != col.key_bytes or out.numel() < idx.numel():
        raise ValueError("idx: 64-bit indices; out: one key of the column's width per index")
    _check(lib.lc_access_host(col.handle, idx.data_ptr(), idx.numel(), out.data_ptr(), _stream(stream)),
           "lc_access_host")
    return out


def lc_lower_bound_host(col: Column, values: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    lib = load()
    _host(values, "values")
    _host(out, "out")
    if values.element_size() != col.key_bytes or out.element_size() != 8 or out.numel() < values.numel():
        raise ValueError("values: keys of the column's width; out: one 64-bit position per value")
    _check(lib.lc_lower_bound_host(col.handle, values.data_ptr(), values.numel(), out.data_ptr(), _stream(stream)),
           "lc_lower_bound_host")
    return out


def lc_pool_usage(reset: bool = False) -> tuple[int, int]:
    """(bytes in use now, most in use since the last reset) of the current
    device's default stream-ordered pool; reset=True resets the mark first."""
    now, high = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().lc_pool_usage(1 if reset else 0, ctypes.byref(now), ctypes.byref(high)), "lc_pool_usage")
    return now.value, high.value


def lc_ratio(col: Column) -> float:
    return load().lc_ratio(col.handle)


def lc_size(col: Column) -> int:
    v = ctypes.c_uint64()
    _check(load().lc_size(col.handle, ctypes.byref(v)), "lc_size")
    return v.value


def lc_info(col: Column) -> dict:
    inf = _Info()
    _check(load().lc_info(col.handle, ctypes.byref(inf)), "lc_info")
    return {f: getattr(inf, f) for f, _ in _Info._fields_}


def lc_quantile(col: Column, ks: torch.Tensor, q: int, exact: bool = True, out=None, stream=None) -> torch.Tensor:
    """The ks[r]-th q-quantiles (exact keys, or floor(f) from the segments alone)."""
    lib = load()
    _dev(ks, "ks")
    if ks.element_size() != 8:
        raise TypeError("ks must hold 64-bit integers")
    if out is None:
        out = torch.empty(ks.numel(), dtype=col.dtype, device="cuda")
    _out_keys(col, out, ks.numel())
    _check(lib.lc_quantile(col.handle, ks.data_ptr(), ks.numel(), int(q), 1 if exact else 0, out.data_ptr(),
                           _stream(stream)), "lc_quantile")
    return out


def lc_decode_approx(col: Column, begin: int = 0, count: int | None = None, out=None, stream=None) -> torch.Tensor:
    """floor(f(i)) for i in [begin, begin + count): the segments alone, within eps of the keys."""
    lib = load()
    if count is None:
        count = col.n - begin
    if out is None:
        out = torch.empty(count, dtype=col.dtype, device="cuda")
    _out_keys(col, out, int(count))
    _check(lib.lc_decode_approx(col.handle, int(begin), int(count), out.data_ptr(), _stream(stream)),
           "lc_decode_approx")
    return out


def _set_op(name: str, a: Column, la: int, b: Column, lb: int, out, stream) -> torch.Tensor:
    lib = load()
    fn = getattr(lib, name)
    cnt = ctypes.c_uint64()
    if out is None:
        # the result's length first (capacity 0), then the call that writes it
        rc = fn(a.handle, int(la), b.handle, int(lb), None, 0, ctypes.byref(cnt), _stream(stream))
        if rc not in (LC_OK, LC_ERR_INVALID_ARG) or (rc == LC_ERR_INVALID_ARG and cnt.value == 0):
            _check(rc, name)
        out = torch.empty(cnt.value, dtype=a.dtype, device="cuda")
    _dev(out, "out")
    _check(fn(a.handle, int(la), b.handle, int(lb), out.data_ptr() if out.numel() else None, out.numel(),
              ctypes.byref(cnt), _stream(stream)), name)
    return out[: cnt.value]


def lc_intersect(a: Column, b: Column, la: int = -1, lb: int = -1, out=None, stream=None) -> torch.Tensor:
    """Values in both lists (list la of a, lb of b; -1: the whole single column)."""
    return _set_op("lc_intersect", a, la, b, lb, out, stream)


def lc_union(a: Column, b: Column, la: int = -1, lb: int = -1, out=None, stream=None) -> torch.Tensor:
    """Values in either list, each once."""
    return _set_op("lc_union", a, la, b, lb, out, stream)


def lc_chunk_bytes(col: Column) -> np.ndarray:
    """Bytes each chunk adds to K^c (segments, payload words, directory entries)."""
    C = col.info["chunks"]
    out = np.zeros(max(C, 1), dtype=np.uint64)
    _check(load().lc_chunk_bytes(col.handle, out.ctypes.data, out.size), "lc_chunk_bytes")
    return out[:C]


def lc_serialize(col: Column) -> bytes:
    lib = load()
    n = ctypes.c_uint64()
    lib.lc_serialize(col.handle, None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.lc_serialize(col.handle, buf, n.value, ctypes.byref(n)), "lc_serialize")
    return buf.raw[: n.value]


def lc_deserialize(blob: bytes, stream=None) -> Column:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.lc_deserialize(blob, len(blob), _stream(stream), ctypes.byref(h)), "lc_deserialize")
    return Column(h.value)


def lc_status(col: Column, stream=None) -> int:
    return load().lc_status(col.handle, _stream(stream))


def lc_selftest_wait(polls: int = 1024, stream=None) -> int:
    """The decoders' bounded wait run out on purpose; LC_ERR_TIMEOUT expected."""
    return load().lc_selftest_wait(int(polls), _stream(stream))


def lc_free(col: Column) -> None:
    col.free()


def lc_free_async(col: Column, stream=None) -> None:
    col.free_async(stream)


def lc_version() -> int:
    return load().lc_version()


class Graph:
    """A decode recorded into a CUDA graph (lc_graph_decode); replay with launch()."""

    def __init__(self, handle: int, keep):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep  # column and output must outlive the graph

    def launch(self, stream=None) -> None:
        _check(load().lc_graph_launch(self.handle, _stream(stream)), "lc_graph_launch")

    def free(self) -> None:
        if self.handle and self.handle.value and _lib is not None:
            _lib.lc_graph_free(self.handle)
        self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def lc_graph_decode(col: Column, begin: int = 0, count: int | None = None, out=None, stream=None) -> tuple:
    """Record lc_decode(col, begin, count, out) into a CUDA graph; returns (Graph, out)."""
    lib = load()
    if count is None:
        count = col.n - begin
    if out is None:
        out = torch.empty(count, dtype=col.dtype, device="cuda")
    _dev(out, "out")
    h = ctypes.c_void_p()
    _check(lib.lc_graph_decode(col.handle, int(begin), int(count), out.data_ptr(), _stream(stream), ctypes.byref(h)),
           "lc_graph_decode")
    return Graph(h.value, (col, out)), out


def lc_graph_launch(graph: Graph, stream=None) -> None:
    graph.launch(stream)


def lc_graph_free(graph: Graph) -> None:
    graph.free()


def lc_launch_count() -> int:
    return load().lc_launch_count()


# ---------------------------------------------------------------- serving


def _as_request(op: int, column: int, count: int, begin: int, inp: int, out: int, user: int) -> _Request:
    return _Request(int(op), int(column), int(count), int(begin), ctypes.c_void_p(inp or None),
                    ctypes.c_void_p(out or None), int(user))


def _completion_dict(c: _Completion) -> dict:
    return {"ticket": c.ticket, "user": c.user, "status": c.status, "batch_size": c.batch_size,
            "latency_us": c.latency_us}


class Server:
    """lc_server: continuous batching over device-resident columns.  Request
    inputs and outputs are host addresses (page-locked memory overlaps best)."""

    def __init__(self, cols, hbm_budget: int, slots: int = 4):
        lib = load()
        self._cols = list(cols)
        arr = (ctypes.c_void_p * len(self._cols))(*[c.handle.value for c in self._cols])
        h = ctypes.c_void_p()
        _check(lib.lc_server_create(arr, len(self._cols), int(hbm_budget), int(slots), ctypes.byref(h)),
               "lc_server_create")
        self.handle = h
        self._buf = (_Completion * 1024)()

    def submit(self, op: int, column: int, count: int, begin: int = 0, inp: int = 0, out: int = 0,
               user: int = 0) -> int:
        r = _as_request(op, column, count, begin, inp, out, user)
        t = ctypes.c_uint64()
        _check(load().lc_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "lc_server_submit")
        return t.value

    def poll(self, max_n: int = 1024) -> list:
        got = ctypes.c_int()
        _check(load().lc_server_poll(self.handle, self._buf, min(max_n, 1024), ctypes.byref(got)), "lc_server_poll")
        return [_completion_dict(self._buf[i]) for i in range(got.value)]

    def wait(self, max_n: int = 1024, timeout_us: int = 100000) -> list:
        got = ctypes.c_int()
        rc = load().lc_server_wait(self.handle, self._buf, min(max_n, 1024), ctypes.byref(got), int(timeout_us))
        if rc not in (LC_OK, LC_ERR_TIMEOUT):
            raise LcError(rc, "lc_server_wait")
        return [_completion_dict(self._buf[i]) for i in range(got.value)]

    def stats(self) -> dict:
        st = _ServerStats()
        _check(load().lc_server_stats(self.handle, ctypes.byref(st)), "lc_server_stats")
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def close(self) -> None:
        if self.handle and self.handle.value and _lib is not None:
            _lib.lc_server_destroy(self.handle)
        self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lc_server_create(cols, hbm_budget: int, slots: int = 4) -> Server:
    return Server(cols, hbm_budget, slots)


def lc_server_submit(server: Server, op: int, column: int, count: int, begin: int = 0, inp: int = 0, out: int = 0,
                     user: int = 0) -> int:
    return server.submit(op, column, count, begin, inp, out, user)


def lc_server_poll(server: Server, max_n: int = 1024) -> list:
    return server.poll(max_n)


def lc_server_wait(server: Server, max_n: int = 1024, timeout_us: int = 100000) -> list:
    return server.wait(max_n, timeout_us)


def lc_server_stats(server: Server) -> dict:
    return server.stats()


def lc_server_destroy(server: Server) -> None:
    server.close()


def lc_serve_sync(cols, op: int, column: int, count: int, begin: int = 0, inp: int = 0, out: int = 0, user: int = 0,
                  stream=None) -> dict:
    """The plain path: one request alone, synchronously."""
    lib = load()
    arr = (ctypes.c_void_p * len(cols))(*[c.handle.value for c in cols])
    r = _as_request(op, column, count, begin, inp, out, user)
    c = _Completion()
    _check(lib.lc_serve_sync(arr, len(cols), ctypes.byref(r), _stream(stream), ctypes.byref(c)), "lc_serve_sync")
    return _completion_dict(c)


# ---------------------------------------------------------------- tracing


def lc_timing_enable(on: bool = True) -> None:
    _check(load().lc_timing_enable(1 if on else 0), "lc_timing_enable")


def lc_timing_read() -> dict:
    """Per-kernel device time recorded since the last read: {name: (launches, total_ms)}."""
    buf = (_KernelTime * 64)()
    got = ctypes.c_int()
    _check(load().lc_timing_read(buf, 64, ctypes.byref(got)), "lc_timing_read")
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(got.value)}


# ---------------------------------------------------------------- baseline codec (FOR-delta, block 128)


class ForColumn:
    """An lc_for handle: the frame-of-reference delta bit-packing baseline."""

    def __init__(self, handle: int, n: int, key_bytes: int):
        self.handle = ctypes.c_void_p(handle)
        self.n = n
        self.key_bytes = key_bytes

    def free(self) -> None:
        if self.handle and self.handle.value and _lib is not None:
            _lib.lc_for_free(self.handle)
        self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def lc_for_compress(keys: torch.Tensor, stream=None) -> ForColumn:
    lib = load()
    _dev(keys, "keys")
    kb = _key_bytes(keys)
    h = ctypes.c_void_p()
    _check(lib.lc_for_compress(keys.data_ptr(), keys.numel(), kb, _stream(stream), ctypes.byref(h)),
           "lc_for_compress")
    return ForColumn(h.value, keys.numel(), kb)


def lc_for_decode(f: ForColumn, out=None, stream=None) -> torch.Tensor:
    lib = load()
    if out is None:
        out = torch.empty(f.n, dtype=key_dtype(f.key_bytes), device="cuda")
    _dev(out, "out")
    _check(lib.lc_for_decode(f.handle, out.data_ptr(), _stream(stream)), "lc_for_decode")
    return out


def lc_for_size(f: ForColumn) -> int:
    n = ctypes.c_uint64()
    _check(load().lc_for_size(f.handle, ctypes.byref(n)), "lc_for_size")
    return n.value


def lc_for_serialize(f: ForColumn) -> bytes:
    lib = load()
    n = ctypes.c_uint64()
    lib.lc_for_serialize(f.handle, None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.lc_for_serialize(f.handle, buf, n.value, ctypes.byref(n)), "lc_for_serialize")
    return buf.raw[: n.value]


def lc_for_free(f: ForColumn) -> None:
    f.free()
