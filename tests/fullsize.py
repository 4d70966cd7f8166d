"""Byte identity of K^c at full size, chunk range by chunk range.

Test infrastructure: the oracle compresses contiguous pieces of whole chunks
(or, in list mode, of whole lists) on every host core, and each piece's
arrays must equal the matching slices of the GPU blob.  Chunks are
independent in the format (segments, bit offsets and payload words are
per chunk), so the pieces together pin every byte of the GPU blob's content:
the chunk directories (as differences), every segment's intercept, slope,
bit offset, start and width, and every payload word.  The header and the
padding bytes are pinned by the whole-blob comparisons of the smaller tests.

The keys travel to the worker processes through shared memory; the pool is
started with `spawn` (the parent holds a CUDA context).
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

import lcf_reader as R

SEG_ARRAYS = ("seg_icpt", "seg_slope", "seg_bitoff", "seg_start", "seg_width")


def _worker_init():
    import oracle

    oracle.build()


def _piece_blob(shm_name, dtype, total, k0, k1, eps, log2, lists):
    import oracle

    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        keys = np.ndarray((total,), dtype=dtype, buffer=shm.buf)[k0:k1].copy()
    finally:
        shm.close()
    if lists is None:
        return oracle.compress(keys, eps, log2)
    lb, le, lg = lists
    return oracle.compress_lists(keys, np.asarray(lb, dtype=np.uint64) - np.uint64(k0), le, lg)


def _compare(g: dict, o: dict, c0: int, c1: int, where: str):
    """The oracle piece o (chunks c0..c1 of the GPU blob g, re-based at 0)."""
    for nm in ("chunk_key_begin", "chunk_seg_begin", "chunk_word_begin"):
        a = g[nm][c0:c1 + 1].astype(np.int64)
        b = o[nm].astype(np.int64)
        assert np.array_equal(a - a[0], b - b[0]), f"{where}: {nm} differs"
    s0, s1 = int(g["chunk_seg_begin"][c0]), int(g["chunk_seg_begin"][c1])
    for nm in SEG_ARRAYS:
        assert np.array_equal(g[nm][s0:s1], o[nm]), f"{where}: {nm} differs"
    w0, w1 = int(g["chunk_word_begin"][c0]), int(g["chunk_word_begin"][c1])
    assert np.array_equal(g["payload"][w0:w1], o["payload"]), f"{where}: payload differs"


def _run(keys: np.ndarray, tasks, compare):
    procs = os.cpu_count() or 1
    shm = shared_memory.SharedMemory(create=True, size=max(1, keys.nbytes))
    try:
        np.ndarray(keys.shape, dtype=keys.dtype, buffer=shm.buf)[:] = keys
        with mp.get_context("spawn").Pool(procs, initializer=_worker_init) as pool:
            args = [(shm.name, keys.dtype, keys.size) + t[1:] for t in tasks]
            for t, blob in zip(tasks, pool.starmap(_piece_blob, args, chunksize=1)):
                compare(t[0], R.parse(blob))
    finally:
        shm.close()
        shm.unlink()


def check_column(gpu_blob: bytes, keys: np.ndarray, eps: int, log2: int = 16, pieces: int | None = None) -> int:
    """Every chunk of a single column; returns the number of chunks compared."""
    g = R.parse(gpu_blob)
    C = g["chunks"]
    cs = 1 << log2
    P = pieces or 4 * (os.cpu_count() or 1)
    per = max(1, -(-C // P))
    tasks = []
    for c0 in range(0, C, per):
        c1 = min(C, c0 + per)
        tasks.append(((c0, c1), c0 * cs, min(keys.size, c1 * cs), eps, log2, None))

    def cmp(cr, o):
        _compare(g, o, cr[0], cr[1], f"chunks {cr[0]}..{cr[1]}")

    _run(keys, tasks, cmp)
    return C


def check_lists(gpu_blob: bytes, keys: np.ndarray, list_begin: np.ndarray, eps, log2, pieces: int | None = None) -> int:
    """Every list of a list-mode column; returns the number of lists compared."""
    g = R.parse(gpu_blob)
    nl = g["lists"]
    lb = np.asarray(list_begin, dtype=np.uint64)
    le = np.broadcast_to(np.asarray(eps, dtype=np.uint64), (nl,))
    lg = np.broadcast_to(np.asarray(log2, dtype=np.uint8), (nl,))
    assert np.array_equal(g["list_key_begin"], lb), "list_key_begin differs"
    assert np.array_equal(g["list_eps"], le) and np.array_equal(g["list_chunk_log2"], lg)
    lcb = g["list_chunk_begin"]
    P = pieces or 4 * (os.cpu_count() or 1)
    # pieces of about equal key counts, cut at list boundaries
    cuts = np.searchsorted(lb, np.linspace(0, int(lb[-1]), P + 1).astype(np.uint64), side="left")
    cuts = np.unique(np.concatenate([[0], cuts, [nl]]))
    tasks = []
    for l0, l1 in zip(cuts[:-1], cuts[1:]):
        l0, l1 = int(l0), int(l1)
        if l1 <= l0:
            continue
        tasks.append(((l0, l1), int(lb[l0]), int(lb[l1]), None, None,
                      (lb[l0:l1 + 1].copy(), le[l0:l1].copy(), lg[l0:l1].copy())))

    def cmp(lr, o):
        l0, l1 = lr
        c0, c1 = int(lcb[l0]), int(lcb[l1])
        assert np.array_equal(o["list_chunk_begin"].astype(np.int64), lcb[l0:l1 + 1].astype(np.int64) - c0)
        _compare(g, o, c0, c1, f"lists {l0}..{l1}")

    _run(keys, tasks, cmp)
    return nl
