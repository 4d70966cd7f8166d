"""Autotuner of the fit parameters for batches of posting lists.

The paper's only hyper-parameter is eps (Sec. II-A, Sec. IV-A): a larger eps
means fewer segments but wider residuals.  BitTuner's closed form (quoted in
Sec. II-A / IV-A) puts the optimum near eps* = sqrt(2 ln2 sigma^2 C (K + 2F)),
with sigma^2 the variance of the key gaps and C a data-dependent constant the
paper leaves open; Sec. IV-A notes that a single global eps is not optimal
when lists differ.  This tuner therefore picks (eps, chunk_log2) per bucket of
list lengths (powers of two) by measurement: it compresses a sample of each
bucket's lists under every candidate, on the GPU, in batched calls, and keeps
the smallest K^c.  The BitTuner value is computed per bucket beside the choice,
with C fitted across the buckets, as a reference.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import lc

EPS_CANDIDATES = tuple([0] + [(1 << k) - 1 for k in range(1, 25)])
LOG2_CANDIDATES = (10, 12, 14, 16)


def _bucket(length: int) -> int:
    return max(0, int(length).bit_length() - 1)


def _sample_batch(ids: torch.Tensor, begin: np.ndarray, lists: np.ndarray, max_keys: int):
    """Concatenate (prefixes of) the chosen lists, at most max_keys ids in all."""
    parts, lens = [], []
    budget = max_keys
    for l in lists:
        a, b = int(begin[l]), int(begin[l + 1])
        take = min(b - a, max(16, budget // max(1, len(lists))))
        parts.append(ids[a:a + take])
        lens.append(take)
    sb = np.zeros(len(lens) + 1, dtype=np.uint64)
    np.cumsum(lens, out=sb[1:])
    return torch.cat(parts).contiguous(), sb


def _size(ids: torch.Tensor, sb: np.ndarray, eps: int, log2: int) -> int:
    col = lc.lc_compress_batch(ids, sb, eps, log2)
    try:
        return lc.lc_size(col)
    finally:
        col.free()


def tune(ids: torch.Tensor, begin: np.ndarray, sample_lists: int = 24, sample_keys: int = 1 << 20,
         seed: int = 0, eps_candidates=EPS_CANDIDATES, log2_candidates=LOG2_CANDIDATES):
    """Per-list (eps, chunk_log2) for the lists ids[begin[l]:begin[l+1]].

    Returns (eps uint64[nl], chunk_log2 uint8[nl], table) where table lists,
    per length bucket, the chosen parameters, the sample's bits per key, the
    gap variance and the BitTuner reference value."""
    begin = np.asarray(begin, dtype=np.uint64)
    lens = np.diff(begin).astype(np.int64)
    nl = lens.size
    rng = np.random.Generator(np.random.PCG64(seed))
    buckets = {}
    for l in range(nl):
        if lens[l] > 0:
            buckets.setdefault(_bucket(lens[l]), []).append(l)
    eps_of = np.zeros(nl, dtype=np.uint64)
    log2_of = np.full(nl, 16, dtype=np.uint8)
    kb = ids.element_size()
    table = []
    for bkt in sorted(buckets):
        members = np.array(buckets[bkt])
        pick = rng.choice(members, size=min(sample_lists, members.size), replace=False)
        sids, sb = _sample_batch(ids, begin, np.sort(pick), sample_keys)
        nkeys = int(sb[-1])
        # eps first (at the widest chunk), then the chunk length for lists that span chunks
        sizes = {e: _size(sids, sb, e, 16) for e in eps_candidates}
        best_eps = min(sizes, key=lambda e: (sizes[e], e))
        best_log2, best = 16, sizes[best_eps]
        if (1 << bkt) > (1 << min(log2_candidates)):
            for g in log2_candidates:
                if g == 16:
                    continue
                s = _size(sids, sb, best_eps, g)
                if s < best:
                    best, best_log2 = s, g
        h = sids.to(torch.int64)
        gaps = []
        for i in range(len(sb) - 1):
            seg = h[int(sb[i]):int(sb[i + 1])]
            if seg.numel() > 1:
                gaps.append(seg[1:] - seg[:-1])
        var = float(torch.cat(gaps).double().var()) if gaps else 0.0
        eps_of[members] = best_eps
        log2_of[members] = best_log2
        table.append({"bucket_min_len": 1 << bkt, "lists": int(members.size), "sample_keys": nkeys, "eps": best_eps,
                      "chunk_log2": best_log2, "bits_per_key": 8.0 * best / nkeys, "gap_var": var,
                      "raw_bits_per_key": 8 * kb})
    # BitTuner reference: eps* = sqrt(2 ln2 sigma^2 C (K + 2F)); C fitted (median) over the buckets
    K, F = 8 * kb, 64
    ratios = [t["eps"] ** 2 / (2 * math.log(2) * t["gap_var"] * (K + 2 * F)) for t in table
              if t["eps"] > 0 and t["gap_var"] > 0]
    C = float(np.median(ratios)) if ratios else 0.0
    for t in table:
        t["bittuner_eps"] = math.sqrt(2 * math.log(2) * t["gap_var"] * C * (K + 2 * F)) if t["gap_var"] > 0 else 0.0
    return eps_of, log2_of, {"buckets": table, "bittuner_C": C, "K": K, "F": F}


# ---------------------------------------------------------------- eps per partition (Sec. IV-A, Fig. 5)

# Bytes one more partition adds: its list directory entries (key begin, chunk
# begin, eps, chunk_log2).
PART_OVERHEAD = 8 + 8 + 8 + 1


def best_partition(costs: np.ndarray, switch: float = PART_OVERHEAD):
    """The shortest path of the partition graph (Sec. IV-A, Fig. 5) at chunk
    granularity.  costs[e, c] = bytes of chunk c compressed with candidate e.
    Chunks are independent in the format, so a partition's cost is the sum of
    its chunks' costs under its eps, plus `switch` per partition; the best
    partitioning is a shortest path over the states (chunk, eps), solved by
    dynamic programming in O(E C).  Returns (choice[c] = candidate index of
    chunk c, total cost)."""
    E, C = costs.shape
    if C == 0:
        return np.zeros(0, dtype=np.int64), 0.0
    D = costs[:, 0].astype(np.float64) + switch
    back = np.zeros((C, E), dtype=np.int64)
    back[0] = np.arange(E)
    idx = np.arange(E)
    for c in range(1, C):
        a = int(np.argmin(D))
        new = D[a] + switch
        stay = D <= new  # continuing the partition beats opening a new one
        back[c] = np.where(stay, idx, a)
        D = np.where(stay, D, new) + costs[:, c]
    e = int(np.argmin(D))
    total = float(D[e])
    choice = np.empty(C, dtype=np.int64)
    for c in range(C - 1, -1, -1):
        choice[c] = e
        e = int(back[c, e])
    return choice, total


def partition_eps(keys: torch.Tensor, eps_candidates=(0, 1, 3, 7, 15, 31, 63, 127, 255, 511, 1023), chunk_log2: int = 16,
                  switch: float = PART_OVERHEAD, chunk_costs=None):
    """eps per partition of one sorted column (Sec. IV-A): compress the column
    once per candidate eps on the GPU, read every chunk's cost
    (lc_chunk_bytes), take the shortest path of best_partition, and return
    (part_begin uint64[P+1] key offsets, part_eps uint64[P], info).  The
    partitions are whole chunks; lc_compress_batch(keys, part_begin,
    part_eps, chunk_log2) stores them as one list-mode column.  chunk_costs:
    an optional {eps: per-chunk bytes} already measured."""
    n = keys.numel()
    cs = 1 << chunk_log2
    costs = []
    for e in eps_candidates:
        if chunk_costs is not None and e in chunk_costs:
            costs.append(np.asarray(chunk_costs[e], dtype=np.float64))
            continue
        col = lc.lc_compress(keys, eps=int(e), chunk_log2=chunk_log2)
        try:
            costs.append(lc.lc_chunk_bytes(col).astype(np.float64))
        finally:
            col.free()
    costs = np.stack(costs)
    choice, total = best_partition(costs, switch)
    C = costs.shape[1]
    starts = [0] + [c for c in range(1, C) if choice[c] != choice[c - 1]]
    part_begin = np.array([min(n, s * cs) for s in starts] + [n], dtype=np.uint64)
    part_eps = np.array([eps_candidates[choice[s]] for s in starts], dtype=np.uint64)
    single = costs.sum(axis=1)
    info = {"partitions": len(starts), "dp_bytes": total, "best_single_eps": int(eps_candidates[int(np.argmin(single))]),
            "best_single_bytes": float(single.min())}
    return part_begin, part_eps, info


SPAN_CANDIDATES = (5, 6, 7)


def tune_span(ids: torch.Tensor, begin: np.ndarray, eps, log2, spans=SPAN_CANDIDATES, reps: int = 2):
    """The third parameter: keys per speculating thread of the fit (2^span_log2;
    256, 128 or 64 threads per 8192-key window).  It changes the launch, not
    the bytes, so it is picked by time: the batch is compressed reps times
    with each candidate (CUDA events, after one untimed run) and the fastest
    mean wins.  Returns (span_log2, {span_log2: ms})."""
    stream = torch.cuda.current_stream()
    times = {}
    for sp in spans:
        lc.lc_compress_batch(ids, begin, eps, log2, stream=stream, span_log2=sp).free()
        ms = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            col = lc.lc_compress_batch(ids, begin, eps, log2, stream=stream, span_log2=sp)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b) / reps
            col.free()
        times[sp] = ms
    best = min(times, key=lambda k: (times[k], k))
    return best, times
