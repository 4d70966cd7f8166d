"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data: it holds none of the compressor's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.  Every generator is a
pure function of its arguments and a seed (numpy ``PCG64``), and returns sorted
(non-decreasing) keys.

The paper evaluates decompression on CCNews posting lists (Sec. II-C, Fig. 3a),
a dataset that is not available here; these generators stand in for it and for
the wider key distributions a learned compressor meets:

* ``uniform_gaps``      first key U[0, 1000), gaps U{1..64} (uint32)
* ``lognormal_gaps``    gap = 1 + floor(exp(mu + sigma Z))
* ``piecewise_linear``  equal-width regimes, slope log-uniform [1, 1e4], +-8 jitter
* ``clusters``          dense clusters of 2000 keys (gaps 1..3) separated by
                        gaps U[1e6, 1e9]
* ``posting_lists``     inverted-index lists: rank-Zipf lengths, ids uniform
                        without replacement in a fixed universe
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x4C430000


def seed_for(config: int, generator: int) -> int:
    """Seed of generator ``generator`` in benchmark configuration ``config``."""
    return SEED_BASE + 16 * config + generator


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_gaps(n: int, seed: int, dtype=np.uint32, first_hi: int = 1000,
                 gap_lo: int = 1, gap_hi: int = 64) -> np.ndarray:
    """k_1 ~ U[0, first_hi), then i.i.d. integer gaps U{gap_lo..gap_hi}."""
    rng = _rng(seed)
    if n == 0:
        return np.empty(0, dtype=dtype)
    steps = rng.integers(gap_lo, gap_hi + 1, size=n, dtype=np.uint64)
    steps[0] = rng.integers(0, first_hi, dtype=np.uint64)
    return np.cumsum(steps, dtype=np.uint64).astype(dtype)


def lognormal_gaps(n: int, seed: int, mu: float = 2.0, sigma: float = 1.5,
                   dtype=np.uint64) -> np.ndarray:
    """Gaps 1 + floor(exp(mu + sigma Z)), Z standard normal; first key = first gap."""
    rng = _rng(seed)
    out = np.empty(n, dtype=np.uint64)
    block = 1 << 24
    acc = np.uint64(0)
    for b in range(0, n, block):
        m = min(block, n - b)
        g = np.floor(np.exp(mu + sigma * rng.standard_normal(m))).astype(np.uint64) + np.uint64(1)
        c = np.cumsum(g, dtype=np.uint64) + acc
        out[b:b + m] = c
        acc = c[-1]
    return out.astype(dtype)


def piecewise_linear(n: int, seed: int, regimes: int = 1000, slope_lo: float = 1.0,
                     slope_hi: float = 1e4, jitter: int = 8, dtype=np.uint64) -> np.ndarray:
    """Piecewise-smooth CDF: ``regimes`` equal-width linear pieces whose gap slope
    is log-uniform in [slope_lo, slope_hi], each key jittered by U{-jitter..jitter};
    ties and inversions are then repaired to a strictly increasing sequence
    (k_i = max(k_i, k_{i-1} + 1))."""
    rng = _rng(seed)
    if n == 0:
        return np.empty(0, dtype=dtype)
    regimes = max(1, min(regimes, n))
    edges = (np.arange(regimes + 1, dtype=np.int64) * n) // regimes
    slopes = np.exp(rng.uniform(np.log(slope_lo), np.log(slope_hi), size=regimes))
    out = np.empty(n, dtype=np.int64)
    base = jitter + 1
    for r in range(regimes):
        a, b = int(edges[r]), int(edges[r + 1])
        t = np.arange(b - a, dtype=np.float64)
        jit = rng.integers(-jitter, jitter + 1, size=b - a)
        out[a:b] = base + np.floor(slopes[r] * t).astype(np.int64) + jit
        base += int(np.floor(slopes[r] * (b - a)))
    idx = np.arange(n, dtype=np.int64)
    out = np.maximum.accumulate(out - idx) + idx
    return out.astype(dtype)


def clusters(n: int, seed: int, cluster_size: int = 2000, gap_in_lo: int = 1, gap_in_hi: int = 3,
             gap_out_lo: int = 10**6, gap_out_hi: int = 10**9, dtype=np.uint64) -> np.ndarray:
    """Dense clusters (gaps U{1..3}) of ``cluster_size`` keys, separated by gaps
    U[1e6, 1e9]."""
    rng = _rng(seed)
    g = rng.integers(gap_in_lo, gap_in_hi + 1, size=n, dtype=np.uint64)
    heads = np.arange(0, n, cluster_size)
    g[heads] = rng.integers(gap_out_lo, gap_out_hi + 1, size=heads.size, dtype=np.uint64)
    return np.cumsum(g, dtype=np.uint64).astype(dtype)


GENERATORS = {
    "lognormal": lognormal_gaps,
    "piecewise": piecewise_linear,
    "clusters": clusters,
}


def column(kind: str, n: int, seed: int, dtype=np.uint64) -> np.ndarray:
    """One sorted column from the named generator (``lognormal``, ``piecewise``,
    ``clusters``, ``uniform``)."""
    if kind == "uniform":
        return uniform_gaps(n, seed, dtype=dtype)
    return GENERATORS[kind](n, seed, dtype=dtype)


def uniform_ranks(m: int, n: int, seed: int) -> np.ndarray:
    """m ranks drawn uniformly from [0, n)."""
    return _rng(seed).integers(0, n, size=m, dtype=np.uint64)


def uniform_values(m: int, lo: int, hi: int, seed: int, dtype=np.uint64) -> np.ndarray:
    """m values drawn uniformly from [lo, hi] (inclusive)."""
    return _rng(seed).integers(int(lo), int(hi), size=m, dtype=np.uint64, endpoint=True).astype(dtype)


def zipf_lengths(n_lists: int, total: int, alpha: float = 1.1, lo: int = 16,
                 hi: int = 10**7) -> np.ndarray:
    """Rank-Zipf list lengths: len(r) = clip(round(C r^-alpha), lo, hi) for
    r = 1..n_lists, with C found by bisection so that the lengths sum to about
    ``total``."""
    r = np.arange(1, n_lists + 1, dtype=np.float64) ** (-alpha)

    def tot(c):
        return np.clip(np.rint(c * r), lo, hi).sum()

    a, b = 1.0, float(hi) * 1e3
    for _ in range(200):
        mid = 0.5 * (a + b)
        if tot(mid) < total:
            a = mid
        else:
            b = mid
    return np.clip(np.rint(b * r), lo, hi).astype(np.int64)


def posting_lists(n_lists: int, total: int, universe: int, seed: int, alpha: float = 1.1,
                  lo: int = 16, hi: int = 10**7):
    """Inverted-index posting lists: rank-Zipf lengths (shuffled), each list a
    uniform sample without replacement from [0, universe), sorted.  Returns
    (ids uint32 back to back, list_begin uint64[n_lists + 1])."""
    rng = _rng(seed)
    lens = zipf_lengths(n_lists, total, alpha, lo, min(hi, universe))
    rng.shuffle(lens)
    begin = np.zeros(n_lists + 1, dtype=np.uint64)
    np.cumsum(lens, out=begin[1:])
    ids = np.empty(int(begin[-1]), dtype=np.uint32)
    for l in range(n_lists):
        k = int(lens[l])
        a = int(begin[l])
        if 3 * k > universe:
            pick = rng.permutation(universe)[:k]
        else:
            pick = np.unique(rng.integers(0, universe, size=k + k // 8 + 8))
            while pick.size < k:
                pick = np.unique(np.concatenate([pick, rng.integers(0, universe, size=k)]))
            pick = rng.permutation(pick)[:k]
        ids[a:a + k] = np.sort(pick).astype(np.uint32)
    return ids, begin


def posting_lists_device(n_lists: int, total: int, universe: int, seed: int, alpha: float = 1.1, lo: int = 16,
                         hi: int = 10**7, device: str = "cuda", max_sort: int = 1 << 29):
    """The same posting-list recipe as ``posting_lists``, drawn on the GPU for
    workloads too large for the host: every list draws its ids uniformly with
    replacement, duplicates are dropped and the shortfall is redrawn until each
    list holds its length of distinct ids (the result is a uniform sample
    without replacement: the procedure treats every id alike).  Lists are
    processed in groups of at most ``max_sort`` ids.  Returns (ids uint32
    tensor on ``device``, list_begin uint64 numpy array)."""
    import torch

    rng = _rng(seed)
    lens = zipf_lengths(n_lists, total, alpha, lo, min(hi, universe))
    rng.shuffle(lens)
    begin = np.zeros(n_lists + 1, dtype=np.uint64)
    np.cumsum(lens, out=begin[1:])
    out = torch.empty(int(begin[-1]), dtype=torch.int32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    l0 = 0
    while l0 < n_lists:
        l1 = l0 + 1
        while l1 < n_lists and int(begin[l1 + 1] - begin[l0]) <= max_sort:
            l1 += 1
        lens_g = torch.from_numpy(lens[l0:l1]).to(device)
        lid = torch.repeat_interleave(torch.arange(l1 - l0, device=device, dtype=torch.int64), lens_g)
        key = (lid << 32) | torch.randint(0, universe, (lid.numel(),), generator=gen, device=device)
        del lid
        while True:
            key = torch.sort(key).values
            keep = torch.ones_like(key, dtype=torch.bool)
            keep[1:] = key[1:] != key[:-1]
            key = key[keep]
            deficit = lens_g - torch.bincount(key >> 32, minlength=l1 - l0)
            short = int(deficit.sum())
            if short == 0:
                break
            extra = torch.repeat_interleave(torch.arange(l1 - l0, device=device, dtype=torch.int64), deficit)
            key = torch.cat([key, (extra << 32) | torch.randint(0, universe, (short,), generator=gen, device=device)])
        a, b = int(begin[l0]), int(begin[l1])
        out[a:b] = (key & 0xFFFFFFFF).to(torch.int32)
        del key
        l0 = l1
    return out.view(torch.uint32), begin


def column_device(kind: str, n: int, seed: int, device: str = "cuda", mu: float = 2.0, sigma: float = 1.5,
                  block: int = 1 << 27):
    """The generators of ``column`` drawn on the GPU (same recipes, torch RNG),
    for workloads with many large columns.  ``mu`` and ``sigma`` parametrise the
    lognormal gaps (drawn ``block`` at a time).  Returns a uint64 tensor."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    if kind == "lognormal":
        out = torch.empty(n, dtype=torch.int64, device=device)
        acc = 0
        for b in range(0, n, block):
            m = min(block, n - b)
            z = torch.randn(m, generator=g, device=device, dtype=torch.float64)
            gaps = torch.floor(torch.exp(mu + sigma * z)).to(torch.int64) + 1
            del z
            torch.cumsum(gaps, 0, out=out[b:b + m])
            out[b:b + m] += acc
            acc = int(out[b + m - 1])
            del gaps
        return out.view(torch.uint64)
    if kind == "piecewise":
        regimes = max(1, min(1000, n))
        edges = (torch.arange(regimes + 1, device=device, dtype=torch.int64) * n) // regimes
        lens = edges[1:] - edges[:-1]
        slopes = torch.exp(torch.empty(regimes, device=device, dtype=torch.float64).uniform_(
            0.0, float(np.log(1e4)), generator=g))
        base = 9 + torch.cumsum(torch.floor(slopes * lens.double()).to(torch.int64), 0) - \
            torch.floor(slopes * lens.double()).to(torch.int64)
        r = torch.repeat_interleave(torch.arange(regimes, device=device), lens)
        t = torch.arange(n, device=device, dtype=torch.int64) - edges[:-1][r]
        jit = torch.randint(-8, 9, (n,), generator=g, device=device, dtype=torch.int64)
        k = base[r] + torch.floor(slopes[r] * t.double()).to(torch.int64) + jit
        idx = torch.arange(n, device=device, dtype=torch.int64)
        k = torch.cummax(k - idx, 0).values + idx
        return k.view(torch.uint64)
    if kind == "clusters":
        gaps = torch.randint(1, 4, (n,), generator=g, device=device, dtype=torch.int64)
        heads = torch.arange(0, n, 2000, device=device)
        gaps[heads] = torch.randint(10**6, 10**9 + 1, (heads.numel(),), generator=g, device=device,
                                    dtype=torch.int64)
        return torch.cumsum(gaps, 0).view(torch.uint64)
    raise ValueError(kind)
