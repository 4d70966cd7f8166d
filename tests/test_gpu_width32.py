"""Residual width 32, the widest the format allows (Sec. II-A's
ceil(log2(2 eps + 1)) bits at eps = 2^30).

A zigzag code of 32 bits needs a residual of exactly +2^30 = +eps.  The keys
below make one: a line of slope s = 2^20 per index, a key eps above the line
at index t followed by a plateau of equal keys (allowed: keys are
non-decreasing) until the line has risen 2 eps, and a key eps below the line
right after the plateau.  The first key pins the cone's lower edge to s
exactly and the last pins its upper edge to s plus less than 2^32 / i2
(Q32), so the floor-midpoint slope predicts s t at t and the residual there
is +eps.  The segment is one of ~2000 keys with a positive slope, so
lower_bound takes its line-bracket search, whose half-width is 2^(w-1) keys
of value: at w = 32 that is 2^31, which must not wrap to 0.
"""
from __future__ import annotations

import numpy as np
import pytest

import lcf_reader as R
import oracle

EPS = 1 << 30


def width32_keys(s: int = 1 << 20, t: int = 10, tail: int = 200) -> np.ndarray:
    m = 2 * EPS // s  # plateau length: the line rises 2 eps over it
    i2 = t + m + 1
    k = [s * i for i in range(t)]
    k += [s * t + EPS] * (m + 1)  # indices t .. t + m
    k += [s * i2 - EPS]  # index i2
    k += [s * i for i in range(i2 + 1, i2 + 1 + tail)]
    return np.array(k, dtype=np.uint64)


CASES = [(1 << 20, 10), (1 << 18, 5), (1 << 21, 40)]


@pytest.mark.parametrize("s,t", CASES)
def test_oracle_builds_a_width_32_segment(s, t):
    oracle.build()
    keys = width32_keys(s, t)
    blob = oracle.compress(keys, EPS, 16)
    p = R.parse(blob)
    assert p["segments"] == 1 and int(p["seg_width"][0]) == 32 and int(p["seg_slope"][0]) > 0
    # the residual at t is exactly +eps: its zigzag code 2^31 has 32 bits
    res = R.residuals(p)
    assert max(max(int(r) for r in seg) for seg in res) == EPS
    assert [int(x) for x in R.reconstruct(p)] == [int(x) for x in keys]


@pytest.mark.gpu
@pytest.mark.parametrize("s,t", CASES)
def test_gpu_lower_bound_and_decode_at_width_32(s, t):
    import torch

    from paper_2412_10770_gb300 import build, lc

    build.build()
    oracle.build()
    lc.load()
    keys = width32_keys(s, t)
    col = lc.lc_compress(torch.from_numpy(keys).cuda(), eps=EPS)
    assert lc.lc_serialize(col) == oracle.compress(keys, EPS, 16)
    assert np.array_equal(lc.lc_decode(col).cpu().numpy(), keys)
    k = keys.astype(np.int64)
    mids = (k[:-1] + (k[1:] - k[:-1]) // 2)
    vals = np.unique(np.concatenate([k, k - 1, k + 1, mids, [0, int(k[-1]) + 5]])).astype(np.uint64)
    got = lc.lc_lower_bound(col, torch.from_numpy(vals).cuda()).cpu().numpy()
    want = np.searchsorted(keys, vals, side="left")
    assert np.array_equal(got.astype(np.int64), want.astype(np.int64))
    idx = np.arange(keys.size, dtype=np.uint64)
    assert np.array_equal(lc.lc_access(col, torch.from_numpy(idx).cuda()).cpu().numpy(), keys)
    assert lc.lc_status(col) == lc.LC_OK
    col.free()
