"""lc_decode_ranges_noalloc: the multi-range decode for callers that cannot
allocate device memory (a serving loop that must keep cudaMalloc/cudaFree and
their device synchronisation off its request path, or a host that owns all
device memory and hands libraries only its own buffers).

Called through the C ABI, it must write exactly what lc_decode_ranges writes,
on two calls in a row (the second call reuses the file-scope scratch that the
first one left behind), and it must refuse more ranges than its fixed scratch
holds.  The keys are integers, so "the same" means bit-identical.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2412_10770_gb300 import inputs, lc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_10770_gb300 import build

    build.build()
    lc.load()
    torch.cuda.set_device(0)


def _windows(n, m, max_len, seed):
    rng = np.random.default_rng(seed)
    cnt = rng.integers(0, max_len + 1, size=m).astype(np.uint64)
    beg = (rng.random(m) * (n - cnt + 1)).astype(np.uint64)
    off = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.uint64)
    return beg, cnt, off


@pytest.mark.parametrize("dt", [np.uint64, np.uint32])
def test_noalloc_matches_allocating_multi_range_decode(dt):
    n = 400_000
    keys = inputs.lognormal_gaps(n, seed=31, mu=1.5, sigma=1.0, dtype=dt)
    col = lc.lc_compress(torch.from_numpy(keys).cuda(), eps=15)
    for call in range(2):
        m = 3000 if call == 0 else 1200
        beg, cnt, off = _windows(n, m, 5000, seed=100 + call)
        b, c, o = (torch.from_numpy(a).cuda() for a in (beg, cnt, off))
        total = int(cnt.sum())
        want = torch.zeros(total, dtype=col.dtype, device="cuda")
        got = torch.full((total,), 7, dtype=torch.int64 if dt == np.uint64 else torch.int32, device="cuda").view(col.dtype)
        lc.lc_decode_ranges(col, b, c, o, want)
        lc.lc_decode_ranges_noalloc(col, b, c, o, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        ref = np.concatenate([keys[int(x):int(x) + int(k)] for x, k in zip(beg, cnt)])
        assert np.array_equal(got.cpu().numpy(), ref)
    assert lc.lc_status(col) == lc.LC_OK
    col.free()


def test_noalloc_at_its_limit_allocates_nothing():
    """m = LC_NOALLOC_MAX_RANGES (every scan tile of the fixed scratch in use):
    the same keys as lc_decode_ranges, and no growth of the device pool's
    high-water mark during the call (lc_decode_ranges, which allocates its work
    lists, does raise it: the check can see an allocation)."""
    n = 300_000
    keys = inputs.lognormal_gaps(n, seed=37, mu=1.0, sigma=1.0, dtype=np.uint64)
    col = lc.lc_compress(torch.from_numpy(keys).cuda(), eps=31)
    m = lc.LC_NOALLOC_MAX_RANGES
    beg, cnt, off = _windows(n, m, 40, seed=7)
    b, c, o = (torch.from_numpy(a).cuda() for a in (beg, cnt, off))
    total = int(cnt.sum())
    want = torch.zeros(total, dtype=col.dtype, device="cuda")
    got = torch.zeros(total, dtype=col.dtype, device="cuda")
    lc.lc_decode_ranges_noalloc(col, b, c, o, got)  # first call on the device: looks the scratch up
    torch.cuda.synchronize()
    got.zero_()
    torch.cuda.synchronize()
    base, _ = lc.lc_pool_usage(reset=True)
    lc.lc_decode_ranges_noalloc(col, b, c, o, got)
    torch.cuda.synchronize()
    _, high = lc.lc_pool_usage()
    assert high == base, f"the no-allocation call raised the pool's use from {base} to {high} bytes"
    lc.lc_pool_usage(reset=True)
    lc.lc_decode_ranges(col, b, c, o, want)
    torch.cuda.synchronize()
    _, high_alloc = lc.lc_pool_usage()
    assert high_alloc > base, "control: lc_decode_ranges allocates its work lists from the pool"
    assert torch.equal(got, want)
    ref = np.concatenate([keys[int(x):int(x) + int(k)] for x, k in zip(beg, cnt)])
    assert np.array_equal(got.cpu().numpy(), ref)
    assert lc.lc_status(col) == lc.LC_OK
    col.free()


def test_noalloc_skips_a_range_past_the_output():
    """A range whose output would end past out's capacity is skipped and
    reported in the status word; the ranges before it are still decoded."""
    n = 50_000
    keys = inputs.uniform_gaps(n, seed=5, dtype=np.uint64)
    col = lc.lc_compress(torch.from_numpy(keys).cuda(), eps=7)
    beg = np.array([10, 2000, 30000], dtype=np.uint64)
    cnt = np.array([100, 300, 500], dtype=np.uint64)
    off = np.array([0, 100, 400], dtype=np.uint64)  # the last range needs 900 keys of output
    b, c, o = (torch.from_numpy(a).cuda() for a in (beg, cnt, off))
    out = torch.zeros(600, dtype=col.dtype, device="cuda")
    lc.lc_decode_ranges_noalloc(col, b, c, o, out)
    assert lc.lc_status(col) == lc.LC_ERR_OUT_OF_RANGE
    h = out.cpu().numpy()
    assert np.array_equal(h[:100], keys[10:110]) and np.array_equal(h[100:400], keys[2000:2300])
    assert not h[400:].any()
    col.free()


def test_noalloc_refuses_more_ranges_than_its_scratch_holds():
    keys = inputs.uniform_gaps(10_000, seed=3, dtype=np.uint64)
    col = lc.lc_compress(torch.from_numpy(keys).cuda(), eps=7)
    m = lc.LC_NOALLOC_MAX_RANGES + 1
    z = torch.zeros(m, dtype=torch.uint64, device="cuda")
    out = torch.zeros(1, dtype=torch.uint64, device="cuda")
    with pytest.raises(lc.LcError) as e:
        lc.lc_decode_ranges_noalloc(col, z, z, z, out)
    assert e.value.code == lc.LC_ERR_INVALID_ARG
    col.free()
