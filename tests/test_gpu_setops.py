"""GPU parity of posting-list AND / OR over compressed lists (Sec. III-A,
Fig. 4) through the C ABI: lc_intersect and lc_union equal the plain set
intersection and union of the decoded keys (numpy), for whole columns and for
lists of list-mode columns, with short-vs-long, disjoint, identical, empty and
duplicate-key cases."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _ids(rng, n, universe, dt=np.uint32):
    return np.sort(rng.choice(universe, size=n, replace=False)).astype(dt)


PAIRS = [(10, 100_000), (5000, 5000), (70_000, 300_000), (1, 1), (300_000, 17), (40_000, 0)]


@pytest.mark.parametrize("na,nb", PAIRS)
@pytest.mark.parametrize("eps", [0, 15, 255])
def test_and_or_single_columns(na, nb, eps):
    rng = np.random.default_rng(na * 7 + nb + eps)
    universe = 2_000_000
    a, b = _ids(rng, na, universe), _ids(rng, nb, universe)
    ca, cb = lc.lc_compress(dev(a), eps=eps), lc.lc_compress(dev(b), eps=eps)
    assert np.array_equal(lc.lc_intersect(ca, cb).cpu().numpy(), np.intersect1d(a, b))
    assert np.array_equal(lc.lc_union(ca, cb).cpu().numpy(), np.union1d(a, b))
    ca.free()
    cb.free()


def test_and_or_uint64_duplicates_and_identical():
    rng = np.random.default_rng(9)
    a = np.sort(rng.integers(0, 1 << 62, size=50_000, dtype=np.uint64))
    a = np.repeat(a, rng.integers(1, 3, size=a.size))  # non-decreasing with repeats
    b = np.sort(np.concatenate([a[::3], rng.integers(0, 1 << 62, size=20_000, dtype=np.uint64)]))
    ca, cb = lc.lc_compress(dev(a), eps=7), lc.lc_compress(dev(b), eps=31)
    assert np.array_equal(lc.lc_intersect(ca, cb).cpu().numpy(), np.intersect1d(a, b))
    assert np.array_equal(lc.lc_union(ca, cb).cpu().numpy(), np.union1d(a, b))
    assert np.array_equal(lc.lc_intersect(ca, ca).cpu().numpy(), np.unique(a))
    ca.free()
    cb.free()


def test_and_or_lists_of_batch_columns():
    ids, begin = inputs.posting_lists(400, 600_000, 5 * 10**6, seed=21)
    col = lc.lc_compress_batch(dev(ids), begin, 15, 16)
    other_ids, other_begin = inputs.posting_lists(50, 200_000, 5 * 10**6, seed=22)
    col2 = lc.lc_compress_batch(dev(other_ids), other_begin, 63, 12)
    rng = np.random.default_rng(4)
    for _ in range(25):
        la, lb = int(rng.integers(0, 400)), int(rng.integers(0, 50))
        x = ids[begin[la]:begin[la + 1]]
        y = other_ids[other_begin[lb]:other_begin[lb + 1]]
        assert np.array_equal(lc.lc_intersect(col, col2, la, lb).cpu().numpy(), np.intersect1d(x, y))
        assert np.array_equal(lc.lc_union(col, col2, la, lb).cpu().numpy(), np.union1d(x, y))
        la2 = int(rng.integers(0, 400))
        z = ids[begin[la2]:begin[la2 + 1]]
        assert np.array_equal(lc.lc_intersect(col, col, la, la2).cpu().numpy(), np.intersect1d(x, z))
    with pytest.raises(lc.LcError):
        lc.lc_intersect(col, col2, 400, 0)
    with pytest.raises(lc.LcError):
        lc.lc_intersect(col, col2, -1, 0)
    col.free()
    col2.free()


def test_capacity_too_small_reports_the_length():
    a = np.arange(0, 1000, 2, dtype=np.uint32)
    b = np.arange(0, 1000, 3, dtype=np.uint32)
    ca, cb = lc.lc_compress(dev(a)), lc.lc_compress(dev(b))
    out = torch.empty(3, dtype=torch.uint32, device="cuda")
    with pytest.raises(lc.LcError) as e:
        lc.lc_intersect(ca, cb, out=out)
    assert e.value.code == lc.LC_ERR_INVALID_ARG
    ca.free()
    cb.free()
