"""Both plans of a batch of random queries give the plain definitions (Def. 1
decoding; Sec. III-A lower_bound): out[q] = K[idx[q]] for access and the
first i with K[i] >= v[q] (numpy searchsorted) for lower_bound.

* direct: one query per thread in the caller's order;
* partitioned: queries sorted into key-range buckets, run bucket by bucket
  through the directories, results scattered back (forced here on small
  columns with at least 16 buckets, so that every bucket boundary, ragged
  tile and empty bucket case is reached);
* decoded: the column decoded whole first, then the same buckets answered
  from the decoded keys;
* the automatic choice (decoded for dense batches, partitioned for large
  sparse access batches on columns whose directories exceed L2, else
  direct), with the same results.
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


@pytest.fixture(autouse=True)
def _restore_plan():
    prev = lc.lc_set_query_plan(lc.LC_QUERIES_AUTO)
    yield
    lc.lc_set_query_plan(prev)


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


def _values(keys: np.ndarray, m: int, seed: int) -> np.ndarray:
    """m values: uniform over the key range, the keys themselves, keys - 1 and
    keys + 1, values below the first and above the last key."""
    rng = np.random.default_rng(seed)
    mx = np.iinfo(keys.dtype).max
    lo, hi = int(keys[0]), int(keys[-1])
    pool = np.concatenate([
        rng.integers(lo, hi, size=m, dtype=np.uint64, endpoint=True).astype(keys.dtype),
        keys[rng.integers(0, keys.size, size=m)],
        np.maximum(keys[rng.integers(0, keys.size, size=m)], 1) - 1,
        np.minimum(keys[rng.integers(0, keys.size, size=m)], mx - 1) + 1,
        np.array([0, lo, hi, mx], dtype=keys.dtype),
    ]).astype(keys.dtype)
    return pool[rng.permutation(pool.size)[:m]]


PLANS = (lc.LC_QUERIES_PARTITIONED, lc.LC_QUERIES_DECODED, lc.LC_QUERIES_DIRECT)


def _both_plans(col, keys, idx, vals):
    want_a = keys[idx.astype(np.int64)]
    want_l = np.searchsorted(keys, vals, side="left")
    for plan in PLANS:
        lc.lc_set_query_plan(plan)
        assert np.array_equal(host(lc.lc_access(col, dev(idx))), want_a), plan
        assert np.array_equal(host(lc.lc_lower_bound(col, dev(vals))), want_l), plan
        assert lc.lc_status(col) == lc.LC_OK


COLS = [("lognormal", np.uint64, 63), ("lognormal", np.uint32, 7), ("piecewise", np.uint64, 15),
        ("clusters", np.uint64, 1), ("uniform", np.uint32, 15)]


@pytest.mark.parametrize("gen,dt,eps", COLS)
@pytest.mark.parametrize("m", [1, 7, 4095, 3 * 4096 + 17, 300_000])
def test_partitioned_equals_definitions(gen, dt, eps, m):
    n = 700_000
    keys = inputs.column(gen, n, seed=inputs.seed_for(9, COLS.index((gen, dt, eps))), dtype=dt)
    col = lc.lc_compress(dev(keys), eps=eps)
    idx = inputs.uniform_ranks(m, n, seed=m)
    idx[: min(m, 2)] = [0, n - 1][: min(m, 2)]
    _both_plans(col, keys, idx, _values(keys, m, seed=m + 1))
    col.free()


@pytest.mark.parametrize("n", [1, 2, 17, 65536, 65537])
def test_partitioned_on_tiny_columns(n):
    """Fewer keys than buckets: empty buckets, repeated splitters."""
    keys = inputs.uniform_gaps(n, seed=n, dtype=np.uint64)
    col = lc.lc_compress(dev(keys), eps=3)
    idx = inputs.uniform_ranks(20_000, n, seed=1)
    _both_plans(col, keys, idx, _values(keys, 20_000, seed=2))
    col.free()


def test_partitioned_sorted_and_repeated_queries():
    """Every query in one bucket, and queries already in key order."""
    n = 500_000
    keys = inputs.column("lognormal", n, seed=5)
    col = lc.lc_compress(dev(keys), eps=15)
    same = np.full(100_000, 123_456, dtype=np.uint64)
    ordered = np.arange(0, n, 3, dtype=np.uint64)
    for idx in (same, ordered):
        _both_plans(col, keys, idx, keys[idx.astype(np.int64)])
    col.free()


def test_partitioned_out_of_range_indices():
    n = 300_000
    keys = inputs.column("piecewise", n, seed=6)
    col = lc.lc_compress(dev(keys), eps=15)
    idx = inputs.uniform_ranks(50_000, n, seed=3)
    bad = np.array([1, 77, 49_999])
    idx[bad] = [n, n + 12345, np.iinfo(np.uint64).max]
    want = np.where(idx < n, keys[np.minimum(idx, n - 1).astype(np.int64)], 0)
    for plan in (lc.LC_QUERIES_PARTITIONED, lc.LC_QUERIES_DECODED):
        lc.lc_set_query_plan(plan)
        assert np.array_equal(host(lc.lc_access(col, dev(idx))), want)
        assert lc.lc_status(col) == lc.LC_ERR_OUT_OF_RANGE
        assert lc.lc_status(col) == lc.LC_OK
    col.free()


def test_partitioned_list_mode_access():
    ids, begin = inputs.posting_lists(300, 400_000, 5_000_000, seed=8)
    col = lc.lc_compress_batch(dev(ids), begin, 7, 12)
    idx = inputs.uniform_ranks(100_000, ids.size, seed=4)
    for plan in PLANS:
        lc.lc_set_query_plan(plan)
        assert np.array_equal(host(lc.lc_access(col, dev(idx))), ids[idx.astype(np.int64)])
    col.free()


def _traced(fn):
    lc.lc_timing_read()
    lc.lc_timing_enable(True)
    try:
        out = fn()
        torch.cuda.synchronize()
    finally:
        lc.lc_timing_enable(False)
    return out, lc.lc_timing_read()


def test_auto_plans():
    """6e7 lognormal keys at eps 63 (about 2.8M segments: 105 MB of records
    and rank words): a dense access batch (8e6 queries, more than one per 8
    keys) runs decoded, a sparse large one (5e6) partitioned through the
    directories, a small one direct; lower_bound runs direct.  On a piecewise
    column (few segments) a dense access batch runs decoded too.  The plans
    show in the launch trace; every result is the definition."""
    n = 60_000_000
    keys = inputs.column("lognormal", n, seed=7)
    col = lc.lc_compress(dev(keys), eps=63)
    for m, want_acc in ((8_000_000, {"access.decode", "access.lookup"}), (5_000_000, {"access.lookup"}),
                        (1000, set())):
        idx = inputs.uniform_ranks(m, n, seed=9)
        vals = _values(keys, m, seed=10)
        got, names = _traced(lambda: host(lc.lc_access(col, dev(idx))))
        assert np.array_equal(got, keys[idx.astype(np.int64)])
        assert {k for k in names if k.startswith("access.")} >= want_acc, (m, sorted(names))
        assert ("access.decode" in names) == ("access.decode" in want_acc)
        assert ("access.lookup" in names) == ("access.lookup" in want_acc)
        got, names = _traced(lambda: host(lc.lc_lower_bound(col, dev(vals))))
        assert np.array_equal(got, np.searchsorted(keys, vals, side="left"))
        assert not any(k.startswith("lower_bound.") for k in names), (m, sorted(names))
    assert lc.lc_status(col) == lc.LC_OK
    col.free()
    few = inputs.column("piecewise", n, seed=8)
    col = lc.lc_compress(dev(few), eps=63)
    idx = inputs.uniform_ranks(8_000_000, n, seed=11)
    vals = _values(few, 8_000_000, seed=12)
    got, names = _traced(lambda: host(lc.lc_access(col, dev(idx))))
    assert np.array_equal(got, few[idx.astype(np.int64)])
    assert "access.decode" in names
    got, names = _traced(lambda: host(lc.lc_lower_bound(col, dev(vals))))
    assert np.array_equal(got, np.searchsorted(few, vals, side="left"))
    assert "lower_bound.lookup" not in names
    col.free()


def test_plan_setting():
    assert lc.lc_set_query_plan(lc.LC_QUERIES_DIRECT) == lc.LC_QUERIES_AUTO
    assert lc.lc_set_query_plan(lc.LC_QUERIES_PARTITIONED) == lc.LC_QUERIES_DIRECT
    assert lc.lc_set_query_plan(lc.LC_QUERIES_DECODED) == lc.LC_QUERIES_PARTITIONED
    for bad in (4, -1):
        with pytest.raises(lc.LcError) as e:
            lc.lc_set_query_plan(bad)
        assert e.value.code == lc.LC_ERR_INVALID_ARG
    assert lc.lc_set_query_plan(lc.LC_QUERIES_AUTO) == lc.LC_QUERIES_DECODED
