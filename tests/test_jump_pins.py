"""Pins of the oracle's jump fit (fewest anchored segments, Sec. II-A's
objective; lco_compress_jump): on inputs whose segments are all short it
reaches the true anchored optimum, found by a dynamic program over every
segmentation with feasibility re-derived by bisection on Def. 2; every slope
is the floor midpoint of its segment's exact feasible interval; the bytes
decode exactly with the eps bound; no chunk has more segments than the
greedy's.  No GPU."""
from __future__ import annotations

import numpy as np
import pytest

import lcf_reader as R
import oracle
from paper_2412_10770_gb300 import inputs
from test_oracle_pins import _anchored_optimum, _feasible_interval, check_invariants


def _jump_cases():
    rng = np.random.default_rng(5)
    cases = []
    for trial in range(100):
        n = int(rng.integers(6, 40))
        g = rng.integers(0, [40, 6, 200, 3, 1000][trial % 5], size=n)
        cases.append(([int(x) for x in np.cumsum(g)], int([0, 1, 2, 4, 7][trial % 5])))
    return cases


def check_jump(keys, eps, blob):
    """Every segment feasible, its slope the floor midpoint of its exact
    feasible interval; segments tile each chunk."""
    p = R.parse(blob)
    for j, (c, s, n) in enumerate(R.segments(p)):
        M = int(p["seg_slope"][j])
        assert int(p["seg_icpt"][j]) == keys[s]
        if n == 1:
            assert M == 0
        else:
            iv = _feasible_interval(keys[s:s + n], eps)
            assert iv is not None and M == iv[0] + (iv[1] - iv[0]) // 2


@pytest.mark.parametrize("case", range(100))
def test_jump_reaches_the_anchored_optimum_on_short_segments(case):
    keys, eps = _jump_cases()[case]
    blob = oracle.compress_jump(np.array(keys, dtype=np.uint64), eps, 8)
    assert R.parse(blob)["segments"] == _anchored_optimum(keys, eps)
    check_jump(keys, eps, blob)
    check_invariants(keys, eps, blob)


def test_the_optimum_is_sometimes_below_the_greedy():
    """The pins above have teeth: on these inputs the greedy is not optimal."""
    worse = 0
    for keys, eps in _jump_cases():
        g = R.parse(oracle.compress(np.array(keys, dtype=np.uint64), eps, 8))["segments"]
        worse += g > _anchored_optimum(keys, eps)
    assert worse >= 3


@pytest.mark.parametrize("kind,eps", [("lognormal", 63), ("lognormal", 255), ("uniform", 15), ("clusters", 1)])
def test_jump_columns_roundtrip_and_never_exceed_the_greedy_per_chunk(kind, eps):
    keys = inputs.column(kind, 150_000, seed=31, dtype=np.uint64)
    gj, gg = R.parse(oracle.compress_jump(keys, eps, 14)), R.parse(oracle.compress(keys, eps, 14))
    assert np.array_equal(oracle.decode(oracle.compress_jump(keys, eps, 14)), keys)
    cj, cg = np.diff(gj["chunk_seg_begin"]), np.diff(gg["chunk_seg_begin"])
    assert np.all(cj <= cg)
    for r in R.residuals(gj):
        assert all(-eps <= x <= eps for x in r)
