"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's formulas: the segment slopes and
boundaries are re-derived by bisection on the definition |K[i] - floor(f(i))|
<= eps (Def. 2), decoding is redone by an independent reader, sizes come from
the closed form of Sec. II-A, and queries are compared with numpy's own
searchsorted / indexing (Def. 1).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import lcf_reader as R
import oracle
from paper_2412_10770_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
I64_MIN, I64_MAX = -(1 << 63), (1 << 63) - 1


# ---------------------------------------------------------------- helpers

def _feasible_interval(keys, eps):
    """Integer Q32 slopes M with |K[s+t] - (K[s] + floor(M t / 2^32))| <= eps for
    every key of the run, found by bisection on the definition (Def. 2).
    Returns (LO, HI) or None when no int64 slope fits."""
    k0 = int(keys[0])
    D = [int(k) - k0 for k in keys]
    n = len(keys)

    def ok_lo(M):  # every prediction high enough
        return all(((M * t) >> 32) >= D[t] - eps for t in range(1, n))

    def ok_hi(M):  # every prediction low enough
        return all(((M * t) >> 32) <= D[t] + eps for t in range(1, n))

    if not ok_lo(I64_MAX) or not ok_hi(I64_MIN):
        return None
    a, b = I64_MIN, I64_MAX  # smallest M with ok_lo
    while a < b:
        m = (a + b) // 2
        if ok_lo(m):
            b = m
        else:
            a = m + 1
    lo = a
    a, b = I64_MIN, I64_MAX  # largest M with ok_hi
    while a < b:
        m = (a + b + 1) // 2
        if ok_hi(m):
            a = m
        else:
            b = m - 1
    hi = a
    return (lo, hi) if lo <= hi else None


def _chunk_bounds(p):
    ckb = p["chunk_key_begin"]
    return [(int(ckb[c]), int(ckb[c + 1])) for c in range(p["chunks"])]


def check_greedy(keys, eps, blob):
    """The segmentation is the greedy one: chained from each chunk start, every
    segment feasible with its slope the floor midpoint of its exact feasible
    interval, and maximal (the next key of the chunk cannot join)."""
    p = R.parse(blob)
    keys = [int(k) for k in keys]
    segs = R.segments(p)
    bounds = _chunk_bounds(p)
    by_chunk = {}
    for j, (c, s, n) in enumerate(segs):
        by_chunk.setdefault(c, []).append((j, s, n))
    for c, (a, b) in enumerate(bounds):
        pos = a
        for j, s, n in by_chunk[c]:
            assert s == pos
            pos += n
            M = int(p["seg_slope"][j])
            assert int(p["seg_icpt"][j]) == keys[s]
            if n == 1:
                assert M == 0
            else:
                iv = _feasible_interval(keys[s:s + n], eps)
                assert iv is not None
                lo, hi = iv
                assert M == lo + (hi - lo) // 2
            if s + n < b:
                assert _feasible_interval(keys[s:s + n + 1], eps) is None
        assert pos == b


def check_invariants(keys, eps, blob):
    """Def. 1 roundtrip, Def. 2 error bound, Sec. II-A width bound and size."""
    p = R.parse(blob)
    assert p["n"] == len(keys)
    rec = R.reconstruct(p)
    assert rec == [int(k) for k in keys]
    bound = math.ceil(math.log2(2 * eps + 1)) if eps > 0 else 0
    for r in R.residuals(p):
        assert all(-eps <= x <= eps for x in r)
    assert all(int(w) <= bound for w in p["seg_width"])
    assert R.closed_form_size(p) == len(blob)


def _size_formula(kb, C, L, W):
    pad = lambda x: (x + 15) // 16 * 16  # noqa: E731
    return 64 + 3 * pad(8 * (C + 1)) + pad(kb * L) + pad(8 * L) + pad(4 * L) + pad(2 * L) + pad(L) + 8 * W


# ---------------------------------------------------------------- tiny inputs

def _tiny_cases():
    rng = np.random.default_rng(7)
    cases = []
    for trial in range(60):
        n = int(rng.integers(1, 40))
        kind = trial % 4
        if kind == 0:
            g = rng.integers(0, 64, size=n)
        elif kind == 1:
            g = rng.integers(0, 4, size=n)
        elif kind == 2:
            g = np.where(rng.random(n) < 0.1, rng.integers(0, 1 << 40, size=n), rng.integers(0, 9, size=n))
        else:
            g = rng.geometric(0.05, size=n)
        k = np.cumsum(g).astype(np.uint64)
        eps = int([0, 1, 2, 4, 15][trial % 5])
        cases.append((k, eps))
    return cases


@pytest.mark.parametrize("case", range(60))
def test_greedy_matches_definition_on_tiny_inputs(case):
    keys, eps = _tiny_cases()[case]
    for log2 in (8,):
        blob = oracle.compress(keys, eps, log2)
        check_greedy(keys, eps, blob)
        check_invariants(keys, eps, blob)


def test_greedy_chunk_restart_and_ragged_tail():
    keys = inputs.uniform_gaps(700, seed=3, dtype=np.uint64)  # 3 chunks of 256, last ragged
    for eps in (0, 3, 15):
        blob = oracle.compress(keys, eps, 8)
        p = R.parse(blob)
        assert p["chunks"] == 3
        assert [int(x) for x in p["chunk_key_begin"]] == [0, 256, 512, 700]
        check_greedy(keys, eps, blob)
        check_invariants(keys, eps, blob)


def test_hypothesis_properties():
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(st.lists(st.integers(0, 200), min_size=0, max_size=60),
               st.sampled_from([0, 1, 2, 5, 31]), st.integers(0, (1 << 63)))
    def prop(gaps, eps, base):
        keys = (base + np.cumsum(np.array(gaps, dtype=np.uint64))).astype(np.uint64) if gaps else np.zeros(0, np.uint64)
        blob = oracle.compress(keys, eps, 8)
        check_invariants(keys, eps, blob)
        check_greedy(keys, eps, blob)
        assert np.array_equal(oracle.decode(blob), keys)

    prop()


def _anchored_optimum(keys, eps):
    """Fewest anchored segments covering keys (dynamic programming over every
    feasible run, feasibility by bisection)."""
    n = len(keys)
    best = [0] + [None] * n
    for e in range(1, n + 1):
        for s in range(e):
            if best[s] is None:
                continue
            if e - s == 1 or _feasible_interval(keys[s:e], eps) is not None:
                if best[e] is None or best[s] + 1 < best[e]:
                    best[e] = best[s] + 1
    return best[n]


def test_greedy_never_beats_anchored_optimum():
    rng = np.random.default_rng(11)
    for trial in range(25):
        n = int(rng.integers(2, 24))
        keys = [int(x) for x in np.cumsum(rng.integers(0, 40, size=n))]
        eps = int([0, 1, 2, 4][trial % 4])
        blob = oracle.compress(np.array(keys, dtype=np.uint64), eps, 8)
        L = R.parse(blob)["segments"]
        opt = _anchored_optimum(keys, eps)
        assert opt <= L


# ---------------------------------------------------------------- paper values

def test_width_formula_values_printed_in_paper():
    """ceil(log2(2 eps + 1)) bits per residual (Sec. I, Sec. II-A; Fig. 2 prints
    eps = 4 -> 4 bits) bounds every segment width the encoder picks."""
    g = json.load(open(os.path.join(HERE, "golden", "fig2_toy_example.json")))
    for eps, bits in zip(g["width_formula"]["eps"], g["width_formula"]["bits"]):
        assert (math.ceil(math.log2(2 * eps + 1)) if eps else 0) == bits
        if eps > 1 << 20:
            continue
        for seed in range(3):
            keys = inputs.lognormal_gaps(3000, seed=seed, mu=math.log(eps + 2), sigma=1.0)
            blob = oracle.compress(keys, eps, 8)
            assert max(int(w) for w in R.parse(blob)["seg_width"]) <= bits


def test_fig2_toy_example_segments():
    """Fig. 2: eps = 4 gives 3 segments over indices [0,5], [6,9], [10,20] and
    4-bit residual codes."""
    g = json.load(open(os.path.join(HERE, "golden", "fig2_toy_example.json")))
    pr = g["printed"]
    keys = np.array(g["keys_consistent"], dtype=np.uint32)
    assert len(keys) == pr["n_keys"] and list(keys[:2]) == pr["keys_first"] and keys[-1] == pr["key_last"]
    blob = oracle.compress(keys, pr["eps"], 8)
    p = R.parse(blob)
    got = [[s, s + n - 1] for _, s, n in R.segments(p)]
    assert got == pr["segments_inclusive"]
    assert max(int(w) for w in p["seg_width"]) <= pr["bits_per_residual"]
    assert math.ceil(math.log2(2 * pr["eps"] + 1)) == pr["bits_per_residual"]
    check_greedy(keys, pr["eps"], blob)
    check_invariants(keys, pr["eps"], blob)


def test_width_is_bit_length_of_largest_zigzag_code():
    for eps in (1, 4, 15, 255):
        keys = inputs.uniform_gaps(2000, seed=eps, dtype=np.uint64, gap_hi=4 * eps + 4)
        blob = oracle.compress(keys, eps, 8)
        p = R.parse(blob)
        res = R.residuals(p)
        widths = [int(w) for w in p["seg_width"]]
        for r, w in zip(res, widths):
            zmax = max((2 * x if x >= 0 else -2 * x - 1) for x in r)
            assert w == zmax.bit_length()
        assert max(widths) <= math.ceil(math.log2(2 * eps + 1))


# ---------------------------------------------------------------- special cases

@pytest.mark.parametrize("kb", [4, 8])
def test_arithmetic_progression_is_one_segment_per_chunk(kb):
    n = 3 * 65536 + 123
    g = 7 if kb == 4 else (1 << 30) + 12345
    dt = np.uint32 if kb == 4 else np.uint64
    keys = (5 + g * np.arange(n, dtype=np.uint64)).astype(dt)
    blob = oracle.compress(keys, 0, 16)
    p = R.parse(blob)
    assert p["segments"] == p["chunks"] == 4
    assert all(int(w) == 0 for w in p["seg_width"]) and p["words"] == 0
    assert len(blob) == _size_formula(kb, 4, 4, 0)
    assert np.array_equal(oracle.decode(blob), keys)


def test_constant_keys_have_zero_width():
    keys = np.full(1000, 123456789, dtype=np.uint64)
    for eps in (0, 1, 100):
        p = R.parse(oracle.compress(keys, eps, 8))
        assert all(int(w) == 0 for w in p["seg_width"]) and p["words"] == 0
        assert p["segments"] == p["chunks"]


def test_eps_at_least_key_span_is_one_segment_per_chunk():
    keys = inputs.uniform_gaps(5000, seed=5, dtype=np.uint64)
    span = int(keys[-1] - keys[0])
    blob = oracle.compress(keys, span, 8)
    p = R.parse(blob)
    assert p["segments"] == p["chunks"]
    check_invariants(keys, span, blob)


def test_eps_zero_pairs_always_fit():
    keys = inputs.lognormal_gaps(20000, seed=9)
    blob = oracle.compress(keys, 0, 8)
    p = R.parse(blob)
    ckb, csb = p["chunk_key_begin"], p["chunk_seg_begin"]
    for c in range(p["chunks"]):
        n_c = int(ckb[c + 1] - ckb[c])
        assert int(csb[c + 1] - csb[c]) <= (n_c + 1) // 2
    assert all(int(w) == 0 for w in p["seg_width"])  # eps = 0: exact lines


def test_huge_gaps_start_singleton_segments():
    # slope above 2^31 per index cannot be held by an int64 Q32 slope
    keys = np.array([0, 1 << 40, 1 << 41, (1 << 41) + 1, (1 << 41) + 2, (1 << 63) + 5,
                     (1 << 64) - 2, (1 << 64) - 1], dtype=np.uint64)
    blob = oracle.compress(keys, 1, 8)
    p = R.parse(blob)
    got = [(s, n) for _, s, n in R.segments(p)]
    assert got[0] == (0, 1) and got[1] == (1, 1)
    assert np.array_equal(oracle.decode(blob), keys)
    check_greedy(keys, 1, blob)
    check_invariants(keys, 1, blob)


@pytest.mark.parametrize("n", [0, 1, 2, 255, 256, 257, 511, 65535, 65536, 65537])
def test_edge_sizes_roundtrip(n):
    for kb, dt in ((4, np.uint32), (8, np.uint64)):
        keys = inputs.uniform_gaps(n, seed=n + 1, dtype=dt)
        for log2 in (8, 16):
            blob = oracle.compress(keys, 15, log2)
            p = R.parse(blob)
            assert p["chunks"] == -(-n // (1 << log2))
            assert R.closed_form_size(p) == len(blob)
            assert np.array_equal(oracle.decode(blob), keys)
            if n:
                ix = np.array([0, n - 1, n // 2], dtype=np.uint64)
                assert np.array_equal(oracle.access(blob, ix), keys[ix.astype(np.int64)])


def test_empty_column_is_header_and_directory_only():
    blob = oracle.compress(np.zeros(0, np.uint64), 3, 16)
    assert len(blob) == _size_formula(8, 0, 0, 0) == 112
    assert oracle.decode(blob).size == 0
    assert oracle.lower_bound(blob, np.array([5], np.uint64))[0] == 0


# ---------------------------------------------------------------- generators at moderate size

GEN_CASES = [("uniform", np.uint32, 15), ("lognormal", np.uint64, 1), ("lognormal", np.uint64, 63),
             ("piecewise", np.uint64, 1), ("piecewise", np.uint64, 15), ("clusters", np.uint64, 15),
             ("clusters", np.uint64, 255)]


@pytest.mark.parametrize("kind,dt,eps", GEN_CASES)
def test_generators_roundtrip_and_queries(kind, dt, eps):
    n = 3 * 65536 + 777
    keys = inputs.column(kind, n, seed=inputs.seed_for(2, 1), dtype=dt)
    blob = oracle.compress(keys, eps, 16)
    p = R.parse(blob)
    assert R.closed_form_size(p) == len(blob)
    assert np.array_equal(oracle.decode(blob), keys)
    ix = inputs.uniform_ranks(5000, n, seed=1)
    assert np.array_equal(oracle.access(blob, ix), keys[ix.astype(np.int64)])
    q = inputs.uniform_values(5000, int(keys[0]), int(keys[-1]), seed=2, dtype=dt)
    q = np.concatenate([q, keys[:50], np.array([0, keys[-1], np.iinfo(dt).max], dtype=dt)])
    assert np.array_equal(oracle.lower_bound(blob, q), np.searchsorted(keys, q, side="left"))
    # widths bounded by the paper's ceil(log2(2 eps + 1))
    bound = math.ceil(math.log2(2 * eps + 1))
    assert int(p["seg_width"].max()) <= bound


def test_duplicates_lower_bound_returns_first_index():
    keys = np.repeat(np.arange(0, 4000, 7, dtype=np.uint64), 5)
    blob = oracle.compress(keys, 2, 8)
    q = np.arange(0, 4010, dtype=np.uint64)
    assert np.array_equal(oracle.lower_bound(blob, q), np.searchsorted(keys, q, side="left"))


# ---------------------------------------------------------------- list mode

def test_list_mode_each_list_is_its_own_column():
    rng = np.random.default_rng(3)
    lens = [0, 1, 17, 300, 1000, 0, 2049]
    lists = [np.sort(rng.choice(100000, size=k, replace=False)).astype(np.uint32) for k in lens]
    keys = np.concatenate(lists)
    begin = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    eps = [1, 3, 15, 0, 63, 2, 7]
    log2 = [8, 8, 9, 8, 10, 16, 8]
    blob = oracle.compress_lists(keys, begin, eps, log2)
    assert np.array_equal(oracle.decode(blob), keys)
    p = R.parse(blob)
    assert p["list_mode"] and p["lists"] == len(lens)
    assert R.closed_form_size(p) == len(blob)
    assert R.reconstruct(p) == [int(k) for k in keys]
    # each list's segments and payload equal those of the list compressed alone
    for l, arr in enumerate(lists):
        if arr.size == 0:
            continue
        q = R.parse(oracle.compress(arr, eps[l], log2[l]))
        c0, c1 = int(p["list_chunk_begin"][l]), int(p["list_chunk_begin"][l + 1])
        s0, s1 = int(p["chunk_seg_begin"][c0]), int(p["chunk_seg_begin"][c1])
        w0, w1 = int(p["chunk_word_begin"][c0]), int(p["chunk_word_begin"][c1])
        assert np.array_equal(p["seg_slope"][s0:s1], q["seg_slope"])
        assert np.array_equal(p["seg_start"][s0:s1], q["seg_start"])
        assert np.array_equal(p["seg_width"][s0:s1], q["seg_width"])
        assert np.array_equal(p["payload"][w0:w1], q["payload"])
    with pytest.raises(oracle.OracleError):
        oracle.lower_bound(blob, np.array([1], np.uint32))


# ---------------------------------------------------------------- error handling

def test_invalid_arguments_and_unsorted_input():
    k = np.arange(10, dtype=np.uint64)
    for eps, lg in ((1 << 30, 7), ((1 << 30) + 1, 16), (0, 17)):
        with pytest.raises(oracle.OracleError) as e:
            oracle.compress(k, eps, lg)
        assert e.value.code == -1
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(np.array([3, 2], np.uint64), 1, 16)
    assert e.value.code == -2
    blob = oracle.compress(k, 1, 16)
    with pytest.raises(oracle.OracleError) as e:
        oracle.access(blob, np.array([10], np.uint64))
    assert e.value.code == -3


def test_corrupt_blobs_are_rejected():
    keys = inputs.uniform_gaps(3000, seed=1, dtype=np.uint64)
    blob = oracle.compress(keys, 15, 8)
    p = R.parse(blob)
    offs, _ = R.layout(8, p["chunks"], p["segments"], p["words"], 0, False)
    bad = [blob[:-16], blob + b"\0" * 16, b"LCF2" + blob[4:]]
    ba = bytearray(blob); ba[offs["seg_width"][0]] = 40; bad.append(bytes(ba))
    ba = bytearray(blob); ba[offs["chunk_seg_begin"][0] + 8] ^= 1; bad.append(bytes(ba))
    ba = bytearray(blob); ba[offs["seg_start"][0] + 2] = 0; ba[offs["seg_start"][0] + 3] = 0; bad.append(bytes(ba))
    ba = bytearray(blob); ba[offs["seg_bitoff"][0] + 4] ^= 1; bad.append(bytes(ba))
    ba = bytearray(blob); ba[-1] |= 0x80; bad.append(bytes(ba))  # a pad bit set
    for b in bad:
        with pytest.raises(oracle.OracleError) as e:
            oracle.decode(b)
        assert e.value.code == -5
