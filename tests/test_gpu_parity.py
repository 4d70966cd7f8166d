"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

* compress: the serialized K^c is byte-identical to the oracle's (integer work:
  bit-exact, no tolerance);
* decode / access / lower_bound: identical to the raw keys, indexing and
  numpy searchsorted (Def. 1's plain definitions);
* deserialize: an oracle-written blob decodes on the GPU;
* list mode, edge sizes, ragged tails, error paths.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import lcf_reader as R
import oracle
from paper_2412_10770_gb300 import inputs, lc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_10770_gb300 import build

    build.build()
    oracle.build()
    lc.load()
    torch.cuda.set_device(0)


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


def check_column(keys: np.ndarray, eps: int, log2: int, nq: int = 3000):
    col = lc.lc_compress(dev(keys), eps=eps, chunk_log2=log2)
    blob = lc.lc_serialize(col)
    ref = oracle.compress(keys, eps, log2)
    if blob != ref:
        p, q = R.parse(blob), R.parse(ref)
        for nm in ("chunk_seg_begin", "chunk_word_begin", "seg_start", "seg_slope", "seg_width", "seg_bitoff",
                   "seg_icpt", "payload"):
            a, b = p.get(nm), q.get(nm)
            if a is None or b is None or a.shape != b.shape or not np.array_equal(a, b):
                raise AssertionError(f"K^c differs from the oracle first in {nm}")
        raise AssertionError("K^c differs from the oracle (header or padding)")
    n = keys.size
    assert lc.lc_size(col) == len(ref)
    assert abs(lc.lc_ratio(col) - (len(ref) / (n * keys.itemsize) if n else 0.0)) < 1e-12
    assert np.array_equal(host(lc.lc_decode(col)), keys)
    if n:
        rng = np.random.default_rng(n)
        for _ in range(4):
            b = int(rng.integers(0, n))
            c = int(rng.integers(0, n - b + 1))
            assert np.array_equal(host(lc.lc_decode(col, b, c)), keys[b:b + c])
        idx = inputs.uniform_ranks(nq, n, seed=3)
        idx = np.concatenate([idx, np.array([0, n - 1], dtype=np.uint64)])
        assert np.array_equal(host(lc.lc_access(col, dev(idx))), keys[idx.astype(np.int64)])
        q = inputs.uniform_values(nq, int(keys[0]), int(keys[-1]), seed=4, dtype=keys.dtype)
        q = np.concatenate([q, keys[: min(n, 64)], np.array([0, keys[-1], np.iinfo(keys.dtype).max], keys.dtype)])
        assert np.array_equal(host(lc.lc_lower_bound(col, dev(q))), np.searchsorted(keys, q, side="left"))
    assert lc.lc_status(col) == lc.LC_OK
    return col


CASES = [
    ("uniform", np.uint32, 15, 16), ("uniform", np.uint32, 0, 8), ("uniform", np.uint64, 3, 12),
    ("lognormal", np.uint64, 1, 16), ("lognormal", np.uint64, 15, 16), ("lognormal", np.uint64, 63, 16),
    ("lognormal", np.uint64, 255, 16), ("piecewise", np.uint64, 1, 16), ("piecewise", np.uint64, 15, 16),
    ("piecewise", np.uint64, 255, 16), ("clusters", np.uint64, 1, 16), ("clusters", np.uint64, 15, 16),
    ("clusters", np.uint64, 63, 10), ("lognormal", np.uint32, 7, 9),
]


@pytest.mark.parametrize("kind,dt,eps,log2", CASES)
def test_compress_matches_oracle_and_queries_match_keys(kind, dt, eps, log2):
    n = 3 * 65536 + 5003  # several chunks and tiles, ragged last chunk and tile
    keys = inputs.column(kind, n, seed=inputs.seed_for(2, hash(kind) % 7), dtype=dt)
    if dt == np.uint32 and kind == "lognormal":
        keys = inputs.lognormal_gaps(n, seed=5, mu=1.0, sigma=1.0, dtype=np.uint32)
    check_column(keys, eps, log2).free()


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 63, 64, 65, 255, 256, 257, 2047, 2048, 2049, 65535, 65536, 65537])
def test_edge_sizes(n):
    for dt in (np.uint32, np.uint64):
        keys = inputs.uniform_gaps(n, seed=n, dtype=dt)
        check_column(keys, 5, 16, nq=200).free()
        check_column(keys, 5, 8, nq=200).free()


def test_empty_column():
    col = lc.lc_compress(torch.empty(0, dtype=torch.uint64, device="cuda"), eps=4)
    assert lc.lc_serialize(col) == oracle.compress(np.zeros(0, np.uint64), 4, 16)
    assert lc.lc_decode(col).numel() == 0
    assert lc.lc_ratio(col) == 0.0
    col.free()


def test_special_shapes():
    n = 2 * 65536 + 99
    ap = (7 + 12345 * np.arange(n, dtype=np.uint64)).astype(np.uint64)
    check_column(ap, 0, 16).free()  # one segment per chunk, no payload
    const = np.full(n, (1 << 63) + 5, dtype=np.uint64)
    check_column(const, 2, 16).free()
    dup = np.repeat(np.arange(0, n // 7 + 1, dtype=np.uint64) * 3, 7)[:n]
    check_column(dup, 1, 16).free()
    # huge gaps force single-key segments; keys near 2^64 - 1
    rng = np.random.default_rng(1)
    g = rng.integers(1 << 40, 1 << 44, size=5000, dtype=np.uint64)
    big = np.cumsum(g, dtype=np.uint64) + np.uint64((1 << 64) - (1 << 58))
    big.sort()
    check_column(big, 1, 8).free()
    # eps at its maximum
    check_column(inputs.lognormal_gaps(70000, seed=3), 1 << 30, 16).free()


def test_long_segments_spanning_blocks_and_runs():
    # one straight line per chunk: the fitter's warp walk covers whole chunks
    n = 4 * 65536
    keys = (1000 + (np.arange(n, dtype=np.uint64) * 37) // 3).astype(np.uint64)
    check_column(keys, 1, 16).free()
    # medium segments around the speculation cap
    rng = np.random.default_rng(5)
    parts = []
    base = 0
    while sum(p.size for p in parts) < n:
        m = int(rng.integers(40, 400))
        s = int(rng.integers(1, 1000))
        parts.append(base + s * np.arange(m, dtype=np.uint64) + rng.integers(0, 3, m).astype(np.uint64))
        base = int(parts[-1][-1]) + int(rng.integers(10**5, 10**6))
    keys = np.sort(np.concatenate(parts)[:n]).astype(np.uint64)
    check_column(keys, 2, 16).free()


def test_deserialize_oracle_blob_and_roundtrip():
    keys = inputs.piecewise_linear(150000, seed=11)
    ref = oracle.compress(keys, 7, 14)
    col = lc.lc_deserialize(ref)
    assert np.array_equal(host(lc.lc_decode(col)), keys)
    assert lc.lc_serialize(col) == ref
    idx = inputs.uniform_ranks(1000, keys.size, seed=2)
    assert np.array_equal(host(lc.lc_access(col, dev(idx))), keys[idx.astype(np.int64)])
    col.free()


def test_deserialize_rejects_corrupt_blobs():
    keys = inputs.uniform_gaps(5000, seed=1, dtype=np.uint64)
    ref = oracle.compress(keys, 15, 8)
    p = R.parse(ref)
    offs, _ = R.layout(8, p["chunks"], p["segments"], p["words"], 0, False)
    bad = [ref[:-16], b"LCF0" + ref[4:]]
    ba = bytearray(ref); ba[offs["seg_width"][0] + 3] = 33; bad.append(bytes(ba))
    ba = bytearray(ref); ba[offs["chunk_word_begin"][0] + 8] += 2; bad.append(bytes(ba))
    ba = bytearray(ref); ba[offs["seg_start"][0]] = 1; bad.append(bytes(ba))
    ba = bytearray(ref); ba[offs["seg_icpt"][0] + 8 * p["segments"]] = 1; bad.append(bytes(ba))  # a pad byte
    for b in bad:
        with pytest.raises(lc.LcError) as e:
            lc.lc_deserialize(b)
        assert e.value.code == lc.LC_ERR_CORRUPT


def test_list_mode_matches_oracle():
    rng = np.random.default_rng(9)
    lens = [0, 1, 5, 16, 300, 4000, 70000, 0, 1000, 2]
    lists = [np.sort(rng.choice(5 * 10**7, size=k, replace=False)).astype(np.uint32) for k in lens]
    ids = np.concatenate(lists)
    begin = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    eps = [1, 3, 15, 0, 63, 31, 127, 2, 7, 0]
    log2 = [8, 8, 9, 16, 10, 12, 16, 8, 8, 11]
    col = lc.lc_compress_batch(dev(ids), begin, eps, log2)
    assert lc.lc_serialize(col) == oracle.compress_lists(ids, begin, eps, log2)
    assert np.array_equal(host(lc.lc_decode_batch(col)), ids)
    for l in range(len(lens)):
        a, b = int(begin[l]), int(begin[l + 1])
        assert np.array_equal(host(lc.lc_decode(col, a, b - a)), ids[a:b])
    idx = inputs.uniform_ranks(2000, ids.size, seed=3)
    assert np.array_equal(host(lc.lc_access(col, dev(idx))), ids[idx.astype(np.int64)])
    with pytest.raises(lc.LcError) as e:
        lc.lc_lower_bound(col, dev(np.array([5], np.uint32)))
    assert e.value.code == lc.LC_ERR_UNSUPPORTED
    col.free()


def test_decode_ranges_many_windows():
    n = 300000
    keys = inputs.lognormal_gaps(n, seed=21)
    col = lc.lc_compress(dev(keys), eps=15)
    rng = np.random.default_rng(4)
    m = 500
    cnt = rng.integers(0, 5000, size=m).astype(np.uint64)
    beg = np.array([rng.integers(0, n - c + 1) for c in cnt], dtype=np.uint64)
    off = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.uint64)
    out = torch.zeros(int(cnt.sum()), dtype=torch.uint64, device="cuda")
    lc.lc_decode_ranges(col, dev(beg), dev(cnt), dev(off), out)
    want = np.concatenate([keys[int(b):int(b) + int(c)] for b, c in zip(beg, cnt)])
    assert np.array_equal(host(out), want)
    assert lc.lc_status(col) == lc.LC_OK
    col.free()


@pytest.mark.parametrize("dt", [np.uint32, np.uint64])
def test_decode_into_every_output_alignment(dt):
    # keys are decoded two at a time into vector stores aligned to the pair:
    # an output that starts one key in shifts every pair, and odd begins and
    # counts leave a lone first and last key; a pointer that is not a multiple
    # of the key width is refused
    n = 70001
    keys = inputs.lognormal_gaps(n, seed=33, dtype=dt)
    col = lc.lc_compress(dev(keys), eps=7)
    buf = torch.zeros(n + 2, dtype=col.dtype, device="cuda")
    for shift in (0, 1):
        for b, c in ((0, n), (1, n - 1), (3, 5000), (2048, 2049), (4095, 1), (0, 2), (n - 3, 3)):
            buf.zero_()
            lc.lc_decode(col, b, c, out=buf[shift:shift + c])
            got = host(buf)
            assert np.array_equal(got[shift:shift + c], keys[b:b + c])
            assert not got[:shift].any() and not got[shift + c:].any()
    m = 64
    rng = np.random.default_rng(5)
    cnt = rng.integers(0, 3000, size=m).astype(np.uint64)
    beg = np.array([rng.integers(0, n - c + 1) for c in cnt], dtype=np.uint64)
    off = (np.concatenate([[0], np.cumsum(cnt)[:-1]]) + np.arange(m)).astype(np.uint64)  # odd gaps between ranges
    out = torch.zeros(int(off[-1] + cnt[-1]) + 1, dtype=col.dtype, device="cuda")
    lc.lc_decode_ranges(col, dev(beg), dev(cnt), dev(off), out)
    got = host(out)
    for b, c, o in zip(beg, cnt, off):
        assert np.array_equal(got[int(o):int(o) + int(c)], keys[int(b):int(b) + int(c)])
    raw = torch.zeros(8 * (n + 2), dtype=torch.uint8, device="cuda")
    rc = lc.load().lc_decode(col.handle, 0, 10, raw.data_ptr() + 1, None)
    assert rc == lc.LC_ERR_INVALID_ARG
    assert lc.lc_status(col) == lc.LC_OK
    col.free()


def test_unsorted_input_and_out_of_range_queries():
    keys = inputs.uniform_gaps(10000, seed=2, dtype=np.uint64)
    bad = keys.copy()
    bad[7777], bad[7778] = bad[7778], bad[7777]
    with pytest.raises(lc.LcError) as e:
        lc.lc_compress(dev(bad), eps=3)
    assert e.value.code == lc.LC_ERR_UNSORTED
    col = lc.lc_compress(dev(keys), eps=3)
    got = host(lc.lc_access(col, dev(np.array([5, 10000, 3], np.uint64))))
    assert got[0] == keys[5] and got[1] == 0 and got[2] == keys[3]
    assert lc.lc_status(col) == lc.LC_ERR_OUT_OF_RANGE
    assert lc.lc_status(col) == lc.LC_OK  # cleared
    with pytest.raises(lc.LcError):
        lc.lc_decode(col, 9000, 2000)
    assert lc.lc_access1(col, 4321) == int(keys[4321])
    assert lc.lc_lower_bound1(col, int(keys[100])) == 100
    col.free()


# ------------------------------------------------------------------ full size

def _sample_chunks_match_oracle(keys, blob, eps, log2, chunks):
    """Each sampled chunk of the GPU blob equals the oracle's encoding of that
    chunk's keys compressed alone (chunks are independent)."""
    p = R.parse(blob)
    cs = 1 << log2
    for c in chunks:
        part = keys[c * cs:(c + 1) * cs]
        q = R.parse(oracle.compress(part, eps, log2))
        s0, s1 = int(p["chunk_seg_begin"][c]), int(p["chunk_seg_begin"][c + 1])
        w0, w1 = int(p["chunk_word_begin"][c]), int(p["chunk_word_begin"][c + 1])
        for nm in ("seg_start", "seg_slope", "seg_width", "seg_bitoff", "seg_icpt"):
            assert np.array_equal(p[nm][s0:s1], q[nm]), (c, nm)
        assert np.array_equal(p["payload"][w0:w1], q["payload"]), (c, "payload")


@pytest.mark.parametrize("kind,eps", [("lognormal", 15), ("piecewise", 63), ("clusters", 255), ("lognormal", 1)])
def test_full_size_column(kind, eps):
    """The 2e8-key uint64 column of the large single-column workload: decode
    equals the keys (on the device), sampled chunks equal the oracle's bytes,
    sampled access and lower_bound equal indexing and searchsorted."""
    n = 200_000_000
    keys = inputs.column(kind, n, seed=inputs.seed_for(2, 1 + ["lognormal", "piecewise", "clusters"].index(kind)))
    dk = dev(keys)
    col = lc.lc_compress(dk, eps=eps)
    out = lc.lc_decode(col)
    assert torch.equal(out, dk)
    del out
    blob = lc.lc_serialize(col)
    C = -(-n // 65536)
    _sample_chunks_match_oracle(keys, blob, eps, 16, [0, 1, C // 2, C - 2, C - 1])
    idx = inputs.uniform_ranks(200000, n, seed=7)
    assert np.array_equal(host(lc.lc_access(col, dev(idx))), keys[idx.astype(np.int64)])
    q = inputs.uniform_values(200000, int(keys[0]), int(keys[-1]), seed=8)
    assert np.array_equal(host(lc.lc_lower_bound(col, dev(q))), np.searchsorted(keys, q, side="left"))
    assert lc.lc_status(col) == lc.LC_OK
    col.free()


def _lower_bound_matches(keys, eps, check_bytes=True):
    col = lc.lc_compress(dev(keys), eps=eps)
    if check_bytes:
        assert lc.lc_serialize(col) == oracle.compress(keys, eps, 16)
    rng = np.random.default_rng(7)
    k = keys.astype(np.int64) if keys.dtype == np.uint32 else keys
    lo, hi = int(keys[0]), int(keys[-1])
    q = np.concatenate([
        rng.integers(max(0, lo - 5), hi + 6, size=100_000, dtype=np.uint64).astype(keys.dtype),
        keys, np.maximum(keys, 1) - 1, np.minimum(keys, np.iinfo(keys.dtype).max - 1) + 1,
        np.array([0, hi, np.iinfo(keys.dtype).max], dtype=keys.dtype),
    ]).astype(keys.dtype)
    got = host(lc.lc_lower_bound(col, dev(q)))
    assert np.array_equal(got, np.searchsorted(keys, q, side="left"))
    col.free()


@pytest.mark.parametrize("dt", [np.uint32, np.uint64])
@pytest.mark.parametrize("n,eps", [(1, 0), (20, 0), (3000, 0), (300_000, 0), (300_000, 7)])
def test_lower_bound_radix_table_shapes(n, eps, dt):
    """lower_bound against searchsorted: one segment, a few, and many segments
    per radix bucket; queries on, between and outside the keys."""
    keys = inputs.lognormal_gaps(n, seed=n + eps, mu=1.0, sigma=1.0, dtype=dt)
    _lower_bound_matches(keys, eps)


def test_lower_bound_skewed_buckets_and_capped_table():
    # nearly all intercepts in the first radix bucket: a long run of the table
    rng = np.random.default_rng(11)
    dense = np.cumsum(rng.integers(1, 4, size=400_000, dtype=np.uint64)).astype(np.uint64)
    keys = np.concatenate([dense, np.array([1 << 60, (1 << 60) + 7], np.uint64)])
    _lower_bound_matches(keys, 0)
    # more than 2^21 segments: the table stops growing at 2^22 buckets
    big = inputs.lognormal_gaps(6_000_000, seed=12, mu=1.0, sigma=1.0)
    _lower_bound_matches(big, 0, check_bytes=False)


def test_free_async_in_stream_order():
    # columns released in stream order while their decodes are still queued:
    # the outputs stay right and the memory is reused
    keys = inputs.lognormal_gaps(300000, seed=41)
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        d = dev(keys)
        for r in range(6):
            col = lc.lc_compress(d, eps=7 + r, stream=s)
            out = torch.empty(keys.size, dtype=col.dtype, device="cuda")
            lc.lc_decode(col, 0, keys.size, out, stream=s)
            lc.lc_free_async(col, stream=s)
            assert not col.handle.value
            outs.append(out)
    s.synchronize()
    for out in outs:
        assert np.array_equal(host(out), keys)


@pytest.mark.parametrize("span_log2", [5, 6, 7])
@pytest.mark.parametrize("gen,eps", [("lognormal", 63), ("piecewise", 15), ("clusters", 1), ("lognormal", 0)])
def test_fit_span_is_a_launch_parameter_only(span_log2, gen, eps):
    """K^c is the oracle's for every span of the speculating threads (2^5, 2^6, 2^7 keys)."""
    keys = inputs.column(gen, 700_000 + 333, seed=41, dtype=np.uint64)
    col = lc.lc_compress(dev(keys), eps=eps, span_log2=span_log2)
    assert lc.lc_serialize(col) == oracle.compress(keys, eps, 16)
    col.free()


@pytest.mark.parametrize("span_log2", [5, 7])
def test_fit_span_in_list_mode(span_log2):
    ids, begin = inputs.posting_lists(800, 1_500_000, 10_000_000, seed=9)
    col = lc.lc_compress_batch(dev(ids), begin, 7, 14, span_log2=span_log2)
    assert lc.lc_serialize(col) == oracle.compress_lists(ids, begin, 7, 14)
    col.free()
