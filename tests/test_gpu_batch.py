"""Batching path on the GPU: posting lists with autotuned (eps, chunk_log2) per
list-length bucket, compressed in one batched call and decoded by one
persistent launch replayed from a CUDA graph.  Parity: the batch K^c is
byte-identical to the oracle's list-mode encoding with the same per-list
parameters; every decoded id equals the input."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import lcf_reader as R
import oracle
from paper_2412_10770_gb300 import inputs, lc, tune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_10770_gb300 import build

    build.build()
    oracle.build()
    lc.load()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def lists():
    ids, begin = inputs.posting_lists(3000, 3_000_000, 5 * 10**7, seed=inputs.seed_for(3, 0), hi=400_000)
    return ids, begin


def test_tuned_batch_matches_oracle_and_decodes(lists):
    ids, begin = lists
    d = torch.from_numpy(ids).cuda()
    eps, log2, table = tune.tune(d, begin, sample_lists=8, sample_keys=1 << 17)
    assert len(table["buckets"]) >= 5
    col = lc.lc_compress_batch(d, begin, eps, log2)
    assert lc.lc_serialize(col) == oracle.compress_lists(ids, begin, eps, log2)
    g, out = lc.lc_graph_decode(col)
    out.zero_()
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out, d)
    for l in np.random.default_rng(1).choice(len(begin) - 1, 50, replace=False):
        a, b = int(begin[l]), int(begin[l + 1])
        assert np.array_equal(lc.lc_decode(col, a, b - a).cpu().numpy(), ids[a:b])
    g.free()
    # the tuned parameters are no worse than one global setting
    for e in (7, 63):
        ref = lc.lc_compress_batch(d, begin, e, 16)
        assert lc.lc_size(col) <= lc.lc_size(ref)
        ref.free()
    col.free()


def test_batched_equals_one_call_per_list(lists):
    ids, begin = lists
    d = torch.from_numpy(ids).cuda()
    col = lc.lc_compress_batch(d, begin, 31, 12)
    dec = lc.lc_decode_batch(col)
    P = R.parse(lc.lc_serialize(col))
    for l in range(0, len(begin) - 1, 97):
        a, b = int(begin[l]), int(begin[l + 1])
        one = lc.lc_compress(d[a:b], eps=31, chunk_log2=12)
        assert torch.equal(lc.lc_decode(one), dec[a:b])
        # the list's chunks inside the batch column hold exactly the single column's model and payload
        Q = R.parse(lc.lc_serialize(one))
        c0, c1 = int(P["list_chunk_begin"][l]), int(P["list_chunk_begin"][l + 1])
        s0, s1 = int(P["chunk_seg_begin"][c0]), int(P["chunk_seg_begin"][c1])
        w0, w1 = int(P["chunk_word_begin"][c0]), int(P["chunk_word_begin"][c1])
        for nm in ("seg_start", "seg_slope", "seg_width", "seg_bitoff", "seg_icpt"):
            assert np.array_equal(P[nm][s0:s1], Q[nm])
        assert np.array_equal(P["payload"][w0:w1], Q["payload"])
        one.free()
    assert torch.equal(dec, d)
    col.free()


def test_device_generator_lists_are_sorted_samples():
    ids, begin = inputs.posting_lists_device(2000, 2_000_000, 5 * 10**7, seed=5, max_sort=1 << 20)
    h = ids.cpu().numpy()
    lens = np.diff(begin)
    assert int(begin[-1]) == h.size and lens.min() >= 16
    for l in range(0, 2000, 7):
        x = h[int(begin[l]):int(begin[l + 1])].astype(np.int64)
        assert (np.diff(x) > 0).all() and x.min() >= 0 and x.max() < 5 * 10**7


def test_many_short_lists_large_directories():
    # 60000 lists of 16-40 ids: the batch's descriptors and header exceed the
    # 1 MB above which the compressor's small-transfer staging hands them to
    # an ordinary copy; the bytes must not change
    rng = np.random.default_rng(11)
    lens = rng.integers(16, 41, size=60000)
    parts = [np.sort(rng.choice(1_000_000, size=int(k), replace=False)).astype(np.uint32) for k in lens]
    ids = np.concatenate(parts)
    begin = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    eps = np.where(lens < 28, 3, 15).astype(np.uint64)
    log2 = np.full(len(lens), 16, dtype=np.uint8)
    d = torch.from_numpy(ids).cuda()
    col = lc.lc_compress_batch(d, begin, eps, log2)
    assert lc.lc_serialize(col) == oracle.compress_lists(ids, begin, eps, log2)
    assert torch.equal(lc.lc_decode_batch(col), d)
    col.free()
