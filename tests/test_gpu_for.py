"""GPU parity of the scale-sweep workload: the FOR-delta bp128 baseline codec
against its CPU reference (byte-identical FOR1 blobs, exact decode), and the
learned compressor on 1e9-key columns of the sweep's generators (decode equal
to the keys on the device, sampled chunks byte-identical to the oracle,
sampled access and lower_bound equal to indexing and searchsorted)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import forf_reader as F
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


def _cases():
    rng = np.random.default_rng(21)
    for n in (1, 2, 127, 128, 129, 4097):
        yield f"gaps{n}", np.cumsum(rng.integers(0, 90, size=n, dtype=np.uint64)).astype(np.uint64)
    yield "const", np.full(1000, 123456789, np.uint64)
    yield "u32", inputs.uniform_gaps(100_003, seed=2, dtype=np.uint32)
    yield "u32-wide", np.sort(rng.integers(0, 1 << 32, size=3000, dtype=np.uint64)).astype(np.uint32)
    yield "u64-64bit-gaps", np.array([0, 5, (1 << 63) + 11, (1 << 64) - 1], np.uint64)
    yield "lognormal", inputs.lognormal_gaps(300_001, seed=8, mu=3.0, sigma=2.0)
    yield "piecewise", inputs.piecewise_linear(200_000, seed=6)


@pytest.mark.parametrize("name,keys", list(_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_for_matches_reference_and_decodes(name, keys):
    d = torch.from_numpy(keys).cuda()
    f = lc.lc_for_compress(d)
    blob = lc.lc_for_serialize(f)
    assert blob == oracle.for_compress(keys)
    assert lc.lc_for_size(f) == len(blob)
    assert torch.equal(lc.lc_for_decode(f), d)
    f.free()


def test_for_empty_and_unsorted():
    f = lc.lc_for_compress(torch.empty(0, dtype=torch.uint64, device="cuda"))
    assert lc.lc_for_serialize(f) == oracle.for_compress(np.empty(0, np.uint64))
    assert lc.lc_for_decode(f).numel() == 0
    f.free()
    bad = torch.tensor([5, 9, 7, 12] * 100, dtype=torch.int64, device="cuda").view(torch.uint64)
    with pytest.raises(lc.LcError) as e:
        lc.lc_for_compress(bad)
    assert e.value.code == lc.LC_ERR_UNSORTED


N_SWEEP = 1_000_000_000


@pytest.fixture(scope="module")
def sweep_lognormal():
    k = inputs.column_device("lognormal", N_SWEEP, seed=inputs.seed_for(5, 1), mu=3.0, sigma=2.0)
    yield k
    del k
    torch.cuda.empty_cache()


def _sample_queries(col, keys, n, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    idx = torch.randint(0, n, (200_000,), generator=g, device="cuda", dtype=torch.int64)
    got = lc.lc_access(col, idx.view(torch.uint64))
    k64 = keys.view(torch.int64)  # the sweep's keys stay below 2^63
    assert torch.equal(got.view(torch.int64), k64[idx])
    lo, hi = int(k64[0]), int(k64[-1])
    q = torch.randint(lo, hi + 1, (200_000,), generator=g, device="cuda", dtype=torch.int64)
    got = lc.lc_lower_bound(col, q.view(torch.uint64))
    assert torch.equal(got.view(torch.int64), torch.searchsorted(k64, q, side="left"))


def _sample_chunks(keys, blob, eps, chunks):
    p = R.parse(blob)
    for c in chunks:
        part = keys[c * 65536:(c + 1) * 65536].cpu().numpy()
        q = R.parse(oracle.compress(part, eps, 16))
        s0, s1 = int(p["chunk_seg_begin"][c]), int(p["chunk_seg_begin"][c + 1])
        w0, w1 = int(p["chunk_word_begin"][c]), int(p["chunk_word_begin"][c + 1])
        for nm in ("seg_start", "seg_slope", "seg_width", "seg_bitoff", "seg_icpt"):
            assert np.array_equal(p[nm][s0:s1], q[nm]), (c, nm)
        assert np.array_equal(p["payload"][w0:w1], q["payload"]), (c, "payload")


@pytest.mark.parametrize("eps", [1023, 0])
def test_scale_sweep_lognormal_full_size(sweep_lognormal, eps):
    """N = 1e9 uint64 keys with lognormal gaps (mu 3, sigma 2), the launch the
    scale sweep times: exact decode, sampled bytes and queries."""
    keys = sweep_lognormal
    n = keys.numel()
    col = lc.lc_compress(keys, eps=eps)
    out = lc.lc_decode(col)
    assert torch.equal(out, keys)
    del out
    C = -(-n // 65536)
    if eps >= 63:  # the blob is small enough to bring back to the host
        _sample_chunks(keys, lc.lc_serialize(col), eps, [0, 1, C // 3, C - 2, C - 1])
    _sample_queries(col, keys, n, seed=eps + 1)
    assert lc.lc_status(col) == lc.LC_OK
    col.free()


def test_scale_sweep_for_baseline_full_size(sweep_lognormal):
    keys = sweep_lognormal
    n = keys.numel()
    f = lc.lc_for_compress(keys)
    out = lc.lc_for_decode(f)
    assert torch.equal(out, keys)
    del out
    blob = lc.lc_for_serialize(f)
    p = F.parse(blob)
    woff = np.concatenate([[0], np.cumsum(4 * p["width"].astype(np.uint64))])
    B = p["blocks"]
    for b0 in (0, B // 2, B - 3):
        m = min(3, B - b0)
        part = keys[128 * b0:min(n, 128 * (b0 + m))].cpu().numpy()
        q = F.parse(oracle.for_compress(part))
        assert np.array_equal(p["base"][b0:b0 + m], q["base"])
        assert np.array_equal(p["width"][b0:b0 + m], q["width"])
        a, e = 4 * int(woff[b0]), 4 * int(woff[b0 + m])
        assert p["payload"][a:e] == q["payload"]
    f.free()


def test_scale_sweep_piecewise_full_size():
    keys = inputs.column_device("piecewise", N_SWEEP, seed=inputs.seed_for(5, 2))
    n = keys.numel()
    col = lc.lc_compress(keys, eps=15)
    out = lc.lc_decode(col)
    assert torch.equal(out, keys)
    del out
    C = -(-n // 65536)
    _sample_chunks(keys, lc.lc_serialize(col), 15, [0, C // 2, C - 1])
    _sample_queries(col, keys, n, seed=3)
    col.free()
    f = lc.lc_for_compress(keys)
    out = lc.lc_for_decode(f)
    assert torch.equal(out, keys)
    f.free()
