"""GPU parity of the quantile and segments-only queries (Sec. III-C) through
the C ABI: exact quantiles equal the key at floor(N k / q); approximate
quantiles and the segments-only decode equal the oracle's floor(f(i)) byte
for byte, and stay within eps of the keys."""
from __future__ import annotations

import numpy as np
import pytest
import torch

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [("lognormal", 63, np.uint64, 300_007), ("uniform", 15, np.uint32, 200_003),
         ("clusters", 0, np.uint64, 131_072), ("piecewise", 1023, np.uint64, 70_001)]


@pytest.mark.parametrize("kind,eps,dt,n", CASES)
def test_quantiles_exact_and_approx(kind, eps, dt, n):
    keys = inputs.column(kind, n, seed=n, dtype=dt)
    blob = oracle.compress(keys, eps, 16)
    col = lc.lc_compress(dev(keys), eps=eps)
    for q in (1, 2, 4, 100, 1000, 1 << 20, 2**40):
        ks = np.unique(np.concatenate([np.array([0, 1, q // 2, q - 1, q], np.uint64),
                                       np.random.default_rng(q).integers(0, q + 1, 500, dtype=np.uint64)]))
        ks = ks[ks <= q]
        idx = np.array([oracle.quantile_index(n, int(k), q) for k in ks], np.uint64)
        got = lc.lc_quantile(col, dev(ks), q, exact=True).cpu().numpy()
        assert np.array_equal(got, keys[idx.astype(np.int64)]), q
        got = lc.lc_quantile(col, dev(ks), q, exact=False).cpu().numpy()
        assert np.array_equal(got, oracle.predict(blob, idx)), q
    assert lc.lc_status(col) == lc.LC_OK
    # k > q: 0 and an out-of-range status
    got = lc.lc_quantile(col, dev(np.array([5], np.uint64)), 4).cpu().numpy()
    assert got[0] == 0 and lc.lc_status(col) == lc.LC_ERR_OUT_OF_RANGE
    col.free()


@pytest.mark.parametrize("kind,eps,dt,n", CASES)
def test_segments_only_decode_matches_oracle(kind, eps, dt, n):
    keys = inputs.column(kind, n, seed=n + 1, dtype=dt)
    blob = oracle.compress(keys, eps, 16)
    col = lc.lc_compress(dev(keys), eps=eps)
    want = oracle.predict(blob, np.arange(n, dtype=np.uint64))
    assert np.array_equal(lc.lc_decode_approx(col).cpu().numpy(), want)
    for b, c in ((0, 1), (n - 1, 1), (12345, 4099), (n // 2, n - n // 2)):
        assert np.array_equal(lc.lc_decode_approx(col, b, c).cpu().numpy(), want[b:b + c])
    with pytest.raises(lc.LcError):
        lc.lc_decode_approx(col, n - 1, 2)
    col.free()


def test_segments_only_decode_list_mode():
    rng = np.random.default_rng(3)
    lens = [1, 50, 3000, 70_000, 17]
    keys = np.concatenate([np.sort(rng.integers(0, 10**6, size=m, dtype=np.uint64)).astype(np.uint32) for m in lens])
    begin = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    eps = np.array([3, 0, 15, 63, 7], np.uint64)
    log2 = np.array([16, 8, 10, 16, 12], np.uint8)
    blob = oracle.compress_lists(keys, begin, eps, log2)
    col = lc.lc_compress_batch(dev(keys), begin, eps, log2)
    want = oracle.predict(blob, np.arange(keys.size, dtype=np.uint64))
    assert np.array_equal(lc.lc_decode_approx(col).cpu().numpy(), want)
    col.free()


def test_full_size_column_segments_only():
    """The 2e8-key lognormal column of the large single-column workload at eps
    63: every approximate key within eps of the exact one (on the device);
    sampled chunks equal the oracle's predictions; sampled quantiles exact."""
    n = 200_000_000
    keys = inputs.column("lognormal", n, seed=inputs.seed_for(2, 1))
    dk = dev(keys)
    col = lc.lc_compress(dk, eps=63)
    approx = lc.lc_decode_approx(col)
    diff = approx.view(torch.int64) - dk.view(torch.int64)  # keys < 2^63
    assert int(diff.abs().max()) <= 63
    for c in (0, 1500, 3051):
        part = keys[c * 65536:(c + 1) * 65536]
        want = oracle.predict(oracle.compress(part, 63, 16), np.arange(part.size, dtype=np.uint64))
        assert np.array_equal(approx[c * 65536:c * 65536 + part.size].cpu().numpy(), want), c
    del approx
    ks = np.arange(0, 1001, dtype=np.uint64)
    idx = np.array([oracle.quantile_index(n, int(k), 1000) for k in ks])
    assert np.array_equal(lc.lc_quantile(col, dev(ks), 1000).cpu().numpy(), keys[idx])
    col.free()


def _mixed_column(seed: int) -> np.ndarray:
    """Consecutive regimes of whole chunks from different generators (a column
    whose best eps changes along the keys)."""
    parts, base = [], np.uint64(0)
    gens = [lambda n, s: inputs.uniform_gaps(n, s, dtype=np.uint64),
            lambda n, s: inputs.clusters(n, s),
            lambda n, s: inputs.lognormal_gaps(n, s, mu=3.0, sigma=2.0),
            lambda n, s: inputs.piecewise_linear(n, s)]
    for r in range(8):
        k = gens[r % 4](3 * 65536, seed + r)
        k = k - k[0] + base + np.uint64(1)
        parts.append(k)
        base = k[-1]
    return np.concatenate(parts)


def test_eps_per_partition_column():
    """Sec. IV-A: eps chosen per partition of whole chunks by the shortest path
    over measured chunk costs; stored as a list-mode column that equals the
    oracle's bytes, decodes exactly and is no larger than the best single eps."""
    from paper_2412_10770_gb300 import tune

    keys = _mixed_column(5)
    dk = dev(keys)
    cands = (0, 1, 3, 15, 63, 255, 1023)
    pb, pe, info = tune.partition_eps(dk, cands)
    assert pb[0] == 0 and pb[-1] == keys.size and info["partitions"] >= 2
    col = lc.lc_compress_batch(dk, pb, pe, 16)
    blob = lc.lc_serialize(col)
    assert blob == oracle.compress_lists(keys, pb, pe, np.full(pe.size, 16, np.uint8))
    assert torch.equal(lc.lc_decode(col), dk)
    single = lc.lc_compress(dk, eps=info["best_single_eps"])
    assert lc.lc_size(col) <= lc.lc_size(single)
    single.free()
    col.free()
