"""The host-buffer entry points (lc_compress_host, lc_decode_host,
lc_decode_ranges_host, lc_access_host, lc_lower_bound_host): the same K^c
bytes as the oracle and the same results as the device calls' plain
definitions (Def. 1), with page-locked and with pageable host memory."""
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


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dt", [np.uint64, np.uint32])
def test_host_calls_match_the_definitions(pinned, dt):
    n = 300_000
    keys = inputs.lognormal_gaps(n, seed=21, mu=1.5, sigma=1.2, dtype=dt)

    def h(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.pin_memory() if pinned else t

    s = torch.cuda.Stream()
    col = lc.lc_compress_host(h(keys), eps=15, stream=s)
    assert lc.lc_serialize(col) == oracle.compress(keys, 15, 16)
    kt = torch.uint64 if dt == np.uint64 else torch.uint32
    dec = h(np.zeros(n - 100, dtype=dt))
    lc.lc_decode_host(col, dec, begin=50, count=n - 100, stream=s)
    rng = np.random.default_rng(4)
    m = 5000
    idx = rng.integers(0, n, size=m).astype(np.uint64)
    acc = h(np.zeros(m, dtype=dt))
    lc.lc_access_host(col, h(idx), acc, stream=s)
    vals = np.sort(rng.integers(0, int(keys[-1]) + 10, size=m)).astype(dt)
    lb = h(np.zeros(m, dtype=np.uint64))
    lc.lc_lower_bound_host(col, h(vals), lb, stream=s)
    beg = rng.integers(0, n - 700, size=200).astype(np.uint64)
    cnt = rng.integers(0, 700, size=200).astype(np.uint64)
    off = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.uint64)
    out = h(np.zeros(int(cnt.sum()) + 3, dtype=dt))
    lc.lc_decode_ranges_host(col, h(beg), h(cnt), h(off), out, stream=s)
    s.synchronize()
    assert dec.dtype == kt or dec.element_size() == keys.itemsize
    assert np.array_equal(dec.numpy(), keys[50:n - 50])
    assert np.array_equal(acc.numpy(), keys[idx.astype(np.int64)])
    assert np.array_equal(lb.numpy().astype(np.int64), np.searchsorted(keys, vals, side="left"))
    want = np.concatenate([keys[int(b):int(b) + int(c)] for b, c in zip(beg, cnt)])
    assert np.array_equal(out.numpy()[:want.size], want)
    assert lc.lc_status(col, s) == lc.LC_OK
    col.free()


def test_host_calls_refuse_device_tensors():
    keys = torch.arange(1000, dtype=torch.int64).view(torch.uint64)
    with pytest.raises(ValueError):
        lc.lc_compress_host(keys.cuda(), eps=3)
