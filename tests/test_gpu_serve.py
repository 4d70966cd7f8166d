"""Serving with continuous batching (lc_server_*): a mixed stream of access,
lower_bound and range-decode requests over several device-resident columns.

Every result served in the mix equals the same request served alone through
the plain synchronous path (lc_serve_sync) and the raw-key definition
(indexing, searchsorted, slicing): integer results, compared bit for bit.
The server never holds more device memory than its budget, runs batches
concurrently, and fails requests that can never fit or that are out of range.
"""
from __future__ import annotations

import time

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


@pytest.fixture(scope="module")
def columns():
    keys = [inputs.column(kind, 300_000 + 1111 * i, seed=100 + i)
            for i, kind in enumerate(["lognormal", "piecewise", "clusters", "uniform", "lognormal"])]
    keys = [k.astype(np.uint64) for k in keys]
    cols = [lc.lc_compress(torch.from_numpy(k).cuda(), eps=63) for k in keys]
    yield keys, cols
    for c in cols:
        c.free()


def make_requests(keys, n, seed, max_dec=200_000):
    rng = np.random.default_rng(seed)
    reqs = []
    for u in range(n):
        c = int(rng.integers(0, len(keys)))
        N = keys[c].size
        r = rng.random()
        if r < 0.4:
            cnt = int(rng.integers(1, 4097))
            inp = rng.integers(0, N, size=cnt, dtype=np.uint64)
            reqs.append(dict(op=lc.LC_OP_ACCESS, column=c, count=cnt, begin=0, inp=inp,
                             out=np.zeros(cnt, np.uint64), want=keys[c][inp.astype(np.int64)]))
        elif r < 0.8:
            cnt = int(rng.integers(1, 4097))
            inp = rng.integers(0, int(keys[c][-1]) + 2, size=cnt, dtype=np.uint64)
            reqs.append(dict(op=lc.LC_OP_LOWER_BOUND, column=c, count=cnt, begin=0, inp=inp,
                             out=np.zeros(cnt, np.uint64), want=np.searchsorted(keys[c], inp, side="left")))
        else:
            cnt = int(np.exp(rng.uniform(0, np.log(max_dec))))
            b = int(rng.integers(0, N - cnt + 1))
            reqs.append(dict(op=lc.LC_OP_DECODE, column=c, count=cnt, begin=b, inp=None,
                             out=np.zeros(cnt, np.uint64), want=keys[c][b:b + cnt]))
    return reqs


def submit(srv, reqs, gap_s=0.0, first=0):
    for u, q in enumerate(reqs):
        srv.submit(q["op"], q["column"], q["count"], q["begin"], 0 if q["inp"] is None else q["inp"].ctypes.data,
                   q["out"].ctypes.data, user=first + u)
        if gap_s:
            time.sleep(gap_s)


def drain(srv, n, timeout_s=60):
    got = {}
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        for c in srv.wait(1024, 200_000):
            got[c["user"]] = c
    assert len(got) == n, f"{len(got)} of {n} completed"
    return got


def test_mixed_stream_equals_each_request_alone(columns):
    keys, cols = columns
    reqs = make_requests(keys, 400, seed=1)
    budget = 12 << 20
    srv = lc.lc_server_create(cols, budget, slots=4)
    submit(srv, reqs[:150])
    submit(srv, reqs[150:], gap_s=0.0002, first=150)  # more arrive while the first ones run
    got = drain(srv, len(reqs))
    st = srv.stats()
    srv.close()
    for u, q in enumerate(reqs):
        assert got[u]["status"] == lc.LC_OK, (u, got[u])
        assert np.array_equal(q["out"], q["want"]), (u, q["op"])
    assert st["peak_hbm_bytes"] <= budget
    assert st["batches"] < len(reqs)           # requests were batched
    assert st["peak_inflight"] >= 2            # batches overlapped on the device
    # the same requests, one at a time on the plain path
    for u, q in enumerate(reqs[:120]):
        alone = np.zeros_like(q["out"])
        c = lc.lc_serve_sync(cols, q["op"], q["column"], q["count"], q["begin"],
                             0 if q["inp"] is None else q["inp"].ctypes.data, alone.ctypes.data)
        assert c["status"] == lc.LC_OK
        assert np.array_equal(alone, q["out"])


def test_admission_and_errors(columns):
    keys, cols = columns
    srv = lc.lc_server_create(cols, 1 << 20, slots=2)
    big = np.zeros(keys[0].size, np.uint64)  # 2.4 MB of output: more than the whole budget
    bad_idx = np.array([keys[1].size], np.uint64)
    out1 = np.zeros(1, np.uint64)
    ok_out = np.zeros(1000, np.uint64)
    srv.submit(lc.LC_OP_DECODE, 0, keys[0].size, 0, 0, big.ctypes.data, user=1)
    srv.submit(lc.LC_OP_ACCESS, 1, 1, 0, bad_idx.ctypes.data, out1.ctypes.data, user=2)
    srv.submit(lc.LC_OP_DECODE, 2, 1000, 5, 0, ok_out.ctypes.data, user=3)
    got = drain(srv, 3)
    st = srv.stats()
    srv.close()
    assert got[1]["status"] == lc.LC_ERR_NOMEM
    assert got[2]["status"] == lc.LC_ERR_OUT_OF_RANGE
    assert got[3]["status"] == lc.LC_OK and np.array_equal(ok_out, keys[2][5:1005])
    assert st["peak_hbm_bytes"] <= 1 << 20
