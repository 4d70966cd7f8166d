"""The batching path as one CUDA graph (lc_batch_*): the replayed compress
writes the oracle's list-mode bytes (Def. 1, byte identity) and the replayed
decode returns every id, on repeated launches; a replay on keys whose K^c
no longer fits the planned layout reports LC_ERR_STALE instead of writing."""
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


def test_graph_replays_compress_and_decode():
    ids, begin = inputs.posting_lists(2000, 3_000_000, 20_000_000, seed=13)
    eps = (np.arange(2000) % 5 * 3).astype(np.uint64)
    log2 = np.where(np.arange(2000) % 2 == 0, 16, 12).astype(np.uint8)
    d = torch.from_numpy(ids).cuda()
    out = torch.zeros_like(d)
    s = torch.cuda.Stream()
    b = lc.Batch(d, begin, out, eps, log2, stream=s)
    ref = oracle.compress_lists(ids, begin, eps, log2)
    assert lc.lc_serialize(b.column) == ref  # the planning compress
    for _ in range(3):
        out.zero_()
        torch.cuda.synchronize()
        b.launch(stream=s)
        s.synchronize()
        assert lc.lc_status(b.column, s) == lc.LC_OK
        assert torch.equal(out, d)
        assert lc.lc_serialize(b.column) == ref
    # queries on the replayed column
    idx = torch.from_numpy(np.arange(0, ids.size, 997, dtype=np.uint64)).cuda()
    assert np.array_equal(lc.lc_access(b.column, idx).cpu().numpy(), ids[idx.cpu().numpy().astype(np.int64)])
    b.free()


def test_replay_on_keys_that_do_not_fit_is_flagged():
    ids, begin = inputs.posting_lists(500, 600_000, 10_000_000, seed=17)
    d = torch.from_numpy(ids).cuda()
    out = torch.zeros_like(d)
    b = lc.Batch(d, begin, out, 7, 16)
    # every list becomes an arithmetic progression: far fewer segments than planned
    d.copy_(torch.arange(ids.size, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32))
    out.zero_()
    b.launch()
    torch.cuda.synchronize()
    assert lc.lc_status(b.column) == lc.LC_ERR_STALE
    assert not out.view(torch.int32).any()  # the gated decode wrote nothing
    b.free()
