"""Byte-identical K^c at the full sizes of the benchmark workloads (Def. 1 and
the LCF1 format: the GPU writes the oracle's bytes), every chunk compared:

* the large single column: 2e8 uint64 keys from each generator (lognormal,
  piecewise-linear, clusters) at eps 1 and 63;
* the scale sweep: 1e9 uint64 keys from the lognormal generator (mu 3,
  sigma 2) at eps 0, the largest blob of the sweep;
* the posting-list batch: 1e6 lists of uint32 ids, 2e9 ids in all, in one
  batched compress with the autotuner's eps and chunk size per list.

The oracle runs on every host core in chunk-aligned (or list-aligned) pieces
(tests/fullsize.py); each piece's arrays must equal the GPU blob's.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import fullsize
from paper_2412_10770_gb300 import inputs, lc

pytestmark = pytest.mark.gpu

GENS = ("lognormal", "piecewise", "clusters")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2412_10770_gb300 import build

    build.build()
    lc.load()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("gen", GENS)
def test_large_column_every_chunk(gen):
    n = 200_000_000
    keys = inputs.column(gen, n, seed=inputs.seed_for(2, 1 + GENS.index(gen)), dtype=np.uint64)
    d = torch.from_numpy(keys).cuda()
    for eps in (1, 63):
        col = lc.lc_compress(d, eps=eps)
        blob = lc.lc_serialize(col)
        col.free()
        assert fullsize.check_column(blob, keys, eps) == -(-n // 65536)
    del d


def test_scale_sweep_column_every_chunk_at_eps0():
    n = 1_000_000_000
    d = inputs.column_device("lognormal", n, seed=inputs.seed_for(5, 1), mu=3.0, sigma=2.0)
    col = lc.lc_compress(d, eps=0)
    keys = d.cpu().numpy()
    del d
    blob = lc.lc_serialize(col)
    col.free()
    torch.cuda.empty_cache()
    assert fullsize.check_column(blob, keys, 0) == -(-n // 65536)


def test_posting_list_batch_every_list():
    from paper_2412_10770_gb300 import tune

    ids, begin = inputs.posting_lists_device(1_000_000, 2_000_000_000, 50_000_000, seed=inputs.seed_for(3, 1))
    eps, log2, _ = tune.tune(ids, begin, sample_lists=16, sample_keys=1 << 20)
    col = lc.lc_compress_batch(ids, begin, eps, log2)
    keys = ids.cpu().numpy()
    del ids
    blob = lc.lc_serialize(col)
    col.free()
    torch.cuda.empty_cache()
    assert fullsize.check_lists(blob, keys, begin, eps, log2) == 1_000_000
