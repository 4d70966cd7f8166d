"""The fit's window size is a launch shape only: K^c stays the oracle's bytes.

A window is one CTA of the speculative walks and of the short-segment models.
A run takes 2048-key windows when its chunks average fewer than 16384 keys
(at spans of 32 and 64 keys), else 4096-key windows, and always 4096 at the
128-key span.  The cases below reach both sizes from each side: single
columns with chunks of 2^8 to 2^16 keys, posting lists whose mean length
falls below and above the threshold, and every span, each against the
oracle's serialized column (Def. 1) and the keys decoded back.
"""
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


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("span_log2", [5, 6, 7])
@pytest.mark.parametrize("chunk_log2", [8, 11, 13, 14, 16])
@pytest.mark.parametrize("gen,eps", [("lognormal", 15), ("clusters", 3)])
def test_single_column_any_window(span_log2, chunk_log2, gen, eps):
    # 150077 keys: with 2^14-key chunks the mean chunk (15007 keys) is just
    # under the threshold, with 2^16 above it; the last chunk is ragged
    keys = inputs.column(gen, 150_077, seed=61 + chunk_log2, dtype=np.uint64)
    col = lc.lc_compress(dev(keys), eps=eps, chunk_log2=chunk_log2, span_log2=span_log2)
    assert lc.lc_serialize(col) == oracle.compress(keys, eps, chunk_log2)
    assert np.array_equal(lc.lc_decode(col).cpu().numpy(), keys)
    col.free()


@pytest.mark.parametrize("span_log2", [5, 6, 7])
@pytest.mark.parametrize("n_lists,total", [(2000, 600_000), (24, 600_000)])
def test_lists_any_window(span_log2, n_lists, total):
    # mean list length 300 (narrow windows) and 25000 (wide windows, lists
    # spanning several 2^14-key chunks)
    ids, begin = inputs.posting_lists(n_lists, total, 5_000_000, seed=7 + n_lists)
    col = lc.lc_compress_batch(dev(ids), begin, 31, 14, span_log2=span_log2)
    assert lc.lc_serialize(col) == oracle.compress_lists(ids, begin, 31, 14)
    assert np.array_equal(lc.lc_decode(col).cpu().numpy(), ids)
    col.free()
