"""Failure detection on the GPU without a fault: the decoders' bounded
mbarrier wait is made to run out (a barrier that nothing completes) and must
give up with LC_ERR_TIMEOUT, promptly, leaving the context usable."""
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


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    t0 = time.perf_counter()
    assert lc.lc_selftest_wait(1024) == lc.LC_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    assert lc.lc_selftest_wait(0) == lc.LC_ERR_INVALID_ARG
    keys = inputs.uniform_gaps(100000, seed=3, dtype=np.uint64)
    col = lc.lc_compress(torch.from_numpy(keys).cuda(), eps=7)
    assert np.array_equal(lc.lc_decode(col).cpu().numpy(), keys)
    assert lc.lc_status(col) == lc.LC_OK
    col.free()
