"""Pins of the CPU reference of the FOR-delta bp128 baseline (``oracle/for_bp128.c``)
against the format's definition: an independent reader decodes the keys back,
the length equals the closed form, the padding is zero, unsorted input is
refused.  No GPU."""
from __future__ import annotations

import numpy as np
import pytest

import forf_reader as F
import oracle
from paper_2412_10770_gb300 import inputs


def _cases():
    rng = np.random.default_rng(5)
    yield "empty", np.empty(0, np.uint64)
    for n in (1, 2, 127, 128, 129, 255, 256, 1000):
        yield f"gaps{n}", np.cumsum(rng.integers(0, 50, size=n, dtype=np.uint64)).astype(np.uint64)
    yield "const", np.full(300, 7, np.uint64)
    yield "u32", inputs.uniform_gaps(5000, seed=3, dtype=np.uint32)
    yield "u32-max-gap", np.array([0, 0xFFFFFFFF] * 1, np.uint32)
    yield "u64-max-gap", np.array([0, 1, (1 << 64) - 1], np.uint64)
    yield "lognormal", inputs.lognormal_gaps(20000, seed=9, mu=3.0, sigma=2.0)
    yield "clusters", inputs.clusters(9000, seed=4)


@pytest.mark.parametrize("name,keys", list(_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_reference_roundtrips_and_matches_closed_form(name, keys):
    blob = oracle.for_compress(keys)
    assert len(blob) == F.size(keys)
    p = F.parse(blob)
    assert p["pads_zero"]
    assert np.array_equal(F.decode(blob), keys)
    assert np.array_equal(oracle.for_decode(blob), keys)
    # widths are the bit lengths of each block's largest gap
    k = keys.astype(object)
    for b in range(p["blocks"]):
        blk = k[128 * b:128 * b + 128]
        g = max((int(blk[i]) - int(blk[i - 1]) for i in range(1, len(blk))), default=0)
        assert int(p["width"][b]) == g.bit_length()
        assert int(p["base"][b]) == int(blk[0])


def test_reference_refuses_unsorted_keys():
    with pytest.raises(oracle.OracleError):
        oracle.for_compress(np.array([3, 2], np.uint64))


def test_gap_of_two_to_the_64_minus_one_takes_64_bits():
    keys = np.array([0, (1 << 64) - 1], np.uint64)
    p = F.parse(oracle.for_compress(keys))
    assert int(p["width"][0]) == 64 and p["words"] == 256
