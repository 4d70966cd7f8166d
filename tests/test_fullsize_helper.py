"""The full-size comparison helper (tests/fullsize.py) on the CPU: an oracle
blob compared against the oracle's own pieces passes, for a single column and
for list mode, and a blob with one payload word, one slope or one chunk
offset changed fails."""
from __future__ import annotations

import numpy as np
import pytest

import fullsize
import lcf_reader as R
import oracle
from paper_2412_10770_gb300 import inputs


def _mutate(blob: bytes, name: str, idx: int) -> bytes:
    p = R.parse(blob)
    off = p[name].ctypes.data - np.frombuffer(blob, dtype=np.uint8).ctypes.data
    b = bytearray(blob)
    b[off + idx * p[name].itemsize] ^= 1
    return bytes(b)


def test_single_column_pieces():
    oracle.build()
    keys = inputs.lognormal_gaps(5 * 65536 + 777, seed=2, dtype=np.uint64)
    blob = oracle.compress(keys, 15, 16)
    assert fullsize.check_column(blob, keys, 15, pieces=3) == 6
    p = R.parse(blob)
    for name, idx in (("payload", int(p["words"]) - 3), ("seg_slope", int(p["segments"]) // 2),
                      ("chunk_word_begin", 4)):
        with pytest.raises(AssertionError):
            fullsize.check_column(_mutate(blob, name, idx), keys, 15, pieces=3)


def test_list_mode_pieces():
    oracle.build()
    keys, begin = inputs.posting_lists(300, 400_000, 5_000_000, seed=4)
    eps = (np.arange(300) % 4 * 5).astype(np.uint64)
    log2 = np.full(300, 12, dtype=np.uint8)
    blob = oracle.compress_lists(keys, begin, eps, log2)
    assert fullsize.check_lists(blob, keys, begin, eps, log2, pieces=5) == 300
    p = R.parse(blob)
    with pytest.raises(AssertionError):
        fullsize.check_lists(_mutate(blob, "seg_width", int(p["segments"]) - 2), keys, begin, eps, log2, pieces=5)
