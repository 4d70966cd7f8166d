"""Pins of the oracle's quantile and segments-only (approximate) answers
(Sec. III-C): the model prediction floor(f(i)) equals an independent reader's
exact-integer evaluation of the stored segments, stays within eps of every key
(Def. 2), and the quantile index is floor(N k / q).  No GPU."""
from __future__ import annotations

import numpy as np
import pytest

import lcf_reader as R
import oracle
from paper_2412_10770_gb300 import inputs


@pytest.mark.parametrize("kind,eps,dt", [("lognormal", 0, np.uint64), ("lognormal", 63, np.uint64),
                                         ("clusters", 15, np.uint64), ("uniform", 15, np.uint32),
                                         ("piecewise", 255, np.uint64)])
def test_prediction_is_the_segment_line_and_within_eps(kind, eps, dt):
    keys = inputs.column(kind, 150_000, seed=17, dtype=dt)
    blob = oracle.compress(keys, eps, 16)
    idx = np.arange(keys.size, dtype=np.uint64)
    pred = oracle.predict(blob, idx)
    assert pred.tolist() == R.predictions(R.parse(blob))
    bits = 8 * keys.itemsize
    diff = (keys.astype(object) - pred.astype(object)) % (1 << bits)
    diff = np.array([d - (1 << bits) if d >= 1 << (bits - 1) else d for d in diff.tolist()])
    assert np.abs(diff).max() <= eps
    # an anchor predicts itself exactly (residual 0)
    starts = [s for (_, s, _) in R.segments(R.parse(blob))]
    assert np.array_equal(pred[starts], keys[starts])


def test_quantile_index_is_floor_n_k_over_q():
    for n in (1, 2, 7, 1000, 2**40 + 3):
        for q in (1, 2, 3, 4, 100, 2**20):
            for k in (0, 1, q // 3, q // 2, q - 1, q):
                if k < 0 or k > q:
                    continue
                want = (n * k) // q
                assert oracle.quantile_index(n, k, q) == (want if want < n else n - 1)
    # the median of an odd count is the middle key; k = q is the maximum
    assert oracle.quantile_index(5, 1, 2) == 2 and oracle.quantile_index(5, 2, 2) == 4
