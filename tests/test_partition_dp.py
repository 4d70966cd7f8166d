"""The per-partition eps search (Sec. IV-A, Fig. 5) at chunk granularity:
the dynamic program equals a brute force over every partitioning of a few
chunks with every eps assignment, and never costs more than the best single
eps plus one partition's overhead.  No GPU."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from paper_2412_10770_gb300.tune import best_partition


def _brute(costs, switch):
    E, C = costs.shape
    best = np.inf
    for choice in itertools.product(range(E), repeat=C):
        parts = 1 + sum(choice[c] != choice[c - 1] for c in range(1, C))
        cost = sum(costs[choice[c], c] for c in range(C)) + switch * parts
        best = min(best, cost)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_dp_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    E, C = int(rng.integers(1, 4)), int(rng.integers(1, 7))
    costs = rng.integers(0, 60, size=(E, C)).astype(np.float64)
    switch = float(rng.integers(0, 40))
    choice, total = best_partition(costs, switch)
    parts = 1 + int(np.sum(choice[1:] != choice[:-1]))
    assert total == pytest.approx(costs[choice, np.arange(C)].sum() + switch * parts)
    assert total == pytest.approx(_brute(costs, switch))


def test_dp_is_never_worse_than_one_eps():
    rng = np.random.default_rng(99)
    costs = rng.random((7, 300)) * 1000
    _, total = best_partition(costs, 25.0)
    assert total <= costs.sum(axis=1).min() + 25.0 + 1e-9


def test_switches_pay_off_only_when_chunks_differ():
    # two regimes: eps 0 best on the first half, eps 1 on the second
    costs = np.array([[1.0] * 5 + [100.0] * 5, [100.0] * 5 + [1.0] * 5])
    choice, total = best_partition(costs, 10.0)
    assert choice.tolist() == [0] * 5 + [1] * 5 and total == pytest.approx(10 + 20)
    choice, _ = best_partition(costs, 1e6)  # too dear to switch: one partition
    assert len(set(choice.tolist())) == 1
