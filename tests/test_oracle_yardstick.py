"""The segmentation-quality yardstick of the oracle's greedy fit.

Sec. II-A measures a fit by its number of segments L; the fewest segments for
a bound eps is what an optimal (free-line) fit reaches.  On tiny inputs three
optima are computed here by brute force, none of them through the oracle:

* L*_free(eps): the fewest segments when every segment may take any real line
  f(i) = alpha + beta (i - start) with |K[i] - floor(f(i))| <= eps (Def. 2 with
  a free intercept and slope).  Feasibility of one run is a two-variable linear
  program, decided exactly in integers below.
* L*_anch(eps): the fewest anchored segments of the format (intercept = the
  run's first key, integer Q32 slope), by bisection on the definition.
* L_greedy(eps): the oracle's greedy (the segment count of its blob).

They must satisfy L*_free(eps) <= L*_anch(eps) <= L_greedy(eps) (an anchored Q32
line is one of the free lines; the greedy is one anchored segmentation) and
L_greedy(2 eps + 2) <= L*_free(eps): a free line of one optimal segment,
re-anchored at any key of it, keeps every floor within 2 eps + 1 of the keys,
and rounding its slope to Q32 moves a floor by at most one more; the greedy
at 2 eps + 2 therefore reaches at least as far as each optimal segment from
every anchor inside it, so by induction its k-th anchor is never before the
optimum's.  A greedy that closed segments early (a wrong cone bound, a dropped
key) breaks the last inequality; one that accepted a run it should not have
breaks L*_anch <= L_greedy.
"""
from __future__ import annotations

import numpy as np
import pytest

import lcf_reader as R
import oracle
from test_oracle_pins import _anchored_optimum


@pytest.fixture(scope="module", autouse=True)
def _oracle():
    oracle.build()


def _free_feasible(K, eps):
    """Is there a real (alpha, beta) with K[i] - eps <= alpha + beta i < K[i] + eps + 1
    for every i of the run (floor(f(i)) within eps of K[i])?

    For a fixed beta, alpha exists iff h(beta) = min_j (U_j - beta j) -
    max_i (L_i - beta i) > 0 (U = K + eps + 1, L = K - eps).  h is the minimum
    of the lines c_e - e beta over e = j - i, with c_e the least U_j - L_i at
    that offset: concave, piecewise linear, and -> -inf on both sides when the
    run has two keys or more.  Its maximum lies where a line of slope -e <= 0
    meets one of slope -e' >= 0, so h is evaluated there, at beta = p / q,
    exactly: q h(p / q) = min_e (c_e q - e p)."""
    n = len(K)
    if n <= 1:
        return True
    c = {}
    for j in range(n):
        for i in range(n):
            e = j - i
            v = (K[j] + eps + 1) - (K[i] - eps)
            if e not in c or v < c[e]:
                c[e] = v
    lines = sorted(c.items())
    for e1, c1 in lines:
        if e1 < 0:
            continue
        for e2, c2 in lines:
            if e2 > 0 or e2 == e1:
                continue
            p, q = c1 - c2, e1 - e2  # beta = p / q, q > 0
            if min(ce * q - e * p for e, ce in lines) > 0:
                return True
    return False


def _free_optimum(K, eps):
    n = len(K)
    best = [0] + [None] * n
    for e in range(1, n + 1):
        for s in range(e):
            if best[s] is not None and _free_feasible(K[s:e], eps):
                if best[e] is None or best[s] + 1 < best[e]:
                    best[e] = best[s] + 1
    return best[n]


def _greedy(K, eps):
    return R.parse(oracle.compress(np.array(K, dtype=np.uint64), eps, 8))["segments"]


def test_free_feasibility_on_hand_cases():
    # collinear keys fit one line for any eps
    assert _free_feasible([0, 3, 6, 9, 12], 0)
    # a kink of height 2 needs eps >= 1 under the floor model
    assert not _free_feasible([0, 0, 2], 0)
    assert _free_feasible([0, 0, 2], 1)
    # 0, 1, 1, 2 at eps 0: floor(i / 2 + 1 / 2) = 0, 1, 1, 2
    assert _free_feasible([0, 1, 1, 2], 0)
    # a zigzag 0, 5, 0 cannot be followed within eps 2
    assert not _free_feasible([0, 5, 0], 2)


@pytest.mark.parametrize("eps", [0, 1, 2, 4])
def test_greedy_between_the_optima(eps):
    rng = np.random.default_rng(100 + eps)
    strict = 0
    for trial in range(60):
        n = int(rng.integers(2, 11))
        K = [int(x) for x in np.sort(rng.integers(0, 65, size=n))]
        free = _free_optimum(K, eps)
        anch = _anchored_optimum(K, eps)
        greedy = _greedy(K, eps)
        assert free <= anch <= greedy, (K, eps, free, anch, greedy)
        assert _greedy(K, 2 * eps + 2) <= free, (K, eps, free)
        strict += free < anch
    assert strict > 0  # the free optimum is sometimes strictly better: the yardstick is not vacuous
