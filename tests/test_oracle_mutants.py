"""The pins have teeth: each plausible mistake planted in a copy of the oracle
(compiled on the CPU into a temporary library) must fail at least one pin.

The planted mistakes cover the places a reading of the paper can go wrong: a
dropped term in the cone bounds (Def. 2), the slope tie-break, the cone reset at
a new anchor, the residual width, the zigzag sign, the residual bit position, the
segment boundary, and the chunk restart.
"""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2412_10770_gb300 import inputs
from test_oracle_pins import _tiny_cases, check_greedy, check_invariants

SRC = os.path.join(os.path.dirname(oracle.__file__), "lc_oracle.c")
HDR = os.path.join(os.path.dirname(oracle.__file__), "lc_oracle.h")

MUTANTS = {
    "hi_bound_drops_minus_one": ("(D + (i128)eps + 1) * TWO32 - 1, d)", "(D + (i128)eps + 1) * TWO32, d)"),
    "lo_bound_floor_not_ceil": ("i128 lo = ceil_div(", "i128 lo = floor_div("),
    "slope_quarter_not_midpoint": ("LO + ((HI - LO) >> 1)", "LO + ((HI - LO) >> 2)"),
    "cone_not_reset_after_close": ("s = i;\n        LO = INT64_MIN;\n", "s = i;\n"),
    "width_one_bit_short": ("g.width = bit_length(zmax);", "g.width = bit_length(zmax >> 1);"),
    "zigzag_sign_dropped": ("(uint64_t)(-(r + 1)) * 2u + 1u", "(uint64_t)(-(r + 1)) * 2u"),
    "pack_position_off_by_one": ("g->bitoff + (uint64_t)g->width * (t - 1);",
                                 "g->bitoff + (uint64_t)g->width * t;"),
    "eps_off_by_one": ("i128 lo = ceil_div((D - (i128)eps)", "i128 lo = ceil_div((D - (i128)eps - 1)"),
    "chunks_do_not_restart": ("ch[c].key_end = (c + 1) * cs < n ? (c + 1) * cs : n;",
                              "ch[c].key_end = n;"),
}


def _pin_suite():
    for keys, eps in _tiny_cases()[:30]:
        blob = oracle.compress(keys, eps, 8)
        check_invariants(keys, eps, blob)
        check_greedy(keys, eps, blob)
    keys = inputs.lognormal_gaps(3000, seed=4)
    for eps in (0, 1, 15):
        blob = oracle.compress(keys, eps, 8)
        assert np.array_equal(oracle.decode(blob), keys)
        check_invariants(keys, eps, blob)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    (tmp_path / "lc_oracle.c").write_text(src.replace(old, new))
    shutil.copy(HDR, tmp_path / "lc_oracle.h")
    lib = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-o", lib,
                           str(tmp_path / "lc_oracle.c")])
    saved = oracle._L()
    oracle._lib = oracle.bind(lib)
    try:
        with pytest.raises((AssertionError, oracle.OracleError)):
            _pin_suite()
    finally:
        oracle._lib = saved


def test_unmutated_oracle_passes_the_same_suite():
    _pin_suite()
