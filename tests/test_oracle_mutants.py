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
SRC_FOR = os.path.join(os.path.dirname(oracle.__file__), "for_bp128.c")
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
# mistakes planted in the jump fit (fewest segments)
MUTANTS.update({
    "jump_takes_the_greedy_anchor": ("            nx = best;\n", "            nx = r[a - b];\n"),
    "jump_picks_the_nearest_reach": ("                if (r[q - b] > bk) {", "                if (r[q - b] < bk) {"),
})
JUMP_MUTANTS = {"jump_takes_the_greedy_anchor", "jump_picks_the_nearest_reach"}
# mistakes planted in the FOR-delta bp128 baseline's reference (for_bp128.c)
FOR_MUTANTS = {
    "for_first_gap_not_zero": ("if (i == 0 || k >= n) return 0;", "if (k == 0 || k >= n) return 0;"),
    "for_width_one_bit_short": ("width[b] = fo_bitlen(m);", "width[b] = fo_bitlen(m >> 1);"),
    "for_gap_bit_position_shifted": ("const uint64_t bit = (uint64_t)i * w + t; /* bit of the block payload */",
                                     "const uint64_t bit = (uint64_t)i * w + t + 1; /* bit of the block payload */"),
    "for_block_words_not_4w": ("word += 4 * (uint64_t)w;\n    }\n    free(width);",
                               "word += 3 * (uint64_t)w;\n    }\n    free(width);"),
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


def _jump_pin_suite():
    from test_jump_pins import _jump_cases, test_jump_reaches_the_anchored_optimum_on_short_segments

    for case in range(len(_jump_cases())):
        test_jump_reaches_the_anchored_optimum_on_short_segments(case)


def _for_pin_suite():
    from test_for_pins import _cases, test_reference_roundtrips_and_matches_closed_form

    for name, keys in _cases():
        test_reference_roundtrips_and_matches_closed_form(name, keys)


def _mutant_lib(tmp_path, lc_src: str, for_src: str) -> str:
    (tmp_path / "lc_oracle.c").write_text(lc_src)
    (tmp_path / "for_bp128.c").write_text(for_src)
    shutil.copy(HDR, tmp_path / "lc_oracle.h")
    lib = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-o", lib,
                           str(tmp_path / "lc_oracle.c"), str(tmp_path / "for_bp128.c")])
    return lib


@pytest.mark.parametrize("name", sorted(MUTANTS) + sorted(FOR_MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    lc_src, for_src = open(SRC).read(), open(SRC_FOR).read()
    if name in MUTANTS:
        old, new = MUTANTS[name]
        assert lc_src.count(old) == 1, f"mutation site for {name} not found exactly once"
        lc_src, suite = lc_src.replace(old, new), (_jump_pin_suite if name in JUMP_MUTANTS else _pin_suite)
    else:
        old, new = FOR_MUTANTS[name]
        assert for_src.count(old) == 1, f"mutation site for {name} not found exactly once"
        for_src, suite = for_src.replace(old, new), _for_pin_suite
    lib = _mutant_lib(tmp_path, lc_src, for_src)
    saved = oracle._L()
    oracle._lib = oracle.bind(lib)
    try:
        with pytest.raises((AssertionError, oracle.OracleError)):
            suite()
    finally:
        oracle._lib = saved


def test_unmutated_oracle_passes_the_same_suite():
    _pin_suite()
    _for_pin_suite()
