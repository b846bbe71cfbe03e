"""Plant mistakes in a copy of the oracle (on the CPU) and check that the pins
catch each one: a dropped bias, a transposed weight index, a reversed digit
order, a missing clip, "at least one" instead of "exactly one" in SS-Cover, a
sign error in the sigmoid, hidden layers left linear, and in the literal of
Eq. 11 a reversed comparison or a dropped tie band."""
import ctypes
import os
import subprocess

import pytest

import oracle
from oracle import oracle as orc_mod
import test_oracle_pins as pins
import test_oracle_threshold as thr

MUTANTS = {
    "dropped_bias": ("double u = acc + (double)b[i];", "double u = acc;"),
    "transposed_W": ("acc += (double)W[(size_t)i * n_in + j] * in[j];",
                     "acc += (double)W[(size_t)j * n_out + i] * in[j];"),
    "digit_order": ("for (int p = s - 1; p >= 0; p--) {\n        d[p]",
                    "for (int p = 0; p < s; p++) {\n        d[p]"),
    "no_clip_high": ("if (v > 255) v = 255;", ""),
    "ss_at_least_one": ("int certain = (n_tie == 0 && n_flip == 1 && j == only);",
                        "int certain = (n_tie == 0 && n_flip >= 1 && j == only);"),
    "sigmoid_sign": ("return 1.0 / (1.0 + exp(-u));", "return 1.0 / (1.0 + exp(u));"),
    "hidden_not_activated": ("out[i] = (l + 1 < net->L) ? orc_activation(net->act, u) : u;",
                             "out[i] = u;"),
    "threshold_reversed": ("if (y[D] - V <= -tau) lit_d = 1;", "if (y[D] - V >= tau) lit_d = 1;"),
    "threshold_no_tie_band": ("else if (y[i] - V > -tau && any == 0) any = 2;", ""),
}

PINS = [
    lambda: pins.test_digits_follow_lexicographic_order(3, 1),
    pins.test_table1_forward_matches_printed_values,
    pins.test_table1_ss_cover_ex1_ex2,
    pins.test_table2_ss_cover_and_eq3_fraction,
    pins.test_hand_222_fixture,
    pins.test_clipped_duplicates_share_verdicts,
    pins.test_affine_single_pixel_closed_form,
    lambda: pins.test_bruteforce_high_precision(*pins.BRUTE[0]),
    lambda: pins.test_bruteforce_high_precision(*pins.BRUTE[4]),
    thr.test_literal_hand_cases,
    lambda: thr.test_exact_bruteforce(23, 1.5),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(orc_mod.SRC).read()
    assert old in src, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", str(so),
                           str(path), "-lm"])
    saved = orc_mod._lib
    orc_mod._lib = orc_mod.configure(ctypes.CDLL(os.fspath(so)))
    failed = []
    try:
        for pin in PINS:
            try:
                pin()
            except (AssertionError, ValueError):
                failed.append(pin)
                break
    finally:
        orc_mod._lib = saved
    assert failed, f"no pin caught mutant {name}"
