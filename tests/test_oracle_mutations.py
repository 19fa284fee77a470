"""Planted mistakes: each mutant of the C oracle (a dropped term, a loosened
tie-break, a wrong constant, transposed cell axes, a wrong normaliser, a
loosened comparison) must be caught by at least one pin.  Mutants are compiled from a text-edited copy in a
temporary directory; the committed oracle is never touched."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import test_oracle_core as pins
from tests import test_oracle_frontier_rules as rules
from tests import test_oracle_knn as knn
from tests import test_oracle_rho as rho

MUTANTS = {
    "drop_dz": ("s = s + dz * dz;", "s = s;"),
    "tie_le": ("if (D < b1) {", "if (D <= b1) {"),
    "frontier_2eps": ("float rhs = 4.0f * eps + tau;", "float rhs = 2.0f * eps + tau;"),
    "cells_transposed": ("(k[2] * g + k[1]) * g + k[0]", "(k[0] * g + k[1]) * g + k[2]"),
    "entropy_norm_m": ("H = s / log((double)C);", "H = s / log((double)m);"),
    "eps_first_point": ("if (D > m)\n            m = D;", "if (i == 0)\n            m = D;"),
    "point_budget_halved": ("float rhs = 2.0f * (disp[i] + eps) + tau;", "float rhs = (disp[i] + eps) + tau;"),
    "point_budget_own_only": ("float rhs = 2.0f * (disp[i] + eps) + tau;", "float rhs = 2.0f * disp[i] + tau;"),
    "rho_no_factor": ("out[i] = (uint8_t)(2.0f * disp[i] > c);", "out[i] = (uint8_t)(disp[i] > c);"),
    "rho_not_strict": ("out[i] = (uint8_t)(2.0f * disp[i] > c);", "out[i] = (uint8_t)(2.0f * disp[i] >= c);"),
    "rho_squared_clearance": ("float c = sqrtf(d2sq[i]) - sqrtf(d1sq[i]);", "float c = d2sq[i] - d1sq[i];"),
    "knn_tie_le": ("while (s > 0 && D < bd[s - 1]) {", "while (s > 0 && D <= bd[s - 1]) {"),
    "knn_keeps_equal_last": ("if (have == m && !(D < bd[m - 1]))", "if (have == m && D > bd[m - 1])"),
}

PIN_CALLS = [
    lambda o: pins.test_top2_matches_exact_rational_bruteforce(o, 17, 3),
    lambda o: pins.test_hand_enumerated_square(),
    lambda o: pins.test_duplicates_allowed(o),
    lambda o: pins.test_lattice_known_equal_distances(o, 3),
    lambda o: pins.test_tightness_construction_thm_a1(o, 2, ("i", "a", "k")),
    lambda o: pins.test_tightness_construction_thm_a1(o, 3, ("i", "k", "a")),
    lambda o: pins.test_cells_dyadic_and_clamped(o),
    lambda o: pins.test_entropy_closed_forms(o),
    lambda o: pins.test_eps_is_max_displacement(o),
    lambda o: rules.test_point_and_clock_rules_never_miss("adversarial_crossing", 3),
    lambda o: rules.test_point_and_clock_rules_never_miss("clustered_drift", 2),
    lambda o: rules.test_point_rule_leaves_out_a_static_point_with_clearance_three_eps(),
    lambda o: rho.test_rho_dyadic_closed_forms(),
    lambda o: rho.test_rho_step_level_dyadic(),
    lambda o: knn.test_knn_matches_exact_rational_bruteforce(17, 3, 2),
    lambda o: knn.test_knn_matches_a_lexsort_of_the_distance_matrix(3),
    lambda o: knn.test_knn_tightness_at_rank_three(True),
    lambda o: knn.test_knn_tightness_at_rank_three(False),
]


def _build_mutant(tmp_path, name):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(so), str(path), "-lm"], check=True)
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name, monkeypatch):
    so = _build_mutant(tmp_path, name)
    saved_lib, saved_path = oracle._lib, oracle._LIB
    try:
        oracle._lib = None
        monkeypatch.setattr(oracle, "_LIB", so)
        monkeypatch.setattr(oracle, "build", lambda force=False: so)
        caught = 0
        for call in PIN_CALLS:
            try:
                call(oracle)
            except AssertionError:
                caught += 1
        assert caught > 0, f"mutant {name} passed every pin"
    finally:
        oracle._lib = saved_lib


def test_unmutated_passes_all_pins():
    for call in PIN_CALLS:
        call(oracle)
