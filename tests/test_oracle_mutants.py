"""The pins detect plausible mistakes in the oracle.

Each case compiles the oracle with one deliberate error (on the CPU, in a
temporary directory) and checks that at least one of the named pins of
tests/test_oracle_pins.py fails against it; the unmodified build passes them
(the pins themselves run in that file).  Planted errors: a dropped factor in
the force law, the wrong sign of the energy shift, no minimum image, a missing
layer of neighbour cells, a dropped term of the velocity update, a dropped
term of the position update, a virial without its r^2 factor, a strict
cutoff instead of the inclusive one, a mirror wall that reflects positions but
not velocities, pairs that still meet across the mirror walls, a thermostat
that forgets its own previous scaling, a thermostat factor without its
square root, slice profiles that count whole pair energies, and a subset
force call (the one behind the full-size sampled parity tests) that
evaluates the neighbouring atom instead of the one asked for.
"""
import os

import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_nvt as nvt
from tests import test_oracle_walls as walls

CASES = {
    1: [lambda: pins.test_pair_law_closed_form(1.0)],
    2: [pins.test_pair_law_special_points],
    3: [lambda: pins.test_dimer_across_periodic_boundary("brute")],
    4: [lambda: pins.test_bruteforce_equals_cell_list(5, 0.15)],
    5: [pins.test_dimer_trajectory_matches_ode_solver, pins.test_nve_run_conserves_momentum_and_energy],
    6: [pins.test_dimer_trajectory_matches_ode_solver, pins.test_nve_run_conserves_momentum_and_energy],
    7: [pins.test_fcc_lattice_sums],
    8: [pins.test_pair_law_special_points],
    9: [walls.test_free_flight_into_a_wall_reflects],
    10: [walls.test_no_pair_across_the_walls],
    11: [nvt.test_ideal_gas_reaches_the_target_in_one_scaling],
    12: [lambda: nvt.test_fcc_profiles_are_the_lattice_sums()],
    13: [nvt.test_ideal_gas_reaches_the_target_in_one_scaling],
    14: [pins.test_subset_matches_full],
}


@pytest.mark.parametrize("mutant", sorted(CASES))
def test_pins_catch_planted_mistake(mutant, tmp_path):
    lib = oracle.build_variant(os.path.join(tmp_path, f"mutant{mutant}.so"), [f"ORACLE_MUTANT={mutant}"])
    prev = oracle.use_library(lib)
    try:
        caught = 0
        for pin in CASES[mutant]:
            try:
                pin()
            except (AssertionError, RuntimeError):
                caught += 1
        assert caught >= 1, f"no pin detects planted mistake {mutant}"
    finally:
        oracle.use_library(None)
        del prev


def test_unmodified_oracle_passes_the_same_pins():
    for pins_of_case in CASES.values():
        for pin in pins_of_case:
            pin()
