"""Mutation check of the oracle's pins: copies of the oracle are built with one known, plausible
mistake planted each (a wrong sign, a dropped term, a wrong divisor; see OR_PLANT in
oracle/isira_oracle.c), and the pins of tests/test_oracle_pins.py must fail on every one of them.
The unmodified oracle passes the same pins (that file).  CPU only."""
import shutil

import pytest

import oracle
import synthgraphs as sg
from tests import closed_forms as cf
from tests import test_oracle_pins as pins
from tests import test_oracle_weighted as wpins

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc is needed to build the variants")

# planted mistake -> the pin that must catch it
MUTANTS = {
    1: ("neighbour term of L x added instead of subtracted (Eq. 1.1)",
        lambda: pins.test_laplacian_apply_and_invariants(sg.grid2d(4, 5))),
    2: ("wrong sign of the Jacobi rotation applied to the eigenvectors",
        lambda: pins.test_sym_eig_matches_lapack(7)),
    3: ("rank-one term (sigma/n) 1 1^T dropped from the trimmed operator (Theorem 2.6)",
        lambda: pins.test_theorem_2_6_trimmed_solution_solves_singular_system(5, 0, 0.35)),
    4: ("deflation term delta V V^T with the wrong sign (Eq. 2.14)",
        lambda: pins.test_theorem_2_6_trimmed_solution_solves_singular_system(5, 3, 0.8)),
    5: ("back-map shift divided by n - 1 instead of n (Eq. 2.5)",
        lambda: pins.test_backmap_is_orthogonal_to_ones_and_places_zero()),
    6: ("wrong sign in the MINRES Givens recurrence",
        lambda: pins.test_minres_matches_direct_solve("spd")),
    7: ("SMW correction of the preconditioner with the wrong sign (Eq. 3.6)",
        lambda: pins.test_preconditioner_smw_inverts_its_matrix()),
    8: ("the lock records the second Ritz value instead of the first (Algorithm 2, lock step)",
        lambda: pins.test_isira_closed_forms(sg.path(40), cf.path(40), 6)),
    9: ("the restart keeps the q largest Ritz vectors instead of the q smallest (Algorithm 2)",
        lambda: pins.test_isira_restart_branch_keeps_the_closed_form_pairs()),
    10: ("the diagonal of the weighted Laplacian counts edges instead of summing weights",
         lambda: wpins.test_weighted_laplacian_definition(sg.grid2d(4, 5))),
}


@pytest.mark.parametrize("plant", sorted(MUTANTS))
def test_pin_catches_planted_mistake(plant, tmp_path):
    what, pin = MUTANTS[plant]
    lib = oracle.build_variant(str(tmp_path / f"liboracle_plant{plant}.so"), plant)
    with oracle.using_library(lib):
        with pytest.raises(AssertionError):
            pin()


def test_unplanted_copy_passes_the_same_pins(tmp_path):
    """The variant build itself (plant 0) changes nothing: every pin above passes on it."""
    lib = oracle.build_variant(str(tmp_path / "liboracle_plant0.so"), 0)
    with oracle.using_library(lib):
        for _, pin in MUTANTS.values():
            pin()
