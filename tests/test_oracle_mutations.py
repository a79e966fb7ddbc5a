"""The pins of the oracle catch plausible mistakes.

Each planted mistake (MUTATION m in oracle/sl_oracle.c: a wrong sign, index,
factor, operand order or a missing special case) is switched on in the C
oracle in turn, and at least one pin of tests/test_oracle_pins.py must then
fail; with none planted every pin used here passes.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import test_oracle_pins as P

# the pins, each with fixed parameters (a failing assertion or an error both count)
PINS = {
    "gauss_numpy": lambda: [P.test_gauss_legendre_matches_numpy(n) for n in (3, 5, 12)],
    "gauss_monomials": lambda: [P.test_gauss_legendre_exact_on_monomials(n) for n in (4, 12)],
    "legendre_numpy": P.test_legendre_matches_numpy,
    "ab_symbolic": lambda: [P.test_ab_matches_exact_symbolic_integrals(k, a)
                            for k in (1, 2) for a in (Fraction(3, 8), Fraction(1, 3))],
    "k0_donor_cell": lambda: [P.test_k0_is_donor_cell(a) for a in (0.1, 0.37)],
    "ab_identities": lambda: [P.test_ab_identities(k) for k in (1, 2)],
    "shift_split": P.test_shift_split,
    "integer_roll": lambda: [P.test_integer_shift_is_bit_exact_roll(n, d, sd, k)
                             for (n, d, sd) in [((7,), 0, -1), ((5, 3), 1, 0)] for k in (0, 2)],
    "full_period": P.test_full_period_shift_returns_bit_exactly,
    "bruteforce": lambda: [P.test_bruteforce_projection_agrees(n, k) for (n, k) in [((8,), 1), ((5, 4), 2)]],
    "mass_l2": P.test_mass_conserved_and_l2_nonincreasing,
    "convergence": lambda: P.test_convergence_order_vs_exact_translation(1, 1.9),
    "projection_polynomials": P.test_projection_of_polynomials_is_exact,
    "projection_tensor_order": P.test_projection_tensor_order_in_several_dimensions,
    "projection_quadrature": P.test_projection_matches_adaptive_quadrature,
    "maxwellian_mass": P.test_mass_of_maxwellian_workload_closed_form,
    "sample_after": P.test_sample_after_matches_full_grid,
    "nodal_bruteforce": lambda: P.test_nodal_sweep_agrees_with_bruteforce((5, 4), 1),
    "nodal_round_trip_mass": P.test_nodal_round_trip_and_mass,
    "nodal_free_streaming": lambda: P.test_nodal_sweep_converges_to_free_streaming(1),
}

MUTATIONS = {
    1: "Legendre recurrence divides by n instead of n + 1",
    2: "Gauss weight with |P_n'| instead of P_n'^2",
    3: "shift split truncates toward zero instead of flooring",
    4: "A integrand evaluates the source polynomial at xi + 2 alpha",
    5: "B integrand evaluates the source polynomial at eta - 2 + 2 alpha",
    6: "A normalised by (2j + 1) instead of (2j + 1) / 2",
    7: "sweep applies the transposed matrices",
    8: "sweep swaps A and B",
    9: "second source cell i - sigma + 1 instead of i - sigma - 1",
    10: "first source cell i + sigma instead of i - sigma",
    11: "sweep drops the B term",
    12: "mass without the cell volume",
    13: "projection normalised by (2j + 1) instead of (2j + 1) / 2",
    14: "projection maps the nodes with h instead of h / 2",
    15: "projection reverses the tensor index order",
    16: "alpha = 0 not an exact copy",
    17: "brute-force sweep puts the break point one half cell off",
    18: "per-cell update swaps its source cells",
    19: "shift split keeps alpha = 1 instead of moving to the next cell",
    20: "nodal sweep: node velocity at eta instead of eta / 2 from the v-cell centre",
    21: "nodal sweep: back-transform without the 1/2 of (2 jv + 1) / 2",
    22: "nodal sweep: values taken at the mirrored node",
}


def _failing_pins():
    failed = []
    for name, pin in PINS.items():
        try:
            pin()
        except Exception:    # AssertionError, or an error raised by the mutated oracle
            failed.append(name)
    return failed


def test_all_pins_pass_without_a_planted_mistake():
    with O.planted_mistake(0):
        assert _failing_pins() == []


@pytest.mark.parametrize("m", sorted(MUTATIONS))
def test_each_planted_mistake_fails_a_pin(m):
    with O.planted_mistake(m):
        failed = _failing_pins()
    assert failed, f"no pin catches mutation {m}: {MUTATIONS[m]}"
    assert O.lib().or_get_mutation() == 0


# Planted mistakes in the host-side split-storage mask ("# double",
# Sec. III-A): each replaces oracle.fp64_coefficients, and the pins of the
# split stores must catch it.
def _mask_from(test):
    def mask(k, ndim, ndouble):
        o = k + 1
        m = np.zeros(o ** ndim, dtype=bool)
        for J in range(o ** ndim):
            digits = [(J // o ** d) % o for d in range(ndim)]
            m[J] = test(digits, ndouble)
        return m
    return mask


MASK_MUTATIONS = {
    "index bound j_m <= q": _mask_from(lambda j, q: all(x <= q for x in j)),
    "only dimension 0 tested": _mask_from(lambda j, q: j[0] < q),
    "any index below q instead of every": _mask_from(lambda j, q: any(x < q for x in j)),
    "sum of the indices below q": _mask_from(lambda j, q: sum(j) < q),
}
SPLIT_PINS = {
    "memorydown": P.test_storage_bytes_reproduce_the_printed_memory_reductions,
    "mask_structure": lambda: [P.test_fp64_coefficients_structure(k, d) for (k, d) in [(1, 1), (3, 1), (2, 2)]],
    "round_storage": P.test_round_storage_and_stored_sweeps,
}


def test_split_pins_pass_and_the_unmutated_mask_is_the_reading():
    for pin in SPLIT_PINS.values():
        pin()
    for k, d in [(1, 1), (2, 2), (3, 3)]:
        for q in range(k + 2):
            assert np.array_equal(_mask_from(lambda j, q: all(x < q for x in j))(k, d, q),
                                  O.fp64_coefficients(k, d, q))


@pytest.mark.parametrize("name", sorted(MASK_MUTATIONS))
def test_each_planted_mask_mistake_fails_a_split_pin(name, monkeypatch):
    monkeypatch.setattr(O, "fp64_coefficients", MASK_MUTATIONS[name])
    failed = []
    for pin_name, pin in SPLIT_PINS.items():
        try:
            pin()
        except Exception:
            failed.append(pin_name)
    assert failed, f"no pin catches the mask mistake: {name}"
