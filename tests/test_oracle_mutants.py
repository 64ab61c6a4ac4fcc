"""Planted mistakes in the oracle (on the CPU) must each fail a pin.

Every mutant is a one-token slip of the kind that could plausibly be made
when writing the oracle -- a dropped term, a wrong sign or index, a
transposed operand, an inverted comparison.  The pins of
``test_oracle_pins.py`` are run against a compiled copy of the mutated
source; at least one of them has to fail, otherwise the pins would not be
pinning that part of the oracle.
"""
import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = {
    "wrong_root_sign": ("(ux + uy + sqrt(", "(ux + uy - sqrt("),
    "dropped_factor_2": ("2.0 * f * f - d * d", "f * f - d * d"),
    "inverted_branch": ("if (fabs(d) < f) {", "if (fabs(d) > f) {"),
    "dropped_one_sided_term": ("    return lo + f;\n}", "    return lo;\n}"),
    "halved_root": ("return (ux + uy + sqrt(2.0 * f * f - d * d)) / 2.0;",
                    "return (ux + uy + sqrt(2.0 * f * f - d * d)) / 4.0;"),
    "wrong_neighbour_index": ("nb(V, nx, ny, i, j + 1)", "nb(V, nx, ny, i + 1, j + 1)"),
    "missing_quadrant": ("quadrant_update(uw, us, f)", "quadrant_update(uw, un, f)"),
    "transposed_speed": ("h / Fk", "Fk / h"),
    "duplicate_source_max": ("sq[s] < p->q[k]", "sq[s] > p->q[k]"),
    "fmm_keeps_larger": ("    if (t < V[k]) {\n        V[k] = t;\n        if (label",
                         "    if (t > V[k]) {\n        V[k] = t;\n        if (label"),
    "outside_is_zero": ("        return INFINITY;\n    return V[(size_t)j * nx + i];",
                        "        return 0.0;\n    return V[(size_t)j * nx + i];"),
}

PINS = [
    pins.test_local_update_solves_eik_discr_exactly,
    pins.test_local_update_special_values,
    pins.test_corner_source_closed_form,
    lambda o: pins.test_one_dimensional_reduction(o, 1),
    lambda o: pins.test_one_dimensional_reduction(o, 2),
    pins.test_unreachable_and_obstacles,
    pins.test_duplicate_sources_keep_min,
    pins.test_distance_function_converges_first_order,
    pins.test_d4_symmetry,
    pins.test_scaling_and_shift,
]


def _source():
    with open(oracle.SOURCE) as fh:
        return fh.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutant = oracle.Oracle.from_source(src.replace(old, new))
    caught = []
    for pin in PINS:
        try:
            pin(mutant)
        except Exception as e:  # AssertionError, OracleError, ...
            caught.append((getattr(pin, "__name__", "pin"), type(e).__name__))
            break
    assert caught, f"no pin fails on mutant {name}"


def test_unmutated_source_passes_the_same_pins():
    clean = oracle.Oracle.from_source(_source())
    for pin in PINS:
        pin(clean)
