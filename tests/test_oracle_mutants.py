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


# ---------------------------------------------------------------- cell methods
CELL_MUTANTS = {
    # HCM that stops after one sweep is no longer exact
    "hcm_single_sweep": ("            } while (changed);", "            } while (0);"),
    # a source on a cell border that never activates across it leaves cells unreached
    "no_first_removal_activation": ("if ((ch || (first && p.src[qb])) && vb < U[qa] && !p.src[qa]) act = 1;",
                                    "if (ch && vb < U[qa] && !p.src[qa]) act = 1;"),
}
# mistakes that keep HCM exact and FHCM an upper bound, caught by the
# paper's printed cell-method statistics (slow)
CELL_MUTANTS_TABLE = {
    "fhcm_one_flag_when_not_monotone": ("                else set = (1 << up) | (1 << down);",
                                        "                else set = 1 << up;"),
    "sweep_i_order_swapped": ("    int i_up = (dir == 0 || dir == 1), j_up = (dir == 0 || dir == 3);",
                              "    int i_up = (dir == 2 || dir == 3), j_up = (dir == 0 || dir == 3);"),
    "monotone_flags_swapped": ("                if (noninc) { set = 1 << down; ++mono_ok; }",
                               "                if (noninc) { set = 1 << up; ++mono_ok; }"),
}


def _caught_by(mutant, pin_fns):
    for pin in pin_fns:
        try:
            pin(mutant)
        except (AssertionError, oracle.OracleError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(CELL_MUTANTS))
def test_cell_pins_catch_planted_mistake(name):
    old, new = CELL_MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutant = oracle.Oracle.from_source(src.replace(old, new))
    assert _caught_by(mutant, [pins.test_hcm_is_exact_and_fhcm_an_upper_bound]), name


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(CELL_MUTANTS_TABLE))
def test_cell_table_pin_catches_planted_mistake(name):
    old, new = CELL_MUTANTS_TABLE[name]
    src = _source()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutant = oracle.Oracle.from_source(src.replace(old, new))
    assert _caught_by(mutant, [pins.test_cell_methods_reproduce_tab_sinu_1]), name


# ---------------------------------------------------------------- FMSM
FMSM_MUTANTS = {
    # sweep-directional update from the neighbours ahead of the sweep
    "fmsm_front_neighbour": ("double ux = nb(V, nx, ny, i_up ? i - 1 : i + 1, j);",
                             "double ux = nb(V, nx, ny, i_up ? i + 1 : i - 1, j);"),
    # a direction whenever one of its sides was accepted before
    "fmsm_either_side": ("            if (xs[d] && ys[d]) dirs |= 1 << d;",
                         "            if (xs[d] || ys[d]) dirs |= 1 << d;"),
    # exit-set cells treated like the others (no Alg. FSM)
    "fmsm_exit_cells_not_swept": ("        if (pc.src[c]) {\n            /* Alg. FSM on the cell",
                                  "        if (0 && pc.src[c]) {\n            /* Alg. FSM on the cell"),
    # earlier and later neighbours swapped
    "fmsm_later_as_earlier": ("const int w = cx > 0 && rank[c - 1] < e,",
                              "const int w = cx > 0 && rank[c - 1] > e,"),
    # the coarse speed from the node k/2 into the cell, not the centre
    "fmsm_coarse_speed_corner": ("Fc[cy * cxn + cx] = 0.25 * (((a + b) + c) + d);",
                                 "Fc[cy * cxn + cx] = d;"),
}
FMSM_PINS = [pins.test_fmsm_checkerboard_acceptance_order, pins.test_fmsm_one_node_cells_are_fast_marching,
             pins.test_fmsm_is_an_upper_bound, pins.test_fmsm_reproduces_tab_const]
# caught only by the paper's sin20 table (slow)
FMSM_MUTANTS_TABLE = {"fmsm_coarse_speed_corner"}


@pytest.mark.parametrize("name", sorted(set(FMSM_MUTANTS) - FMSM_MUTANTS_TABLE))
def test_fmsm_pins_catch_planted_mistake(name):
    old, new = FMSM_MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutant = oracle.Oracle.from_source(src.replace(old, new))
    assert _caught_by(mutant, FMSM_PINS), name


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(FMSM_MUTANTS_TABLE))
def test_fmsm_table_pin_catches_planted_mistake(name):
    old, new = FMSM_MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutant = oracle.Oracle.from_source(src.replace(old, new))
    assert _caught_by(mutant, [pins.test_fmsm_reproduces_tab_sinu_1]), name


# ---------------------------------------------------------------- locking (LSM)
LSM_MUTANTS = {
    # a decrease unlocks the smaller neighbours instead of the larger ones
    "lsm_unlocks_smaller": ("if (V[kn] > V[k] && !unl[kn] && !p->src[kn]) {",
                            "if (V[kn] < V[k] && !unl[kn] && !p->src[kn]) {"),
    # the east border of a cell is not unlocked at a removal
    "lsm_east_border_locked": ("(i == i1 - 1 && i1 < nx)", "(i == i1 - 1 && i1 > nx)"),
    # the source neighbours are unlocked on every removal but the first
    "lsm_source_neighbours_later": ("if (!u && first)", "if (!u && !first)"),
    # whole-grid LSM starts from the neighbours of the non-sources
    "lsm_starts_at_non_sources": ("            if (!p.src[(size_t)j * nx + i]) continue;\n            const int ni[4]",
                                  "            if (p.src[(size_t)j * nx + i]) continue;\n            const int ni[4]"),
}
LSM_PINS = [pins.test_lsm_matches_fsm_sweep_for_sweep, pins.test_hcm_with_locking_is_hcm]


@pytest.mark.parametrize("name", sorted(LSM_MUTANTS))
def test_lsm_pins_catch_planted_mistake(name):
    old, new = LSM_MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutant = oracle.Oracle.from_source(src.replace(old, new))
    assert _caught_by(mutant, LSM_PINS), name
