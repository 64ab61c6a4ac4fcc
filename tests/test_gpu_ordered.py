"""The value-ordered round-free schedule (EIK_SCHED_ORDERED: requested cells
wait in buckets of the value their activation proposes, eq. cell_value --
Dial's buckets of Sec. 2 without rounds; warps take cells from the buckets
within a window of the lowest one still counting a cell) against the oracle,
node by node, in every arithmetic mode it runs: FP64, the FP32 pass and the
double-float pass of FP32_REFINE.  Cell sizes 8 to 64, windows from the
lowest bucket alone to all 32, narrow and wide buckets, single grids,
batches, the full-size benchmark grids, the degenerate inputs, the deadline
path, and the update efficiency the order buys over first-in first-out.

By Theorem convergence any removal order reaches the unique solution of
eq. Eik_discr; tolerances are those of the other parity tests (FP64
1e-12 * max|u| with +inf at the same nodes; FP32_REFINE: error within the
certificate, certificate <= 1e-5, error <= 5e-8 on grids with h <= 1/64).
On coarser grids the FP32 two-sided increment, whose rounding error is a few
units of 2^-24 of f = h/F, weighs more against max|u|: the empirical bound
there grows with h (5e-8 * 64 h)."""
import numpy as np
import pytest

from paper_1110_6220_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
TOL32 = 1e-5
ORDERED_BIT = 32  # eik_stats.schedule: a pass ran in value order


@pytest.fixture(scope="module")
def eik():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6220_gb300 import build
    build.build()
    from paper_1110_6220_gb300 import eik as e
    e.eik_tune_reset()
    return e


_ORACLE = {}


def oracle_U(orc, I):
    if I.name not in _ORACLE:
        _ORACLE[I.name] = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
    return _ORACLE[I.name]


def check(U, V, st, prec, what, h=0.0):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all(), f"{what}: +inf pattern"
    if not fin.any():
        return 0.0
    scale = np.abs(V[fin]).max()
    err = np.abs(U[fin] - V[fin]).max() / max(scale, 1e-300)
    if prec == 0:
        assert err <= TOL64, f"{what}: {err:.3e}"
    else:
        assert st.err_bound <= TOL32, f"{what}: certificate {st.err_bound:.3e}"
        assert err <= max(st.err_bound, 1e-15) * 1.0001, f"{what}: {err:.3e} above its certificate"
        assert err <= 5e-8 * max(1.0, 64.0 * h), f"{what}: {err:.3e}"
    return err


def instances():
    rng = np.random.default_rng(2024)
    out = [W.sin_point(257), W.checker_maze(257, seed=3, n_walls=6, n_src=3), W.const_point(129),
           W.sin_boundary(129)]
    out += [W.tiny_random(rng, n_max=40) for _ in range(4)]
    out += [W.random_instance(rng, 150, 300, kinds=("blocks",)), W.random_instance(rng, 150, 300, kinds=("sin",))]
    return out


FORMS = [(0, 0), (1, 0), (1, 1)]  # (precision, one double-float pass): FP64; FP32 + refinement; one pass
FORM_IDS = ["fp64", "fp32_then_df", "df_one_pass"]


def _solve(eik, I, k, prec, one_pass, window, m, monkeypatch):
    monkeypatch.setenv("EIK_ONE_PASS", "1" if one_pass else "0")
    return eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=k, precision=prec, bucket_width=-m,
                     schedule=eik.EIK_SCHED_ORDERED, window=window)


@pytest.mark.parametrize("k", [8, 16, 32, 64])
@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("window,m", [(1, 0.5), (3, 4.0), (32, 1.0)])
def test_ordered_single_matches_oracle(eik, orc, monkeypatch, k, form, window, m):
    prec, one_pass = form
    for I in instances():
        U, st = _solve(eik, I, k, prec, one_pass, window, m, monkeypatch)
        assert st.status == 0, (I.name, eik.eik_strerror(st.status))
        assert st.cell_k == k
        assert st.schedule & ORDERED_BIT, I.name
        check(U, oracle_U(orc, I), st, prec, f"{I.name} k={k} w={window} m={m}", I.h)


@pytest.mark.parametrize("k", [8, 16])
@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_ordered_batch_matches_oracle(eik, orc, monkeypatch, k, form):
    """24 uneven grids in one persistent launch per pass, one set of bucket
    rings shared by all of them (ordered by value across instances)."""
    prec, one_pass = form
    monkeypatch.setenv("EIK_ONE_PASS", "1" if one_pass else "0")
    insts = W.batch_mix(24, seed=31, n_lo=17, n_hi=300)
    descs, ins, keep = [], [], []
    for I in insts:
        U = np.empty_like(I.F)
        src = I.src_ij  # a fresh array: kept alive while the library holds its address
        keep.append((I, U, src))
        descs.append(eik.make_desc(I.nx, I.ny, I.h, k, prec, bucket_width=-2.0,
                                   schedule=eik.EIK_SCHED_ORDERED, window=3))
        ins.append(eik.make_instance(I.F, src, I.sq, U))
    rc, st = eik.eik_solve_batch(descs, ins)
    assert rc == 0, eik.eik_strerror(rc)
    for (I, U, _), s in zip(keep, st):
        assert s.schedule & ORDERED_BIT
        check(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), s, prec, f"{I.name} batch k={k}", I.h)


def test_ordered_degenerate_inputs(eik, orc, monkeypatch):
    """No sources (nothing is ever requested), a grid of obstacles around a
    source, a source on an obstacle, one-cell grids, a grid smaller than a
    cell, and strips one cell high with ragged ends."""
    monkeypatch.setenv("EIK_ONE_PASS", "1")
    rng = np.random.default_rng(5)
    cases = []
    F = np.ones((40, 40))
    cases.append(("nosrc", F, 1 / 39, [], [], []))
    F = np.zeros((33, 33))
    F[16, 16] = 1.0
    cases.append(("walled", F, 1 / 32, [16], [16], [0.0]))
    F = rng.uniform(0.5, 2.0, (50, 70))
    F[10, 20] = 0.0
    cases.append(("src_on_obstacle", F, 1 / 69, [20, 3], [10, 40], [0.0, 0.25]))
    cases.append(("one_cell", np.ones((8, 8)), 1 / 7, [3], [4], [1.0]))
    cases.append(("tiny", np.ones((3, 2)), 1.0, [0], [1], [0.0]))
    cases.append(("strip_x", rng.uniform(0.5, 2.0, (5, 600)), 1 / 599, [0, 599], [2, 4], [0.0, 0.1]))
    cases.append(("strip_y", rng.uniform(0.5, 2.0, (700, 9)), 1 / 699, [4], [350], [0.0]))
    for name, F, h, si, sj, sq in cases:
        si, sj, sq = np.array(si, np.int32), np.array(sj, np.int32), np.array(sq, np.float64)
        V = orc.fmm(F, h, si, sj, sq)
        for prec in (0, 1):
            U, st = eik.solve(F, h, si, sj, sq, cell_k=8, precision=prec, schedule=eik.EIK_SCHED_ORDERED,
                              window=2)
            assert st.status == 0, (name, prec, eik.eik_strerror(st.status))
            if not np.isfinite(V).any():
                assert not np.isfinite(U).any(), name
                continue
            check(U, V, st, prec, f"{name} prec={prec}", h)


def test_ordered_fullsize_benchmark_grids(eik, orc):
    """The benchmark's single grids at full size through the value-ordered
    schedule, node by node: 1025^2 sin20 in FP64 at k = 8 and the 4097^2
    checkerboard + maze in FP32_REFINE at k = 16 (4 seeded sources, F = 0
    walls, unreachable pockets that must stay +inf)."""
    I = W.sin_point(1025)
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=0, bucket_width=-4.0,
                      schedule=eik.EIK_SCHED_ORDERED, window=3)
    assert st.status == 0 and st.schedule & ORDERED_BIT
    check(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), st, 0, "sin1025 fp64")
    I = W.checker_maze(4097)
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=16, precision=1, bucket_width=-4.0,
                      schedule=eik.EIK_SCHED_ORDERED, window=4)
    assert st.status == 0 and st.schedule & ORDERED_BIT
    check(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), st, 1, "checker_maze4097 fp32ref")


def test_ordered_cuts_revisits(eik):
    """The point of the order (Sec. 4.2's accounting, Tab. sinu_1 AvHR): on
    the 1025^2 sin20 grid at k = 8 a narrow window removes each cell about
    twice, against ~20 times on the first-in first-out ring; the result is
    the same fixed point either way."""
    I = W.sin_point(1025)
    U0, s0 = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=0, schedule=eik.EIK_SCHED_FIFO)
    U1, s1 = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=0, bucket_width=-1.0,
                       schedule=eik.EIK_SCHED_ORDERED, window=1)
    assert s0.status == 0 and s1.status == 0
    assert s1.avhr <= 3.0, s1.avhr
    assert s0.avhr >= 3 * s1.avhr, (s0.avhr, s1.avhr)
    assert s1.buckets > 50  # the front moved through the value range
    fin = np.isfinite(U0)
    assert np.abs(U1[fin] - U0[fin]).max() <= 2 * TOL64 * np.abs(U0[fin]).max()


def test_ordered_other_methods_fall_back(eik, orc):
    """FHCM and HCM with locking have no value-ordered kernel: naming the
    schedule runs them first in, first out (no ordered bit), still correct
    for the exact one."""
    I = W.sin_point(257)
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=0, method=eik.EIK_METHOD_HCM_LSM,
                      schedule=eik.EIK_SCHED_ORDERED, window=2)
    assert st.status == 0 and not (st.schedule & ORDERED_BIT) and st.schedule & 2
    check(U, oracle_U(orc, I), st, 0, "lsm ordered->fifo")
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=0, method=eik.EIK_METHOD_FHCM,
                      schedule=eik.EIK_SCHED_ORDERED, window=2)
    assert st.status == 0 and not (st.schedule & ORDERED_BIT)
    V = oracle_U(orc, I)
    assert (U >= V - 1e-12 * np.abs(V).max()).all()  # FHCM never undershoots


def test_ordered_deadline_then_correct(eik, orc):
    """Every wait of the ordered queue is bounded: a 1 ns deadline ends the
    solve with EIK_ETIMEDOUT, and the next solve on the same context is
    exact."""
    I = W.sin_point(513)
    for prec in (0, 1):
        with eik.Plan(I.nx, I.ny, I.h, 8, prec, deadline_ns=1, schedule=eik.EIK_SCHED_ORDERED, window=2) as p:
            U = np.empty_like(I.F)
            rc, st = p.solve(I.F, I.src_ij, I.sq, U)
            assert rc == eik.EIK_ETIMEDOUT, eik.eik_strerror(rc)
        U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=prec, schedule=eik.EIK_SCHED_ORDERED,
                          window=2)
        assert st.status == 0
        check(U, oracle_U(orc, I), st, prec, f"after deadline prec={prec}", I.h)
