"""HCM with locking inside cells on the GPU (Sec. 4.2 sweeps a removed cell by
the Locking Sweeping version, Remark locking_FSM).  Locking only skips local
updates that could not change a value, so the result is the exact solution
of eq. Eik_discr, compared node by node with the oracle's Fast Marching at
the FP64 tolerance, for every cell size, both schedules, ragged and
rectangular grids, obstacles, a batch and the benchmarked 1025^2 grid; and
the number of local updates it computes falls well below plain HCM's."""
import math

import numpy as np
import pytest

from paper_1110_6220_gb300 import workloads as W

pytestmark = pytest.mark.gpu
LSM = 3
TOL = 1e-12


@pytest.fixture(scope="module")
def eik():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6220_gb300 import build
    build.build()
    from paper_1110_6220_gb300 import eik as e
    yield e
    e.eik_tune_reset()


def _force(eik, tmp_path, I, k, async_main):
    cls = int(round(0.5 * math.log2(I.nx * I.ny)))
    f = tmp_path / "sched.txt"
    f.write_text(f"eik-tune 4\n0 0 {cls} {k} 256 256 0 {async_main} 0 0 1.0\n")
    eik.eik_tune_reset()
    assert eik.eik_tune_load(str(f)) == 0


def _check(I, U, V):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all(), I.name
    if fin.any():
        scale = np.abs(V[fin]).max()
        err = np.abs(U[fin] - V[fin]).max()
        assert err <= TOL * scale, f"{I.name}: {err / scale:.3e}"


def _instances():
    rng = np.random.default_rng(17)
    c = W.sin_point(257)
    c.F = W.checker_field(257, 16)
    return [W.sin_point(257), W.const_point(129), W.checker_maze(193, 2),
            W.random_instance(rng, 150, 260, kinds=("blocks",)), W.random_instance(rng, 90, 300), c]


@pytest.mark.parametrize("async_main", [0, 1])
@pytest.mark.parametrize("k", [4, 8, 16, 32, 64])
def test_lsm_is_exact(eik, orc, tmp_path, k, async_main):
    if k == 4 and async_main:
        pytest.skip("cells of 4 run two to a warp, on the bucketed schedule only")
    for I in _instances():
        _force(eik, tmp_path, I, k, async_main)
        U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=0, method=LSM)
        assert st.status == 0 and st.cell_k == k
        _check(I, U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq))


@pytest.mark.parametrize("k", [8, 16])
def test_lsm_computes_fewer_updates(eik, orc, k):
    """The serial oracle saves well over half of HCM's local updates on the
    sin20 grid (Remark locking_FSM's purpose); the GPU's concurrent removals
    save a comparable share, and both runs reach the same solution."""
    I = W.sin_point(513)
    V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
    # both on the same (first-in first-out) schedule: locking has no
    # value-ordered form, and plain HCM's built-in one would visit less
    U0, s0 = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=k, method=0, schedule=eik.EIK_SCHED_FIFO)
    U1, s1 = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=k, method=LSM, schedule=eik.EIK_SCHED_FIFO)
    _check(I, U0, V)
    _check(I, U1, V)
    _, c0 = orc.cells(I.F, I.h, I.si, I.sj, I.sq, k)
    _, c1 = orc.cells(I.F, I.h, I.si, I.sj, I.sq, k, lsm=True)
    assert c1["evals"] < 0.6 * c0["evals"]
    assert s1.updates_per_pt < 0.75 * s0.updates_per_pt, (s0.updates_per_pt, s1.updates_per_pt)


def test_lsm_full_size_sin1025(eik, orc):
    """The benchmarked 1025^2 sin20 grid, FP64, in the built-in schedule."""
    I = W.sin_point(1025)
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=0, method=LSM)
    assert st.status == 0
    _check(I, U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq))


def test_lsm_batch_and_rejected_forms(eik, orc):
    import torch
    rng = np.random.default_rng(23)
    insts = [W.random_instance(rng, 70, 300) for _ in range(6)] + [W.sin_point(129), W.checker_maze(97, 4)]
    descs, ins, keep = [], [], []
    for I in insts:
        F = torch.from_numpy(I.F).cuda()
        U = torch.empty_like(F)
        ij = torch.from_numpy(np.stack([I.si, I.sj], 1).reshape(-1).astype(np.int32)).cuda()
        q = torch.from_numpy(I.sq.astype(np.float64)).cuda()
        keep.append((F, U, ij, q))
        descs.append(eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64, method=LSM))
        ins.append(eik.make_instance(F, ij, q, U))
    rc, sts = eik.eik_solve_batch(descs, ins)
    assert rc == 0
    for I, (F, U, _, _), st in zip(insts, keep, sts):
        assert st.status == 0
        _check(I, U.cpu().numpy(), orc.fmm(I.F, I.h, I.si, I.sj, I.sq))
    # FP64 only
    d = eik.make_desc(65, 65, 1.0 / 64, 8, eik.EIK_FP32_REFINE, method=LSM)
    assert eik.eik_plan_workspace_bytes(d) == 0


def test_lsm_degenerate_cases(eik, orc):
    """No sources, a source on every node of a cell border, a grid of one
    row of cells, and sources on obstacles."""
    I = W.sin_point(65)
    U, st = eik.solve(I.F, I.h, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), cell_k=8, method=LSM)
    assert st.status == 0 and np.isinf(U).all()
    si = np.arange(8, 16, dtype=np.int32)
    sj = np.full(8, 8, dtype=np.int32)
    sq = np.linspace(0.0, 0.1, 8)
    U, st = eik.solve(I.F, I.h, si, sj, sq, cell_k=8, method=LSM)
    _check(I, U, orc.fmm(I.F, I.h, si, sj, sq))
    F = np.ones((5, 301))
    F[:, 150] = 0.0
    F[2, 150] = 1.0
    U, st = eik.solve(F, 1.0 / 300, np.array([0, 150], np.int32), np.array([2, 0], np.int32),
                      np.array([0.0, 0.5]), cell_k=16, method=LSM)
    V = orc.fmm(F, 1.0 / 300, np.array([0, 150], np.int32), np.array([2, 0], np.int32), np.array([0.0, 0.5]))
    _check(W.Instance(301, 5, 1.0 / 300, F, None, None, None, name="strip"), U, V)
