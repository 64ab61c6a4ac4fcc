"""Fast Marching-Sweeping Method on the GPU (Sec. 4.1, Alg. FMSM).  The GPU
runs each cell as soon as the neighbours accepted before it are done.  A
cell's result depends only on which of its neighbours ran before it, so the
GPU's result is that of the serial loop over the acceptance order, and it is
compared with the oracle's serial FMSM node by node (FP64: 1e-12 of max |U|,
+inf exactly) and by its number of sweeps."""
import numpy as np
import pytest

from paper_1110_6220_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FMSM = 2


@pytest.fixture(scope="module")
def eik():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6220_gb300 import build
    build.build()
    from paper_1110_6220_gb300 import eik as e
    return e


def _instances():
    rng = np.random.default_rng(9)
    insts = [W.sin_point(257), W.const_point(129),
             W.random_instance(rng, 150, 260, kinds=("blocks",)), W.random_instance(rng, 150, 260, kinds=("sin",)),
             W.checker_maze(385, seed=3, n_walls=6, n_src=3)]
    c = W.sin_point(257)
    c.F = W.checker_field(257, 16)  # checkerboard speeds, centre source
    insts.append(c)
    return insts


def _compare(I, k, U, st, Uo, so):
    fin = np.isfinite(Uo)
    assert (np.isfinite(U) == fin).all(), I.name
    scale = np.abs(Uo[fin]).max()
    err = np.abs(U[fin] - Uo[fin]).max(initial=0.0)
    assert err <= 1e-12 * scale, (I.name, k, err / scale)
    assert abs(st.avhr - 1.0) < 1e-12, (I.name, st.avhr)  # every cell once
    # the sweeps of each cell are the oracle's; a cell holding a source
    # sweeps to convergence, which rounding may end one sweep apart
    src_cells = len({(int(i) // k, int(j) // k) for i, j in zip(I.si, I.sj)})
    assert abs(round(st.avs * so["cells"]) - so["sweeps"]) <= src_cells, (I.name, st.avs * so["cells"], so["sweeps"])


@pytest.mark.parametrize("k", [8, 16, 32])
def test_fmsm_matches_serial_oracle(eik, orc, k):
    for I in _instances():
        U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=k, method=FMSM)
        assert st.status == 0 and st.cell_k == k and st.schedule & 16
        Uo, so = orc.fmsm(I.F, I.h, I.si, I.sj, I.sq, k)
        _compare(I, k, U, st, Uo, so)


@pytest.mark.parametrize("k", [8, 16])
def test_fmsm_full_size_sin1025(eik, orc, k):
    """The 1025^2 sin20 grid with a centre source, element by element."""
    I = W.sin_point(1025)
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=k, method=FMSM)
    assert st.status == 0
    Uo, so = orc.fmsm(I.F, I.h, I.si, I.sj, I.sq, k)
    _compare(I, k, U, st, Uo, so)
    V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
    assert (U >= V - 1e-12 * V.max()).all()  # never below the exact solution


def test_fmsm_k64_and_ragged(eik, orc):
    rng = np.random.default_rng(4)
    I = W.random_instance(rng, 300, 330, kinds=("sin",))
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=64, method=FMSM)
    assert st.status == 0
    Uo, so = orc.fmsm(I.F, I.h, I.si, I.sj, I.sq, 64)
    _compare(I, 64, U, st, Uo, so)


def test_fmsm_batch(eik, orc):
    """Several grids as one job: one coarse job for all of them, one
    persistent pass; each grid's result is its serial FMSM."""
    import torch
    rng = np.random.default_rng(12)
    insts = [W.random_instance(rng, 70, 300) for _ in range(6)] + [W.sin_point(129)]
    descs, ins, keep = [], [], []
    for I in insts:
        F = torch.from_numpy(I.F).cuda()
        U = torch.empty_like(F)
        ij = torch.from_numpy(np.stack([I.si, I.sj], 1).reshape(-1).astype(np.int32)).cuda()
        q = torch.from_numpy(I.sq.astype(np.float64)).cuda()
        keep.append((F, U, ij, q))
        descs.append(eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64, method=FMSM))
        ins.append(eik.make_instance(F, ij, q, U))
    rc, sts = eik.eik_solve_batch(descs, ins)
    assert rc == 0
    for I, (F, U, _, _), st in zip(insts, keep, sts):
        Uo, so = orc.fmsm(I.F, I.h, I.si, I.sj, I.sq, 8)
        _compare(I, 8, U.cpu().numpy(), st, Uo, so)


def test_fmsm_rejected_forms(eik):
    I = W.const_point(65)
    for prec, k in ((eik.EIK_FP32_REFINE, 8), (eik.EIK_FP64, 4)):
        d = eik.make_desc(65, 65, I.h, k, prec, method=FMSM)
        assert eik.eik_plan_workspace_bytes(d) == 0  # the descriptor is refused
    d = eik.make_desc(65, 65, I.h, 0, eik.EIK_FP64, method=FMSM)
    U = np.empty_like(I.F)
    rc, _ = eik.eik_tune([d], [eik.make_instance(I.F, I.src_ij, I.sq, U)])
    assert rc == eik.EIK_EINVAL  # the tuning table holds the cell solver's schedules


def test_fmsm_in_fixed_batch_and_server(eik, orc):
    """FMSM grids mixed with HCM grids: a fixed batch replayed from its
    captured graph (run twice) and the serving loop each give every FMSM grid
    its serial FMSM result and every HCM grid the exact solution."""
    import time
    insts = W.batch_mix(8, seed=43, n_lo=65, n_hi=220)
    methods = [FMSM if e % 2 == 0 else eik.EIK_METHOD_HCM for e in range(len(insts))]
    descs, ins, keep = [], [], []
    for I, m in zip(insts, methods):
        U = np.empty_like(I.F)
        src = I.src_ij
        keep.append((src, U))
        descs.append(eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64, method=m))
        ins.append(eik.make_instance(I.F, src, I.sq, U))

    def verify(what):
        for I, m, (_, U) in zip(insts, methods, keep):
            if m == FMSM:
                Uo, _ = orc.fmsm(I.F, I.h, I.si, I.sj, I.sq, 8)
            else:
                Uo = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
            fin = np.isfinite(Uo)
            assert (np.isfinite(U) == fin).all(), (what, I.name)
            assert np.abs(U[fin] - Uo[fin]).max(initial=0.0) <= 1e-12 * np.abs(Uo[fin]).max(), (what, I.name, m)

    b = eik.eik_batch_create(descs, ins)
    try:
        for r in range(2):
            for _, U in keep:
                U[...] = np.nan
            rc, sts = eik.eik_batch_run(b)
            assert rc == 0
            assert all(s.schedule & 8 for s in sts)  # replayed from the captured graph
            assert all(bool(s.schedule & 16) == (m == FMSM) for s, m in zip(sts, methods))
            verify(f"fixed batch run {r}")
    finally:
        eik.eik_batch_destroy(b)
    for _, U in keep:
        U[...] = np.nan
    srv = eik.eik_server_create(1 << 30, 0)
    try:
        tickets = []
        for d, i in zip(descs, ins):
            rc, t = eik.eik_submit(srv, d, i)
            assert rc == 0
            tickets.append(t)
        for t in tickets:
            t0 = time.perf_counter()
            while True:
                rc, _ = eik.eik_poll(srv, t)
                if rc != eik.EIK_EAGAIN:
                    break
                assert time.perf_counter() - t0 < 60
                time.sleep(2e-4)
            assert rc == 0
    finally:
        eik.eik_server_destroy(srv)
    verify("server")


def test_fmsm_degenerate_cases(eik, orc):
    """Edge cases of the order and of the cells, each against the oracle:
    a grid smaller than one cell, no sources (everything stays +inf), a
    source on an obstacle, a source walled in (most of the grid unreachable,
    its cells ordered last by index), and a grid one cell high."""
    rng = np.random.default_rng(17)
    cases = []
    F = rng.uniform(0.5, 2.0, size=(5, 6))
    cases.append(("one cell", F, 1.0 / 5, [2], [1], [0.0]))
    F = rng.uniform(0.5, 2.0, size=(40, 33))
    cases.append(("no sources", F, 1.0 / 39, [], [], []))
    F = rng.uniform(0.5, 2.0, size=(60, 70))
    F[30, 20] = 0.0
    cases.append(("source on an obstacle", F, 1.0 / 69, [20, 50], [30, 10], [0.0, 0.25]))
    F = rng.uniform(0.5, 2.0, size=(64, 64))
    F[20:31, 20] = 0.0
    F[20:31, 30] = 0.0
    F[20, 20:31] = 0.0
    F[30, 20:31] = 0.0
    cases.append(("walled-in source", F, 1.0 / 63, [25], [25], [0.0]))
    F = rng.uniform(0.5, 2.0, size=(7, 200))
    cases.append(("one cell high", F, 1.0 / 199, [0, 199], [3, 6], [0.0, 0.0]))
    for name, F, h, si, sj, sq in cases:
        si, sj = np.array(si, np.int32), np.array(sj, np.int32)
        sq = np.array(sq, np.float64)
        U, st = eik.solve(F, h, si, sj, sq, cell_k=8, method=FMSM)
        assert st.status == 0, name
        Uo, so = orc.fmsm(F, h, si, sj, sq, 8)
        fin = np.isfinite(Uo)
        assert (np.isfinite(U) == fin).all(), name
        if fin.any():
            assert np.abs(U[fin] - Uo[fin]).max() <= 1e-12 * np.abs(Uo[fin]).max(), name
        assert abs(round(st.avs * so["cells"]) - so["sweeps"]) <= max(len(si), 1), name
