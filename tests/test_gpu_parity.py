"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances: FP64 mode max|U_gpu - U_oracle| <= 1e-12 * max|u| (the
discrete fixed point is unique; in floating point distinct evaluation orders
can land a few ulps apart), with +inf at exactly the same nodes.  FP32 +
FP64 refinement: <= 1e-5 * max|u| and a certificate err_bound <= 1e-5.
"""
import numpy as np
import pytest

from paper_1110_6220_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def eik():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6220_gb300 import build
    build.build()
    from paper_1110_6220_gb300 import eik as e
    return e


def oracle_U(orc, I):
    return orc.fmm(I.F, I.h, I.si, I.sj, I.sq)


def compare(U, V, tol, what=""):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all(), f"{what}: +inf pattern differs"
    if not fin.any():
        return 0.0
    scale = np.abs(V[fin]).max()
    err = np.abs(U[fin] - V[fin]).max()
    assert err <= tol * max(scale, 1e-300), f"{what}: err {err:.3e} > {tol:g} * {scale:.3e}"
    return err / max(scale, 1e-300)


def solve(eik, I, k=8, precision=0, **kw):
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=k, precision=precision, **kw)
    return U, st


def test_config1_const_129_k8(eik, orc):
    """129 x 129, F == 1, centre source, k = 8, FP64 (the small workload)."""
    I = W.const_point(129)
    U, st = solve(eik, I, 8)
    compare(U, oracle_U(orc, I), TOL64, "const129")
    assert st.status == 0


@pytest.mark.parametrize("k", [4, 8, 16, 32, 64])
def test_sin_ragged_all_k(eik, orc, k):
    """Smooth oscillating speed on a ragged grid (not a multiple of k):
    several tiles plus a partial last row/column of cells."""
    n = 201
    I = W.sin_point(n, omega=20.0)
    F = I.F[:, :150].copy()  # 150 x 201: ragged in x
    J = W.Instance(150, n, I.h, F, np.array([70], np.int32), np.array([100], np.int32), np.zeros(1))
    U, st = solve(eik, J, k)
    compare(U, oracle_U(orc, J), TOL64, f"sin k={k}")


@pytest.mark.parametrize("k", [4, 8, 16, 32, 64])
def test_tiny_random_grids(eik, orc, k):
    """Tiny grids (down to 2 x 2) with obstacles, several sources, q != 0."""
    rng = np.random.default_rng(100 + k)
    for _ in range(12):
        I = W.tiny_random(rng)
        U, st = solve(eik, I, k)
        compare(U, oracle_U(orc, I), TOL64, f"tiny {I.name} k={k}")


def test_maze_obstacles_unreachable(eik, orc):
    """Checkerboard + F = 0 maze: unreachable pockets must stay +inf exactly."""
    I = W.checker_maze(513, seed=3, n_walls=12)
    U, st = solve(eik, I, 8)
    compare(U, oracle_U(orc, I), TOL64, "maze513")


def test_no_sources_and_source_on_obstacle(eik, orc):
    I = W.const_point(40)
    U, st = eik.solve(I.F, I.h, [], [], [], cell_k=8)
    assert np.isinf(U).all() and st.status == 0
    F = I.F.copy()
    F[:, 20] = 0.0
    J = W.Instance(40, 40, I.h, F, np.array([20, 3], np.int32), np.array([5, 30], np.int32),
                   np.array([0.25, 0.0]))
    U, st = solve(eik, J, 8)
    compare(U, oracle_U(orc, J), TOL64, "src on obstacle")
    assert U[5, 20] == 0.25


def test_duplicate_sources_and_negative_q(eik, orc):
    I = W.sin_point(65)
    J = W.Instance(65, 65, I.h, I.F, np.array([10, 10, 50], np.int32),
                   np.array([12, 12, 40], np.int32), np.array([0.5, -0.3, 0.1]))
    U, st = solve(eik, J, 16)
    compare(U, oracle_U(orc, J), TOL64, "dups")
    assert U[12, 10] == -0.3


def test_config2_sin_1025_fp64_full(eik, orc):
    """1025 x 1025 sin20 speed, FP64, every node compared."""
    I = W.sin_point(1025)
    V = oracle_U(orc, I)
    for k in (8, 32):
        U, st = solve(eik, I, k)
        compare(U, V, TOL64, f"sin1025 k={k}")


@pytest.mark.parametrize("k", [8, 16])
def test_fp32_refine_certified(eik, orc, k):
    """FP32 cell solves + FP64 refinement: within 1e-5 of the oracle and
    the residual certificate reaches the stated tolerance."""
    for I in (W.sin_point(257), W.checker_maze(257, seed=5, n_walls=6)):
        U, st = solve(eik, I, k, precision=eik.EIK_FP32_REFINE)
        assert st.status == 0, eik.eik_strerror(st.status)
        rel = compare(U, oracle_U(orc, I), TOL32, f"fp32ref {I.name}")
        assert st.err_bound <= TOL32
        assert rel <= max(st.err_bound, 1e-15) * 1.0001
        # the pair arithmetic keeps ~46 bits per step: far below the stated
        # tolerance, so an error in f = h/F or in the update would show here
        assert rel <= 5e-8, f"fp32ref {I.name}: {rel:.3e} above the observed accuracy floor"


@pytest.mark.parametrize("omega,amp", [(20.0, 0.5), (2.0, 0.99)])
def test_boundary_sources(eik, orc, omega, amp):
    """Q = the whole boundary with q = 0 (Sec. 5's general boundary
    conditions): every boundary cell starts queued."""
    I = W.sin_boundary(257, omega, amp)
    V = oracle_U(orc, I)
    for k in (8, 16):
        U, st = solve(eik, I, k)
        compare(U, V, TOL64, f"{I.name} fp64 k={k}")
        U, st = solve(eik, I, k, precision=eik.EIK_FP32_REFINE)
        rel = compare(U, V, TOL32, f"{I.name} fp32ref k={k}")
        assert st.status == 0 and rel <= max(st.err_bound, 1e-15) * 1.0001


def test_device_pointers_match_host_pointers(eik, orc):
    import torch
    I = W.sin_point(300)
    Uh, _ = solve(eik, I, 8)
    F = torch.from_numpy(I.F).cuda()
    src = torch.from_numpy(I.src_ij).cuda()
    q = torch.from_numpy(I.sq).cuda()
    U = torch.empty_like(F)
    with eik.Plan(I.nx, I.ny, I.h, 8) as p:
        rc, st = p.solve(F, src, q, U)
    assert rc == 0
    # bucket rounds run concurrently, so two runs may settle on fixed points a
    # few ulps apart: compare both with the oracle instead of bit for bit
    V = oracle_U(orc, I)
    compare(U.cpu().numpy(), V, TOL64, "device pointers")
    compare(Uh, V, TOL64, "host pointers")


def test_pinned_host_buffers_in_place(eik, orc):
    """Pinned host F and U are read and written by the kernels in place (no
    staging copy): single grids in both precisions, a batch mixing pinned,
    pageable and device buffers, a fixed batch replayed with new speeds in the
    same pinned buffer, and a served request -- each against the oracle."""
    import time
    import torch
    I = W.checker_maze(300, seed=5, n_walls=4, n_src=2)
    V = oracle_U(orc, I)
    Fp = torch.from_numpy(I.F).pin_memory()
    for prec, tol in ((eik.EIK_FP64, TOL64), (eik.EIK_FP32_REFINE, TOL32)):
        Up = torch.full(I.F.shape, -1.0, dtype=torch.float64).pin_memory()
        with eik.Plan(I.nx, I.ny, I.h, 8, prec) as p:
            rc, st = p.solve(Fp, I.src_ij, I.sq, Up)
        assert rc == 0, eik.eik_strerror(rc)
        compare(Up.numpy(), V, tol, f"pinned F and U, precision {prec}")
    # a batch: pinned, pageable and device buffers side by side
    J = W.sin_point(129)
    VJ = oracle_U(orc, J)
    Ud = torch.empty(J.F.shape, dtype=torch.float64, device="cuda")
    Upg = np.full_like(J.F, -1.0)
    Upn = torch.full(I.F.shape, -1.0, dtype=torch.float64).pin_memory()
    Fd = torch.from_numpy(J.F).cuda()
    descs = [eik.make_desc(I.nx, I.ny, I.h, 16, eik.EIK_FP64), eik.make_desc(J.nx, J.ny, J.h, 16, eik.EIK_FP64),
             eik.make_desc(J.nx, J.ny, J.h, 16, eik.EIK_FP64)]
    insts = [eik.make_instance(Fp, I.src_ij, I.sq, Upn), eik.make_instance(J.F, J.src_ij, J.sq, Upg),
             eik.make_instance(Fd, J.src_ij, J.sq, Ud)]
    rc, sts = eik.eik_solve_batch(descs, insts)
    assert rc == 0
    compare(Upn.numpy(), V, TOL64, "batch, pinned")
    compare(Upg, VJ, TOL64, "batch, pageable")
    compare(Ud.cpu().numpy(), VJ, TOL64, "batch, device")
    # a fixed batch replayed with new speeds written into the same pinned F
    F2 = np.ascontiguousarray(I.F * 1.5)
    b = eik.eik_batch_create([descs[0]], [insts[0]])
    try:
        assert eik.eik_batch_run(b)[0] == 0
        compare(Upn.numpy(), V, TOL64, "fixed batch, pinned")
        Fp.numpy()[...] = F2
        assert eik.eik_batch_run(b)[0] == 0
        Vs = orc.fmm(F2, I.h, I.si, I.sj, I.sq)
        compare(Upn.numpy(), Vs, TOL64, "fixed batch, pinned, new speeds")
    finally:
        eik.eik_batch_destroy(b)
    # a served request with pinned buffers
    Fp.numpy()[...] = I.F
    Ups = torch.full(I.F.shape, -1.0, dtype=torch.float64).pin_memory()
    srv = eik.eik_server_create(1 << 30, 4)
    try:
        rc, t = eik.eik_submit(srv, eik.make_desc(I.nx, I.ny, I.h, 16, eik.EIK_FP32_REFINE),
                               eik.make_instance(Fp, I.src_ij, I.sq, Ups))
        assert rc == 0
        t0 = time.perf_counter()
        while True:
            rc, st = eik.eik_poll(srv, t)
            if rc != eik.EIK_EAGAIN:
                break
            assert time.perf_counter() - t0 < 60
            time.sleep(2e-4)
        assert rc == 0
    finally:
        eik.eik_server_destroy(srv)
    compare(Ups.numpy(), V, TOL32, "served, pinned")


def test_invalid_inputs_rejected(eik):
    I = W.const_point(33)
    F = I.F.copy()
    F[3, 3] = -1.0
    with pytest.raises(eik.EikError) as e:
        eik.solve(F, I.h, I.si, I.sj, I.sq)
    assert e.value.code == eik.EIK_EINVAL
    F[3, 3] = np.nan
    with pytest.raises(eik.EikError):
        eik.solve(F, I.h, I.si, I.sj, I.sq)
    with pytest.raises(eik.EikError):
        eik.solve(I.F, I.h, [33], [0], [0.0])  # outside the grid
    with pytest.raises(eik.EikError):
        eik.solve(I.F, I.h, [3], [0], [np.inf])


def test_deadline_expiry_reports_timeout_and_context_survives(eik, orc):
    """A wait that runs out (1 ns deadline) ends the launch with
    EIK_ETIMEDOUT instead of hanging; the next solve works."""
    I = W.sin_point(513)
    with eik.Plan(I.nx, I.ny, I.h, 8, deadline_ns=1) as p:
        U = np.empty_like(I.F)
        rc, st = p.solve(I.F, I.src_ij, I.sq, U)
    assert rc == eik.EIK_ETIMEDOUT
    U, st = solve(eik, I, 8)
    compare(U, oracle_U(orc, I), TOL64, "after timeout")
