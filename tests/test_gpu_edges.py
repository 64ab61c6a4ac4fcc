"""Edge cases of the GPU path: deadlines that expire in the middle of a
round-free or FHCM run, batches above the per-launch instance limit, mixed
methods in one batch and one server, the largest cell size, rectangular and
ragged grids in both precisions."""
import time

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


def _check(U, V, tol, what):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all(), f"{what}: +inf pattern"
    if fin.any():
        scale = np.abs(V[fin]).max()
        err = np.abs(U[fin] - V[fin]).max()
        assert err <= tol * scale, f"{what}: {err:.3e} > {tol:g} * {scale:.3e}"


@pytest.mark.parametrize("prec,method", [(1, 0), (0, 1), (0, 0)])
def test_deadline_in_mid_run(eik, orc, prec, method):
    """A 150 us deadline on a solve of ~2-4 ms: the launch ends early with
    EIK_ETIMEDOUT (every wait is bounded, the round-free ring included), and
    the next solve on the same plan is correct."""
    import torch
    I = W.sin_point(1025)
    F = torch.from_numpy(I.F).cuda()
    src = torch.from_numpy(I.src_ij).cuda()
    q = torch.from_numpy(I.sq).cuda()
    U = torch.empty_like(F)
    with eik.Plan(I.nx, I.ny, I.h, 8, prec, deadline_ns=150_000, method=method) as p:
        rc, st = p.solve(F, src, q, U)
    assert rc == eik.EIK_ETIMEDOUT, eik.eik_strerror(rc)
    with eik.Plan(I.nx, I.ny, I.h, 8, prec, method=method) as p:
        rc, st = p.solve(F, src, q, U)
    assert rc == 0
    if method == 0:
        _check(U.cpu().numpy(), orc.fmm(I.F, I.h, I.si, I.sj, I.sq), TOL64 if prec == 0 else TOL32, "after")


def test_batch_above_one_launch(eik, orc):
    """More instances than one persistent launch holds (2048): the batch
    runs as several jobs, and every instance is right."""
    rng = np.random.default_rng(9)
    insts = [W.tiny_random(rng, n_max=12) for _ in range(2100)]
    descs, ins, outs = [], [], []
    keep = []
    for I in insts:
        U = np.empty_like(I.F)
        src = I.src_ij
        keep.append((src, U))
        descs.append(eik.make_desc(I.nx, I.ny, I.h, 4, eik.EIK_FP64))
        ins.append(eik.make_instance(I.F, src, I.sq, U))
    rc, st = eik.eik_solve_batch(descs, ins)
    assert rc == 0, eik.eik_strerror(rc)
    for I, (_, U) in zip(insts[::37], keep[::37]):
        _check(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), TOL64, I.name)


def test_mixed_methods_in_batch_and_server(eik, orc):
    insts = W.batch_mix(8, seed=41, n_lo=65, n_hi=200)
    methods = [e % 2 for e in range(len(insts))]
    descs, ins, keep = [], [], []
    for I, m in zip(insts, methods):
        U = np.empty_like(I.F)
        src = I.src_ij
        keep.append((src, U))
        descs.append(eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64, method=m))
        ins.append(eik.make_instance(I.F, src, I.sq, U))

    def verify(what):
        for I, m, (_, U) in zip(insts, methods, keep):
            V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
            fin = np.isfinite(V)
            if m == 0:
                _check(U, V, TOL64, f"{what} HCM {I.name}")
            else:
                assert (U[fin] >= V[fin] - 1e-12 * np.abs(V[fin]).max()).all(), f"{what} FHCM {I.name}"

    rc, st = eik.eik_solve_batch(descs, ins)
    assert rc == 0
    verify("batch")
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


@pytest.mark.parametrize("prec", [0, 1])
def test_largest_cells_and_rectangular_grids(eik, orc, prec):
    tol = TOL64 if prec == 0 else TOL32
    rng = np.random.default_rng(13)
    base = W.sin_point(301, omega=9.0)
    for nx, ny, k in ((301, 97, 64), (97, 301, 32), (150, 201, 16), (33, 300, 8)):
        F = np.ascontiguousarray(base.F[:ny, :nx])
        ns = 3
        si = rng.integers(0, nx, ns).astype(np.int32)
        sj = rng.integers(0, ny, ns).astype(np.int32)
        I = W.Instance(nx, ny, base.h, F, si, sj, np.zeros(ns))
        U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=k, precision=prec)
        _check(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), tol, f"{nx}x{ny} k={k}")
