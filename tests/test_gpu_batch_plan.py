"""Fixed batches (eik_batch_create / eik_batch_run): the captured launch
sequence replays correctly, picks up new speed values between runs, works
with host buffers, and agrees with eik_solve_batch and the oracle."""
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


def test_fixed_batch_replays_and_follows_new_speeds(eik, orc):
    import torch
    insts = W.batch_mix(10, seed=17, n_lo=33, n_hi=260)
    precs = [eik.EIK_FP64 if e % 2 else eik.EIK_FP32_REFINE for e in range(len(insts))]
    dev, descs, ins = [], [], []
    for I, prec in zip(insts, precs):
        F = torch.from_numpy(I.F.copy()).cuda()
        b = (F, torch.from_numpy(I.src_ij).cuda(), torch.from_numpy(np.ascontiguousarray(I.sq)).cuda(),
             torch.empty_like(F))
        dev.append(b)
        descs.append(eik.make_desc(I.nx, I.ny, I.h, 0, prec))
        ins.append(eik.make_instance(*b))
    batch = eik.eik_batch_create(descs, ins)
    try:
        for run in range(3):
            scale = 1.0 + 0.5 * run  # new speeds in the same buffers
            for (F, _, _, _), I in zip(dev, insts):
                F.copy_(torch.from_numpy(I.F * scale))
            torch.cuda.synchronize()
            rc, st = eik.eik_batch_run(batch)
            assert rc == 0, eik.eik_strerror(rc)
            for I, prec, b, s in zip(insts, precs, dev, st):
                assert s.status == 0
                assert s.schedule & 8, "the launch sequence was not replayed from a graph"
                V = orc.fmm(I.F * scale, I.h, I.si, I.sj, I.sq)
                _check(b[3].cpu().numpy(), V, TOL64 if prec == eik.EIK_FP64 else TOL32, f"{I.name} run {run}")
    finally:
        eik.eik_batch_destroy(batch)


def test_fixed_batch_host_buffers_and_agreement(eik, orc):
    insts = W.batch_mix(6, seed=23, n_lo=65, n_hi=200)
    keep, descs, ins = [], [], []
    for I in insts:
        F = np.ascontiguousarray(I.F.copy())
        U = np.empty_like(F)
        src = I.src_ij
        keep.append((F, src, U))
        descs.append(eik.make_desc(I.nx, I.ny, I.h, 0, eik.EIK_FP32_REFINE))
        ins.append(eik.make_instance(F, src, I.sq, U))
    batch = eik.eik_batch_create(descs, ins)
    try:
        for run in range(2):
            for (F, _, _), I in zip(keep, insts):
                F[...] = I.F * (1.0 + run)  # host speeds are copied in at each run
            rc, st = eik.eik_batch_run(batch)
            assert rc == 0
            for (F, _, U), I in zip(keep, insts):
                _check(U, orc.fmm(F, I.h, I.si, I.sj, I.sq), TOL32, f"{I.name} host run {run}")
    finally:
        eik.eik_batch_destroy(batch)
    # the same instances through eik_solve_batch
    outs = [np.empty_like(F) for F, _, _ in keep]
    ins2 = [eik.make_instance(F, src, I.sq, U) for (F, src, _), I, U in zip(keep, insts, outs)]
    rc, _ = eik.eik_solve_batch(descs, ins2)
    assert rc == 0
    for (_, _, U), U2, I in zip(keep, outs, insts):
        _check(U, U2, 2 * TOL32, f"{I.name} fixed vs one-off batch")


def test_fixed_batch_rejects_bad_input(eik):
    I = W.const_point(33)
    U = np.empty_like(I.F)
    d = [eik.make_desc(1, 33, I.h, 8)]
    with pytest.raises(eik.EikError):
        eik.eik_batch_create(d, [eik.make_instance(I.F, I.src_ij, I.sq, U)])
