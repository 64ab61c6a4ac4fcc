"""Batched solves (one persistent launch for many uneven grids) against the
CPU oracle, instance by instance, plus batch-vs-single equality."""
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


def _batch(eik, insts, k, prec, device=False):
    import torch
    descs, ins, keep, outs = [], [], [], []
    for I in insts:
        descs.append(eik.make_desc(I.nx, I.ny, I.h, k, prec))
        if device:
            F = torch.from_numpy(I.F).cuda()
            src = torch.from_numpy(I.src_ij).cuda()
            q = torch.from_numpy(I.sq).cuda()
            U = torch.empty_like(F)
        else:
            F, src, q = np.ascontiguousarray(I.F), I.src_ij, np.ascontiguousarray(I.sq)
            U = np.empty_like(F)
        keep.append((F, src, q, U))
        ins.append(eik.make_instance(F, src, q, U))
        outs.append(U)
    rc, st = eik.eik_solve_batch(descs, ins)
    res = [u.cpu().numpy() if hasattr(u, "cpu") else u for u in outs]
    return rc, st, res


@pytest.mark.parametrize("k", [4, 8, 16])
def test_batch_fp64_mixed_sizes(eik, orc, k):
    rng = np.random.default_rng(40 + k)
    insts = W.batch_mix(24, seed=k, n_lo=17, n_hi=200)
    insts += [W.tiny_random(rng) for _ in range(8)]
    rc, st, U = _batch(eik, insts, k, eik.EIK_FP64)
    assert rc == 0, eik.eik_strerror(rc)
    for I, u, s in zip(insts, U, st):
        assert s.status == 0
        _check(u, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), TOL64, I.name)


def test_batch_fp32_refine_device_pointers(eik, orc):
    insts = W.batch_mix(16, seed=7, n_lo=65, n_hi=300)
    rc, st, U = _batch(eik, insts, 8, eik.EIK_FP32_REFINE, device=True)
    assert rc == 0, eik.eik_strerror(rc)
    for I, u, s in zip(insts, U, st):
        assert s.status == 0 and s.err_bound <= TOL32
        _check(u, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), TOL32, I.name)


def test_batch_matches_single_solves(eik, orc):
    """Each instance gets the same answer alone (eik_solve) and in a batch
    (both within tolerance of the oracle; concurrent schedules may differ
    by ulps)."""
    insts = W.batch_mix(6, seed=3, n_lo=33, n_hi=150)
    rc, st, U = _batch(eik, insts, 8, eik.EIK_FP64)
    assert rc == 0
    for I, u in zip(insts, U):
        v, _ = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8)
        _check(u, v, TOL64, I.name)


def test_batch_groups_mixed_k_and_precision(eik, orc):
    insts = W.batch_mix(6, seed=5, n_lo=33, n_hi=120)
    import itertools
    descs, ins, keep = [], [], []
    combos = list(itertools.product([8, 16], [eik.EIK_FP64, eik.EIK_FP32_REFINE]))
    for e, I in enumerate(insts):
        k, prec = combos[e % len(combos)]
        descs.append(eik.make_desc(I.nx, I.ny, I.h, k, prec))
        U = np.empty_like(I.F)
        src = I.src_ij  # a new array on each access: keep this one alive
        keep.append((I.F, src, I.sq, U))
        ins.append(eik.make_instance(I.F, src, I.sq, U))
    rc, st = eik.eik_solve_batch(descs, ins)
    assert rc == 0
    for e, (I, kp) in enumerate(zip(insts, keep)):
        tol = TOL64 if combos[e % len(combos)][1] == eik.EIK_FP64 else TOL32
        _check(kp[3], orc.fmm(I.F, I.h, I.si, I.sj, I.sq), tol, I.name)


def test_batch_rejects_bad_instance(eik):
    I = W.const_point(33)
    d = [eik.make_desc(33, 33, I.h, 8), eik.make_desc(1, 33, I.h, 8)]
    U = np.empty_like(I.F)
    ins = [eik.make_instance(I.F, I.src_ij, I.sq, U)] * 2
    rc, _ = eik.eik_solve_batch(d, ins)
    assert rc == eik.EIK_EINVAL
