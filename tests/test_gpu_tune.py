"""Autotuner: eik_tune picks a cell size and bucket widths from timed trial
solves, never slower than the choice in force before; later solves that
leave k open use it and still match the oracle."""
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
    e.eik_tune_reset()
    yield e
    e.eik_tune_reset()


def _check(U, V, tol, what):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all(), f"{what}: +inf pattern"
    scale = np.abs(V[fin]).max()
    err = np.abs(U[fin] - V[fin]).max()
    assert err <= tol * scale, f"{what}: {err:.3e} > {tol:g} * {scale:.3e}"


@pytest.mark.parametrize("prec", [0, 1])
def test_tune_single_then_solve_uses_choice(eik, orc, prec):
    I = W.sin_point(257)
    U = np.empty_like(I.F)
    src = I.src_ij
    d = eik.make_desc(I.nx, I.ny, I.h, 0, prec)
    rc, r = eik.eik_tune([d], [eik.make_instance(I.F, src, I.sq, U)])
    assert rc == 0, eik.eik_strerror(rc)
    assert r.cell_k in (8, 16, 32) and r.trials >= 10
    assert r.bucket_main in (2, 4, 8, 16, 64, 256) or r.ms == r.ms_before
    assert 0 < r.ms <= r.ms_before
    assert r.ordered in (0, 1) and (r.window in (3, 4) if r.ordered else r.window == 0)
    V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
    tol = TOL64 if prec == 0 else TOL32
    _check(U, V, tol, "last trial")
    U2, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=0, precision=prec)
    assert st.cell_k == r.cell_k
    assert bool(st.schedule & 32) == bool(r.ordered)  # the tuned schedule is the one that runs
    _check(U2, V, tol, "tuned solve")


def test_tune_batch_class(eik, orc):
    insts = W.batch_mix(12, seed=21, n_lo=65, n_hi=200)
    keep, descs, ins = [], [], []
    for I in insts:
        U = np.empty_like(I.F)
        src = I.src_ij
        keep.append((I, U, src))
        descs.append(eik.make_desc(I.nx, I.ny, I.h, 0, eik.EIK_FP32_REFINE))
        ins.append(eik.make_instance(I.F, src, I.sq, U))
    rc, r = eik.eik_tune(descs, ins)
    assert rc == 0 and r.cell_k in (8, 16, 32)
    rc, st = eik.eik_solve_batch(descs, ins)
    assert rc == 0
    for (I, U, _), s in zip(keep, st):
        assert s.cell_k == r.cell_k and s.err_bound <= TOL32
        _check(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), TOL32, I.name)


def test_tune_rejects_mixed_precision(eik):
    I = W.const_point(33)
    U = np.empty_like(I.F)
    src = I.src_ij
    ins = [eik.make_instance(I.F, src, I.sq, U)] * 2
    d = [eik.make_desc(33, 33, I.h, 0, 0), eik.make_desc(33, 33, I.h, 0, 1)]
    rc, _ = eik.eik_tune(d, ins)
    assert rc == eik.EIK_EINVAL
