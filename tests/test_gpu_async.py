"""The round-free schedule (a device-side ring, no buckets, no grid barrier
per round) in all three arithmetic modes -- FP64, the FP32 pass and the
double-float refinement pass -- against the oracle.  The schedule is chosen
through a loaded tuning table, as a deployment would."""
import math

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
    yield e
    e.eik_tune_reset()


def _side_class(sizes):
    pts = sum(nx * ny for nx, ny in sizes) / len(sizes)
    return int(round(0.5 * math.log2(max(pts, 1.0))))


def _force(eik, tmp_path, rows):
    """rows: (precision, batch, side class, k, async_first, async_main, one_pass)."""
    f = tmp_path / "sched.txt"
    lines = ["eik-tune 4"] + [f"{p} {b} {s} {k} 4 4 {a1} {a2} {op} 0 1.0" for p, b, s, k, a1, a2, op in rows]
    f.write_text("\n".join(lines) + "\n")
    eik.eik_tune_reset()
    assert eik.eik_tune_load(str(f)) == 0


def _check(U, V, tol, what):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all(), f"{what}: +inf pattern"
    if fin.any():
        scale = np.abs(V[fin]).max()
        err = np.abs(U[fin] - V[fin]).max()
        assert err <= tol * scale, f"{what}: {err:.3e} > {tol:g} * {scale:.3e}"


def _instances():
    rng = np.random.default_rng(77)
    out = [W.sin_point(257), W.checker_maze(257, seed=3, n_walls=6, n_src=3), W.const_point(129)]
    out += [W.tiny_random(rng, n_max=40) for _ in range(6)]
    out += [W.random_instance(rng, 150, 300, kinds=("blocks",)), W.random_instance(rng, 150, 300, kinds=("sin",))]
    return out


@pytest.mark.parametrize("k", [8, 16, 32])
@pytest.mark.parametrize("prec,one_pass", [(0, 0), (1, 0), (1, 1)])
def test_async_single_matches_oracle(eik, orc, tmp_path, k, prec, one_pass):
    """FP64; FP32 + refinement with both passes round-free; one round-free
    double-float pass."""
    insts = _instances()
    rows = {(prec, 0, _side_class([(I.nx, I.ny)]), k, 1, 1, one_pass) for I in insts}
    _force(eik, tmp_path, sorted(rows))
    tol = TOL64 if prec == 0 else TOL32
    for I in insts:
        U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=0, precision=prec)
        assert st.cell_k == k and st.status == 0
        V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
        _check(U, V, tol, f"{I.name} k={k}")
        if prec == 1:
            assert st.err_bound <= TOL32
            fin = np.isfinite(V)
            if fin.any() and np.abs(V[fin]).max() > 0:
                rel = np.abs(U[fin] - V[fin]).max() / np.abs(V[fin]).max()
                assert rel <= max(st.err_bound, 1e-15) * 1.0001  # the certificate holds
                assert rel <= 5e-8


@pytest.mark.parametrize("sched", [(1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (0, 1, 1)])
def test_async_batch_matches_oracle(eik, orc, tmp_path, sched):
    """(async FP32 pass, async main pass, one double-float pass)."""
    insts = W.batch_mix(24, seed=31, n_lo=17, n_hi=300)
    for prec in (0, 1):
        if prec == 0 and sched[2]:
            continue
        _force(eik, tmp_path, [(prec, 1, _side_class([(I.nx, I.ny) for I in insts]), 16) + sched])
        descs, ins, keep = [], [], []
        for I in insts:
            U = np.empty_like(I.F)
            src = I.src_ij
            keep.append((I, U, src))
            descs.append(eik.make_desc(I.nx, I.ny, I.h, 0, prec))
            ins.append(eik.make_instance(I.F, src, I.sq, U))
        rc, st = eik.eik_solve_batch(descs, ins)
        assert rc == 0, eik.eik_strerror(rc)
        tol = TOL64 if prec == 0 else TOL32
        for (I, U, _), s in zip(keep, st):
            assert s.cell_k == 16
            _check(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq), tol, f"{I.name} sched={sched} prec={prec}")
