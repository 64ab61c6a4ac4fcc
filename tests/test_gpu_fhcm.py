"""Fast Heap-Cell Method on the GPU (Sec. 4.3, Alg. FHCM: one sweep per
flagged direction, flags from the Monotonicity Check).  FHCM is not exact and
its result depends on the order in which cells are removed, so the GPU run
(concurrent removals) is compared with what is order independent: it never
goes below the exact solution, reaches the same nodes on obstacle-free
grids, and its additional errors against an h/4 Fast Marching reference
(Sec. 5's ratios) and its Monotonicity Check rate stay close to the serial
FHCM of the oracle."""
import math

import numpy as np
import pytest

from paper_1110_6220_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FHCM = 1


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


def _instances():
    rng = np.random.default_rng(5)
    insts = [W.sin_point(257), W.const_point(129),
             W.random_instance(rng, 150, 260, kinds=("blocks",)), W.random_instance(rng, 150, 260, kinds=("sin",))]
    c = W.sin_point(257)
    c.F = W.checker_field(257, 16)  # checkerboard speeds, centre source, no walls
    insts.append(c)
    return insts


@pytest.mark.parametrize("async_main", [0, 1])
@pytest.mark.parametrize("k", [8, 16])
def test_fhcm_upper_bound_and_reach(eik, orc, tmp_path, k, async_main):
    for I in _instances():
        _force(eik, tmp_path, I, k, async_main)
        U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=0, method=FHCM)
        assert st.status == 0 and st.cell_k == k
        V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
        fin = np.isfinite(V)
        assert (np.isfinite(U) == fin).all(), I.name
        assert (U[fin] >= V[fin] - 1e-12 * np.abs(V[fin]).max()).all(), f"{I.name}: below the exact solution"
        assert 0.0 < st.mono_pct <= 100.0


@pytest.mark.parametrize("async_main", [0, 1])
@pytest.mark.parametrize("k", [8, 16])
def test_fhcm_error_ratios_track_serial_fhcm(eik, orc, tmp_path, k, async_main):
    """Sec. 5: e_i the discretization error (exact solution vs h/4 FMM),
    E_i the method's; rho = mean(E/e), R_max = max E / max e.  The GPU's
    concurrent FHCM stays within a few percent of the serial one."""
    I = W.sin_point(513)
    J = W.sin_point(4 * 512 + 1)
    V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
    truth = orc.fmm(J.F, J.h, J.si, J.sj, J.sq)[::4, ::4]
    e = np.abs(V - truth)
    m = e > 0
    Uo, so = orc.cells(I.F, I.h, I.si, I.sj, I.sq, k, fast=True)
    Eo = np.abs(Uo - truth)
    _force(eik, tmp_path, I, k, async_main)
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=0, method=FHCM)
    E = np.abs(U - truth)
    rho, rho_o = (E[m] / e[m]).mean(), (Eo[m] / e[m]).mean()
    rmax, rmax_o = E.max() / e.max(), Eo.max() / e.max()
    assert rho <= rho_o + 0.05, (rho, rho_o)
    assert rmax <= rmax_o + 0.1, (rmax, rmax_o)
    assert abs(st.mono_pct - so["mon_pct"]) < 6.0, (st.mono_pct, so["mon_pct"])


def test_fhcm_only_in_fp64(eik):
    I = W.const_point(65)
    U = np.empty_like(I.F)
    d = eik.make_desc(65, 65, I.h, 8, eik.EIK_FP32_REFINE, method=FHCM)
    assert eik.eik_plan_workspace_bytes(d) == 0  # the descriptor is refused
    with pytest.raises(eik.EikError):
        eik.eik_plan_create(d)
    dn = eik.make_desc(65, 65, I.h, 8, eik.EIK_FP64, method=FHCM)
    import torch
    F = torch.from_numpy(I.F).cuda()
    rc, _ = eik.eik_solve_noalloc(dn, eik.make_instance(F, torch.from_numpy(I.src_ij).cuda(),
                                                        torch.from_numpy(I.sq).cuda(), torch.empty_like(F)))
    assert rc == eik.EIK_EINVAL  # the no-allocation solve is HCM only
