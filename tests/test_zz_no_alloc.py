"""eik_solve_noalloc: the FP64 solve whose workspace is a fixed device array
inside the library, for callers that cannot call cudaMalloc (device memory
owned by another allocator or a fixed budget, or loops that cannot afford an
allocation's implicit synchronisation).

Its results must agree with the plan-based entry point (eik_solve) within the
FP64 parity tolerance, on two calls in a row (the second call finds the first
call's data in the shared scratch and must not be misled by it).  This file
is named to be collected last.
"""
import numpy as np
import pytest

from paper_1110_6220_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(scope="module")
def eik():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_6220_gb300 import build
    build.build()
    from paper_1110_6220_gb300 import eik as e
    return e


def _close(U, V, what):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all(), what
    scale = np.abs(V[fin]).max()
    assert np.abs(U[fin] - V[fin]).max() <= TOL64 * scale, what


def test_noalloc_matches_plan_solve_on_two_calls(eik):
    import torch
    cases = [(W.sin_point(257), 8), (W.checker_maze(200, seed=4, n_walls=4), 16)]
    for I, k in cases:
        F = torch.from_numpy(I.F).cuda()
        src = torch.from_numpy(I.src_ij).cuda()
        q = torch.from_numpy(I.sq + 0.25).cuda()  # non-zero q exercises the shift
        Uref = torch.empty_like(F)
        with eik.Plan(I.nx, I.ny, I.h, k, eik.EIK_FP64) as p:
            rc, _ = p.solve(F, src, q, Uref)
        assert rc == 0
        V = Uref.cpu().numpy()
        desc = eik.make_desc(I.nx, I.ny, I.h, k, eik.EIK_FP64)
        for call in range(2):
            U = torch.full_like(F, -7.0)
            rc, st = eik.eik_solve_noalloc(desc, eik.make_instance(F, src, q, U))
            assert rc == 0, eik.eik_strerror(rc)
            assert st.status == 0
            _close(U.cpu().numpy(), V, f"{I.name} call {call}")


def test_noalloc_rejects_what_it_cannot_do_without_allocating(eik):
    import torch
    I = W.const_point(65)
    F = torch.from_numpy(I.F).cuda()
    src = torch.from_numpy(I.src_ij).cuda()
    q = torch.from_numpy(I.sq).cuda()
    U = torch.empty_like(F)
    # a grid too large for the fixed scratch
    big = eik.make_desc(4097, 4097, 1 / 4096, 8, eik.EIK_FP64)
    rc, _ = eik.eik_solve_noalloc(big, eik.make_instance(F, src, q, U))
    assert rc == eik.EIK_EINVAL
    # host buffers would need staging memory
    Fh = np.ascontiguousarray(I.F)
    Uh = np.empty_like(Fh)
    desc = eik.make_desc(65, 65, I.h, 8, eik.EIK_FP64)
    rc, _ = eik.eik_solve_noalloc(desc, eik.make_instance(Fh, I.src_ij, I.sq, Uh))
    assert rc == eik.EIK_EINVAL
    # and the scratch is still usable afterwards
    rc, _ = eik.eik_solve_noalloc(desc, eik.make_instance(F, src, q, U))
    assert rc == 0
