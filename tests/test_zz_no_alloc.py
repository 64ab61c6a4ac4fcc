"""eik_solve_noalloc: the FP64 solve whose workspace is a fixed device array
inside the library, for callers that cannot call cudaMalloc (device memory
owned by another allocator or a fixed budget, or loops that cannot afford an
allocation's implicit synchronisation).

Its results must agree with the CPU oracle node by node and with the
plan-based entry point (eik_solve), within the FP64 parity tolerance, on
two calls in a row (the second call finds the first call's data in the
shared scratch and must not be misled by it); the calls after the first
must leave the device's free memory and torch's allocations as they were;
and what it cannot do without allocating is refused.  This file is named to
be collected last.
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


def test_noalloc_matches_oracle_and_plan_solve_on_two_calls(eik, orc):
    import torch
    cases = [(W.sin_point(257), 8), (W.checker_maze(200, seed=4, n_walls=4), 16)]
    for I, k in cases:
        F = torch.from_numpy(I.F).cuda()
        src = torch.from_numpy(I.src_ij).cuda()
        qh = I.sq + 0.25  # non-zero q exercises the shift
        q = torch.from_numpy(qh).cuda()
        V = orc.fmm(I.F, I.h, I.si, I.sj, qh)
        Uref = torch.empty_like(F)
        with eik.Plan(I.nx, I.ny, I.h, k, eik.EIK_FP64) as p:
            rc, _ = p.solve(F, src, q, Uref)
        assert rc == 0
        desc = eik.make_desc(I.nx, I.ny, I.h, k, eik.EIK_FP64)
        for call in range(2):
            U = torch.full_like(F, -7.0)
            rc, st = eik.eik_solve_noalloc(desc, eik.make_instance(F, src, q, U))
            assert rc == 0, eik.eik_strerror(rc)
            assert st.status == 0 and st.queue_left == 0
            _close(U.cpu().numpy(), V, f"{I.name} call {call} vs oracle")
            _close(U.cpu().numpy(), Uref.cpu().numpy(), f"{I.name} call {call} vs eik_solve")


def test_noalloc_allocates_nothing(eik):
    """After the first call on the device, further calls change neither the
    device's free memory nor what torch's allocator holds."""
    import torch
    I = W.sin_point(257)
    F = torch.from_numpy(I.F).cuda()
    src = torch.from_numpy(I.src_ij).cuda()
    q = torch.from_numpy(I.sq).cuda()
    U = torch.empty_like(F)
    desc = eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64)
    inst = eik.make_instance(F, src, q, U)
    rc, _ = eik.eik_solve_noalloc(desc, inst)
    assert rc == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    held0 = torch.cuda.memory_allocated()
    for _ in range(2):
        rc, _ = eik.eik_solve_noalloc(desc, inst)
        assert rc == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == held0


def test_noalloc_rejects_what_it_cannot_do_without_allocating(eik):
    import torch
    I = W.const_point(65)
    F = torch.from_numpy(I.F).cuda()
    src = torch.from_numpy(I.src_ij).cuda()
    q = torch.from_numpy(I.sq).cuda()
    U = torch.empty_like(F)
    desc = eik.make_desc(65, 65, I.h, 8, eik.EIK_FP64)
    # a grid too large for the fixed scratch
    big = eik.make_desc(4097, 4097, 1 / 4096, 8, eik.EIK_FP64)
    rc, _ = eik.eik_solve_noalloc(big, eik.make_instance(F, src, q, U))
    assert rc == eik.EIK_EINVAL
    # host buffers would need staging memory
    Fh = np.ascontiguousarray(I.F)
    Uh = np.empty_like(Fh)
    rc, _ = eik.eik_solve_noalloc(desc, eik.make_instance(Fh, I.src_ij, I.sq, Uh))
    assert rc == eik.EIK_EINVAL
    # more sources than its stack tables hold
    n = eik.EIK_NOALLOC_MAX_SOURCES + 1
    rng = np.random.default_rng(3)
    ij = torch.from_numpy(rng.integers(0, 65, size=2 * n).astype(np.int32)).cuda()
    qq = torch.zeros(n, dtype=torch.float64).cuda()
    rc, _ = eik.eik_solve_noalloc(desc, eik.make_instance(F, ij, qq, U))
    assert rc == eik.EIK_EINVAL
    ij256 = ij[: 2 * (n - 1)].contiguous()
    rc, _ = eik.eik_solve_noalloc(desc, eik.make_instance(F, ij256, qq[: n - 1].contiguous(), U))
    assert rc == 0
    # FP32_REFINE (its second pass's arrays) and the other methods are not offered
    for d in (eik.make_desc(65, 65, I.h, 8, eik.EIK_FP32_REFINE),
              eik.make_desc(65, 65, I.h, 8, eik.EIK_FP64, method=eik.EIK_METHOD_FHCM),
              eik.make_desc(65, 65, I.h, 8, eik.EIK_FP64, method=eik.EIK_METHOD_FMSM),
              eik.make_desc(65, 65, I.h, 8, eik.EIK_FP64, method=eik.EIK_METHOD_HCM_LSM)):
        rc, _ = eik.eik_solve_noalloc(d, eik.make_instance(F, src, q, U))
        assert rc == eik.EIK_EINVAL
    # a stream under capture cannot hold the call's copies and waits
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.capture_begin(capture_error_mode="relaxed")
        rc, _ = eik.eik_solve_noalloc(desc, eik.make_instance(F, src, q, U), s)
        g.capture_end()
    assert rc == eik.EIK_EINVAL
    # and the scratch is still usable afterwards
    rc, st = eik.eik_solve_noalloc(desc, eik.make_instance(F, src, q, U))
    assert rc == 0 and st.status == 0
