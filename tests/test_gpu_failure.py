"""Failure paths and schedule checks, all driven from the host -- nothing
here faults, traps or hangs a GPU:

- EIK_ENOMEM: EIK_ALLOC_LIMIT makes every workspace allocation above it fail
  the way cudaMalloc would; plans, batches, fixed batches and served
  requests report it, and the library works again once it is lifted.
- EIK_ENOTCONVERGED: EIK_MAX_PASSES caps the passes of one removal, a cap a
  cell needs more than is reported, and the context stays usable; an
  FP32_REFINE tolerance the certificate cannot reach reports it too.
- Queue bookkeeping: after every converged solve, on every schedule and in
  every arithmetic mode, no cell is left requested or running
  (eik_stats.queue_left, counted on the device from the cells' flags).
- Schedule perturbation: EIK_JITTER_NS pauses every removal by a random,
  bounded time before its tile load; the removal order changes, the result
  must not (Theorem convergence: any removal order reaches the unique
  solution of eq. Eik_discr)."""
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
    e.eik_tune_reset()
    return e


def _err(U, V):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all()
    return float(np.abs(U[fin] - V[fin]).max() / np.abs(V[fin]).max())


def test_enomem_from_a_host_allocation_limit(eik, orc, monkeypatch):
    I = W.sin_point(257)
    monkeypatch.setenv("EIK_ALLOC_LIMIT", "4096")
    with pytest.raises(eik.EikError) as e:
        eik.eik_plan_create(eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64))
    assert e.value.code == eik.EIK_ENOMEM
    src = I.src_ij
    U = np.empty_like(I.F)
    rc, _ = eik.eik_solve_batch([eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64)],
                                [eik.make_instance(I.F, src, I.sq, U)])
    assert rc == eik.EIK_ENOMEM
    with pytest.raises(eik.EikError) as e:
        eik.eik_batch_create([eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64)], [eik.make_instance(I.F, src, I.sq, U)])
    assert e.value.code == eik.EIK_ENOMEM
    srv = eik.eik_server_create(1 << 30, 4)
    try:
        rc, t = eik.eik_submit(srv, eik.make_desc(I.nx, I.ny, I.h, 8, eik.EIK_FP64), eik.make_instance(I.F, src, I.sq, U))
        assert rc == 0
        import time
        for _ in range(20000):
            rc, st = eik.eik_poll(srv, t)
            if rc != eik.EIK_EAGAIN:
                break
            time.sleep(1e-4)
        assert rc == eik.EIK_ENOMEM
    finally:
        eik.eik_server_destroy(srv)
    monkeypatch.delenv("EIK_ALLOC_LIMIT")
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=0)
    assert st.status == 0 and _err(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq)) <= TOL64


@pytest.mark.parametrize("sched", ["ROUNDS", "FIFO", "ORDERED"])
def test_enotconverged_from_a_pass_cap(eik, orc, monkeypatch, sched):
    """One pass per removal is too few for a cell that an upstream change
    reaches on a side its sweeps meet last; the cap is reported, every wait
    still ends, and the next solve without the cap is exact."""
    I = W.checker_maze(257, seed=3, n_walls=6, n_src=3)
    s = getattr(eik, f"EIK_SCHED_{sched}")
    monkeypatch.setenv("EIK_MAX_PASSES", "1")
    with eik.Plan(I.nx, I.ny, I.h, 16, eik.EIK_FP64, schedule=s) as p:
        U = np.empty_like(I.F)
        rc, st = p.solve(I.F, I.src_ij, I.sq, U)
    assert rc == eik.EIK_ENOTCONVERGED, eik.eik_strerror(rc)
    monkeypatch.delenv("EIK_MAX_PASSES")
    U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=16, precision=0, schedule=s)
    assert st.status == 0 and st.queue_left == 0
    assert _err(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq)) <= TOL64


def test_enotconverged_when_the_certificate_misses_the_tolerance(eik, orc):
    """FP32_REFINE certifies its result against the tolerance asked for; a
    tolerance below what double-float arithmetic reaches is reported as not
    certified, with the result still within the certificate it computed."""
    I = W.sin_point(257)
    with eik.Plan(I.nx, I.ny, I.h, 8, eik.EIK_FP32_REFINE, tol=1e-13) as p:
        U = np.empty_like(I.F)
        rc, st = p.solve(I.F, I.src_ij, I.sq, U)
    assert rc == eik.EIK_ENOTCONVERGED
    assert 1e-13 < st.err_bound <= 1e-5
    assert _err(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq)) <= st.err_bound * 1.0001


@pytest.mark.parametrize("sched", ["ROUNDS", "FIFO", "ORDERED"])
@pytest.mark.parametrize("prec,one_pass", [(0, 0), (1, 0), (1, 1)], ids=["fp64", "fp32_then_df", "df_one_pass"])
def test_no_cell_left_queued_after_a_solve(eik, monkeypatch, sched, prec, one_pass):
    monkeypatch.setenv("EIK_ONE_PASS", "1" if one_pass else "0")
    s = getattr(eik, f"EIK_SCHED_{sched}")
    rng = np.random.default_rng(11)
    for I in [W.sin_point(257), W.checker_maze(257, seed=3, n_walls=6, n_src=3), W.tiny_random(rng, n_max=40)]:
        for k in (8, 16):
            U, st = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=k, precision=prec, schedule=s)
            assert st.status == 0, eik.eik_strerror(st.status)
            assert st.queue_left == 0, (I.name, k)
    # a batch on one launch
    insts = W.batch_mix(16, seed=9, n_lo=17, n_hi=200)
    keep = [(I, np.empty_like(I.F), I.src_ij) for I in insts]
    rc, sts = eik.eik_solve_batch([eik.make_desc(I.nx, I.ny, I.h, 16, prec, schedule=s) for I, _, _ in keep],
                                  [eik.make_instance(I.F, src, I.sq, U) for I, U, src in keep])
    assert rc == 0
    assert all(x.queue_left == 0 for x in sts)


@pytest.mark.parametrize("sched", ["ROUNDS", "FIFO", "ORDERED"])
def test_result_does_not_depend_on_a_perturbed_schedule(eik, orc, monkeypatch, sched):
    """Random pauses of up to 3 us before each removal's tile load reorder
    the removals (the visits change); the FP64 result stays within the
    oracle's tolerance, node by node, and so does the double-float one."""
    s = getattr(eik, f"EIK_SCHED_{sched}")
    for I in [W.sin_point(257), W.checker_maze(257, seed=3, n_walls=6, n_src=3)]:
        V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
        U0, s0 = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=0, schedule=s)
        monkeypatch.setenv("EIK_JITTER_NS", "3000")
        U1, s1 = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=8, precision=0, schedule=s)
        U2, s2 = eik.solve(I.F, I.h, I.si, I.sj, I.sq, cell_k=16, precision=1, schedule=s)
        monkeypatch.delenv("EIK_JITTER_NS")
        assert s0.status == 0 and s1.status == 0 and s2.status == 0
        assert _err(U0, V) <= TOL64 and _err(U1, V) <= TOL64, I.name
        assert _err(U2, V) <= s2.err_bound * 1.0001 and s2.err_bound <= 1e-5
        assert s1.queue_left == 0 and s2.queue_left == 0
