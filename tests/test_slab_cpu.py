"""The slab split of one grid over ranks (paper_1110_6220_gb300/slab.py),
checked on the CPU: the partition, the local problems with their ghost rows,
and the rounds of local solves and boundary exchanges -- in one process and
over 2 and 4 gloo ranks -- reach the whole grid's solution of eq. Eik_discr.

The local solves here are the oracle's Fast Marching (test infrastructure);
on GPUs each rank calls the library's solve instead (tests/test_gpu_slab.py
runs that form on one GPU, slab after slab).  The exchange protocol and the
termination are the same code."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _instances():
    from paper_1110_6220_gb300 import workloads as W
    rng = np.random.default_rng(8)
    return [W.sin_point(65), W.checker_maze(97, seed=2, n_walls=6, n_src=3),
            W.random_instance(rng, 60, 90, kinds=("blocks",)), W.sin_boundary(49)]


def _rel(U, V):
    fin = np.isfinite(V)
    assert (np.isfinite(U) == fin).all()
    return float(np.abs(U[fin] - V[fin]).max() / np.abs(V[fin]).max())


def test_partition_covers_the_rows_in_whole_cells():
    from paper_1110_6220_gb300 import slab
    for ny, P, k in ((65, 1, 8), (65, 2, 8), (129, 4, 8), (100, 3, 16), (17, 3, 4)):
        s = slab.partition(ny, P, k)
        assert len(s) == P and s[0].r0 == 0 and s[-1].r1 == ny
        for a, b in zip(s, s[1:]):
            assert a.r1 == b.r0 and b.r0 % k == 0
        assert all(x.r1 > x.r0 for x in s)
        assert [x.lo for x in s] == [r > 0 for r in range(P)]
        assert [x.hi for x in s] == [r < P - 1 for r in range(P)]
    with pytest.raises(ValueError):
        slab.partition(16, 3, 8)  # 2 rows of cells for 3 slabs


def test_local_problem_ghost_rows():
    """Finite ghost values become sources on obstacle nodes of the extra
    rows, +inf ones stay obstacles; the slab's own sources are kept, shifted
    into its rows."""
    from paper_1110_6220_gb300 import slab
    F = np.ones((20, 6))
    s = slab.Slab(8, 16, True, True)
    lo = np.array([1.0, np.inf, 2.0, np.inf, np.inf, 3.0])
    hi = np.full(6, np.inf)
    src = (np.array([2, 4], np.int32), np.array([3, 9], np.int32), np.array([0.0, 0.5]))
    Fl, si, sj, sq, off = slab.local_problem(F, src, s, lo, hi)
    assert Fl.shape == (10, 6) and off == 1
    assert (Fl[0] == 0).all() and (Fl[-1] == 0).all() and (Fl[1:-1] == 1).all()
    got = sorted(zip(si.tolist(), sj.tolist(), sq.tolist()))
    assert got == sorted([(4, 2, 0.5), (0, 0, 1.0), (2, 0, 2.0), (5, 0, 3.0)])


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_slabs_in_one_process_match_the_whole_grid(orc, P):
    from paper_1110_6220_gb300 import slab
    for I in _instances():
        V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
        U, rounds = slab.solve_slabs(I.F, I.h, I.si, I.sj, I.sq, P, local_solve=orc.fmm, cell_k=8)
        assert _rel(U, V) <= TOL, (I.name, P)
        assert rounds >= 1 and (P > 1 or rounds == 1)


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1110_6220_gb300 import slab
        orc = oracle.default()
        res = []
        for I in _instances():
            s, rows, rounds = slab.solve_slab_rank(I.F, I.h, I.si, I.sj, I.sq, slab.Comm(), local_solve=orc.fmm,
                                                   cell_k=8)
            res.append((I.name, s.r0, s.r1, rows, rounds))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slabs_over_gloo_ranks_match_the_whole_grid(orc, world):
    """Each rank solves its slab and trades boundary rows with its
    neighbours (point-to-point) until an all-reduce finds no change; the
    ranks' rows put together are the oracle's whole-grid solution, and all
    ranks stop after the same round."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for e, I in enumerate(_instances()):
        U = np.full(I.F.shape, np.nan)
        rounds = set()
        for r in range(world):
            name, r0, r1, rows, rnd = got[r][e]
            assert name == I.name
            U[r0:r1] = rows
            rounds.add(rnd)
        assert len(rounds) == 1
        assert not np.isnan(U).any()
        assert _rel(U, orc.fmm(I.F, I.h, I.si, I.sj, I.sq)) <= TOL, (I.name, world)
