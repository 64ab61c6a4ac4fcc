"""A single grid split into horizontal slabs, one per rank: the multi-GPU
form of the solve.

Sec. 4's cell decomposition already treats a cell as a subproblem whose
boundary data are its neighbours' current values, and Theorem convergence
makes label correcting over such subproblems exact for any order in which
they are processed.  A slab is a band of whole rows of cells; each rank
solves its slab with the rows just outside it (its "ghost rows") held at the
neighbouring slab's latest boundary values, then the ranks exchange their
boundary rows and solve again, until no ghost value changes anywhere.

The local problem of a slab covering grid rows [r0, r1) has one extra row
on each side that has a neighbour: ghost nodes with a finite value are
sources with q = that value (fixed, as Sec. 3's exit set), the others are
obstacles (F = 0, held at +inf).  Values only decrease from one round to the
next (every local solution is monotone in its boundary data), so the rounds
end; at the end every slab satisfies eq. Eik_discr with its neighbours'
final values, which is the whole grid's system -- its unique solution.

The exchange needs one collective per round: each rank sends its first and
last rows to its neighbours (point-to-point) and all ranks agree whether
anything changed (an all-reduce).  `Comm` wraps torch.distributed for real
ranks; `LocalComm` runs the same protocol for P slabs inside one process
(one GPU solving the slabs one after another), with no waiting between
kernels.

The local solve is a function (F, h, si, sj, sq) -> U; the default is the
library's own (eik.solve on the CUDA path)."""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Slab:
    r0: int   # first grid row of the slab
    r1: int   # one past its last row
    lo: bool  # a neighbour below (rows < r0)
    hi: bool  # a neighbour above (rows >= r1)


def partition(ny: int, nranks: int, k: int = 8) -> list[Slab]:
    """Rows [0, ny) split into nranks bands of whole rows of k-node cells
    (the last band takes the remainder), as even as the cells allow."""
    if nranks < 1:
        raise ValueError("nranks >= 1")
    cells = (ny + k - 1) // k
    if nranks > cells:
        raise ValueError(f"{nranks} slabs for {cells} rows of cells")
    cuts = [min(ny, (cells * r // nranks) * k) for r in range(nranks + 1)]
    cuts[-1] = ny
    return [Slab(cuts[r], cuts[r + 1], r > 0, r < nranks - 1) for r in range(nranks)]


def local_problem(F, sources, slab: Slab, ghost_lo, ghost_hi):
    """The slab's own problem: its rows of F plus one ghost row per
    neighbour (F = 0 there: obstacles held at +inf, except the finite ghost
    values, which are sources).  sources: (si, sj, sq) of the whole grid.
    Returns (F_local, si, sj, sq, row offset of the slab's first row)."""
    si, sj, sq = sources
    a = slab.r0 - (1 if slab.lo else 0)
    b = slab.r1 + (1 if slab.hi else 0)
    Fl = np.array(F[a:b], dtype=np.float64, copy=True)
    off = slab.r0 - a
    keep = (sj >= slab.r0) & (sj < slab.r1)
    li, lj, lq = [si[keep]], [sj[keep] - a], [sq[keep]]
    for on, row, g in ((slab.lo, 0, ghost_lo), (slab.hi, b - a - 1, ghost_hi)):
        if not on:
            continue
        Fl[row, :] = 0.0
        fin = np.isfinite(g)
        li.append(np.nonzero(fin)[0].astype(np.int32))
        lj.append(np.full(int(fin.sum()), row, dtype=np.int32))
        lq.append(g[fin])
    return (Fl, np.concatenate(li).astype(np.int32), np.concatenate(lj).astype(np.int32),
            np.concatenate(lq).astype(np.float64), off)


class LocalComm:
    """The exchange for P slabs solved in one process: rank r's boundary
    rows are handed to its neighbours directly."""

    def __init__(self, nranks: int):
        self.nranks = nranks

    def exchange(self, lows, highs):
        """lows[r] / highs[r]: rank r's first / last row (None at the grid's
        edge).  Returns (ghost_lo, ghost_hi) per rank: the row below it (the
        last row of rank r - 1) and the row above it (the first row of r + 1)."""
        P = self.nranks
        glo = [highs[r - 1] if r > 0 else None for r in range(P)]
        ghi = [lows[r + 1] if r < P - 1 else None for r in range(P)]
        return glo, ghi

    def any(self, flags):
        return any(flags)


class Comm:
    """The exchange over torch.distributed (one rank per slab): point-to-point
    sends of the boundary rows to the neighbours, an all-reduce for the
    global "anything changed" -- the only collective of a round."""

    def __init__(self, group=None, device="cpu"):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.nranks = dist.get_world_size(group)
        self.device = device

    def exchange_one(self, low, high, width):
        import torch
        dist = self.dist
        r, P = self.rank, self.nranks
        ops = []
        glo = torch.empty(width, dtype=torch.float64, device=self.device) if r > 0 else None
        ghi = torch.empty(width, dtype=torch.float64, device=self.device) if r < P - 1 else None
        peer = (lambda q: q) if self.group is None else (lambda q: dist.get_global_rank(self.group, q))
        if r > 0:
            ops.append(dist.P2POp(dist.isend, torch.as_tensor(low, device=self.device), peer(r - 1), self.group))
            ops.append(dist.P2POp(dist.irecv, glo, peer(r - 1), self.group))
        if r < P - 1:
            ops.append(dist.P2POp(dist.isend, torch.as_tensor(high, device=self.device), peer(r + 1), self.group))
            ops.append(dist.P2POp(dist.irecv, ghi, peer(r + 1), self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return (glo.cpu().numpy() if glo is not None else None,
                ghi.cpu().numpy() if ghi is not None else None)

    def any_one(self, flag):
        import torch
        t = torch.tensor([1 if flag else 0], dtype=torch.int32, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return bool(t.item())


def _default_local_solver(cell_k):
    from . import eik

    def solve(F, h, si, sj, sq):
        U, st = eik.solve(F, h, si, sj, sq, cell_k=cell_k, precision=eik.EIK_FP64)
        return U
    return solve


def solve_slabs(F, h, si, sj, sq, nranks, local_solve=None, cell_k=8, max_rounds=10000):
    """All P slabs in one process (LocalComm): the same rounds as the
    distributed form.  Returns (U of the whole grid, rounds)."""
    F = np.asarray(F, dtype=np.float64)
    ny, nx = F.shape
    src = (np.asarray(si, np.int32), np.asarray(sj, np.int32), np.asarray(sq, np.float64))
    slabs = partition(ny, nranks, cell_k)
    solve = local_solve or _default_local_solver(cell_k)
    comm = LocalComm(nranks)
    inf = np.full(nx, np.inf)
    glo = [inf.copy() if s.lo else None for s in slabs]
    ghi = [inf.copy() if s.hi else None for s in slabs]
    U = np.full((ny, nx), np.inf)
    for rnd in range(1, max_rounds + 1):
        lows, highs = [], []
        for r, s in enumerate(slabs):
            Fl, li, lj, lq, off = local_problem(F, src, s, glo[r], ghi[r])
            Ul = solve(Fl, h, li, lj, lq)
            U[s.r0:s.r1] = Ul[off:off + (s.r1 - s.r0)]
            lows.append(U[s.r0].copy())
            highs.append(U[s.r1 - 1].copy())
        nlo, nhi = comm.exchange(lows, highs)
        changed = []
        for r in range(nranks):
            c = False
            if nlo[r] is not None:
                c |= not np.array_equal(np.minimum(glo[r], nlo[r]), glo[r])
                glo[r] = np.minimum(glo[r], nlo[r])
            if nhi[r] is not None:
                c |= not np.array_equal(np.minimum(ghi[r], nhi[r]), ghi[r])
                ghi[r] = np.minimum(ghi[r], nhi[r])
            changed.append(c)
        if not comm.any(changed):
            return U, rnd
    raise RuntimeError(f"slab rounds did not settle in {max_rounds}")


def solve_slab_rank(F, h, si, sj, sq, comm: Comm, local_solve=None, cell_k=8, max_rounds=10000):
    """This rank's slab of the distributed solve (every rank passes the
    whole problem; each solves and returns its own rows).  Returns (slab,
    U of the slab's rows, rounds)."""
    F = np.asarray(F, dtype=np.float64)
    ny, nx = F.shape
    src = (np.asarray(si, np.int32), np.asarray(sj, np.int32), np.asarray(sq, np.float64))
    s = partition(ny, comm.nranks, cell_k)[comm.rank]
    solve = local_solve or _default_local_solver(cell_k)
    glo = np.full(nx, np.inf) if s.lo else None
    ghi = np.full(nx, np.inf) if s.hi else None
    for rnd in range(1, max_rounds + 1):
        Fl, li, lj, lq, off = local_problem(F, src, s, glo, ghi)
        Ul = solve(Fl, h, li, lj, lq)
        mine = Ul[off:off + (s.r1 - s.r0)]
        nlo, nhi = comm.exchange_one(mine[0].copy(), mine[-1].copy(), nx)
        changed = False
        if nlo is not None:
            m = np.minimum(glo, nlo)
            changed |= not np.array_equal(m, glo)
            glo = m
        if nhi is not None:
            m = np.minimum(ghi, nhi)
            changed |= not np.array_equal(m, ghi)
            ghi = m
        if not comm.any_one(changed):
            return s, mine, rnd
    raise RuntimeError(f"slab rounds did not settle in {max_rounds}")
