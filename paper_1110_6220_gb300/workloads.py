"""Seeded synthetic inputs shaped like the paper's examples.

This module produces problem data only -- speed fields F, source sets and
request streams.  It holds none of the solver's arithmetic, so both the CUDA
path and the CPU oracle may consume what it makes.

Grid convention: an n x n grid on [0,1]^2, nodes x_i = i*h, h = 1/(n-1); F is
returned as a float64 array of shape (ny, nx) with node (i, j) at F[j, i].

Workloads (Sec. 5 of the paper gives the shapes):
  * ``const_point``   -- F == 1, one source at the centre (Sec. 5.3, Tab. const).
  * ``sin_point``     -- F = 1 + A sin(w pi x) sin(w pi y), centre source
                         (Sec. 5.3, Tab. sinu_1 uses A = 0.5, w = 20).
  * ``checker_maze``  -- 64x64 checkerboard of F in {1,2} (Sec. 5.2 shape) plus
                         a seeded maze of 1-node-thick F = 0 walls with gaps
                         (after the comb mazes of Sec. 5.1), 4 seeded sources.
  * ``batch_mix``     -- many grids of log-uniform side length, either a
                         sin-product or random piecewise-constant blocks.
  * ``poisson_stream``-- seeded Poisson arrival times of mixed requests.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Instance:
    nx: int
    ny: int
    h: float
    F: np.ndarray          # (ny, nx) float64, >= 0, 0 = obstacle
    si: np.ndarray         # int32 source x-indices
    sj: np.ndarray         # int32 source y-indices
    sq: np.ndarray         # float64 source values
    name: str = ""

    @property
    def npts(self) -> int:
        return self.nx * self.ny

    @property
    def src_ij(self) -> np.ndarray:
        """Sources as an interleaved (i, j) int32 array of length 2*nsrc."""
        return np.ascontiguousarray(np.stack([self.si, self.sj], axis=1).reshape(-1),
                                    dtype=np.int32)


def _grid(n):
    h = 1.0 / (n - 1)
    x = np.arange(n, dtype=np.float64) * h
    return h, x


def const_point(n: int = 129, F0: float = 1.0) -> Instance:
    h, _ = _grid(n)
    c = (n - 1) // 2
    F = np.full((n, n), F0, dtype=np.float64)
    return Instance(n, n, h, F, np.array([c], np.int32), np.array([c], np.int32),
                    np.zeros(1), name=f"const{n}")


def sin_field(n: int, omega: float, amp: float) -> np.ndarray:
    _, x = _grid(n)
    sx = np.sin(omega * math.pi * x)
    return 1.0 + amp * np.outer(sx, sx)  # symmetric: F[j, i] = 1 + A s(x_i) s(y_j)


def sin_point(n: int = 1025, omega: float = 20.0, amp: float = 0.5) -> Instance:
    h, _ = _grid(n)
    c = (n - 1) // 2
    return Instance(n, n, h, sin_field(n, omega, amp), np.array([c], np.int32),
                    np.array([c], np.int32), np.zeros(1), name=f"sin{int(omega)}_{n}")


def boundary_nodes(n: int):
    """(i, j) of every node on the boundary of an n x n grid, each once."""
    k = np.arange(n)
    i = np.concatenate([k, k, np.zeros(n - 2, int), np.full(n - 2, n - 1)])
    j = np.concatenate([np.zeros(n, int), np.full(n, n - 1), k[1:-1], k[1:-1]])
    return i.astype(np.int32), j.astype(np.int32)


def sin_boundary(n: int = 1025, omega: float = 20.0, amp: float = 0.5) -> Instance:
    """Sec. 5's general boundary conditions: F = 1 + amp sin(omega pi x)
    sin(omega pi y) with q = 0 on the whole boundary of the square (Q = dOmega)."""
    h, _ = _grid(n)
    si, sj = boundary_nodes(n)
    return Instance(n, n, h, sin_field(n, omega, amp), si, sj, np.zeros(si.size),
                    name=f"sin{int(omega)}_gbc_{n}")


def checker_field(n: int, checkers: int = 64, lo: float = 1.0, hi: float = 2.0) -> np.ndarray:
    _, x = _grid(n)
    b = np.minimum(np.floor(checkers * x).astype(np.int64), checkers - 1)
    par = (b[None, :] + b[:, None]) % 2
    return np.where(par == 0, lo, hi).astype(np.float64)


def maze_walls(n: int, rng: np.random.Generator, n_walls: int = 32, gap_w: int = 8,
               p_gap: float = 0.65) -> np.ndarray:
    """Boolean (ny, nx) mask of 1-node-thick axis-aligned walls on ``n_walls``
    distinct seeded rows and as many columns.  The walls cut the square into
    rooms; every wall segment between two crossing walls gets one opening
    ``gap_w`` nodes wide with probability ``p_gap`` (above the bond-percolation
    threshold 1/2, so most rooms connect through winding paths, as in the comb
    mazes of Sec. 5.1)."""
    wall = np.zeros((n, n), dtype=bool)
    lines = np.arange(2, n - 2)
    n_walls = min(n_walls, lines.size // 4)
    rows = np.sort(rng.choice(lines, size=n_walls, replace=False))
    cols = np.sort(rng.choice(lines, size=n_walls, replace=False))
    wall[rows, :] = True
    wall[:, cols] = True

    def cut(line_is_row, k, cross):
        edges = np.concatenate([[-1], cross, [n]])
        for a, b in zip(edges[:-1], edges[1:]):
            lo, hi = a + 1, b  # open interval of the segment
            if hi - lo < gap_w + 2 or rng.random() >= p_gap:
                continue
            s0 = int(rng.integers(lo, hi - gap_w + 1))
            if line_is_row:
                wall[k, s0:s0 + gap_w] = False
            else:
                wall[s0:s0 + gap_w, k] = False

    for r in rows:
        cut(True, r, cols)
    for c in cols:
        cut(False, c, rows)
    wall[rows[:, None], cols[None, :]] = True  # crossings stay closed
    return wall


def checker_maze(n: int = 4097, seed: int = 1, n_walls: int = 32, n_src: int = 4) -> Instance:
    rng = np.random.default_rng(seed)
    h, _ = _grid(n)
    F = checker_field(n)
    wall = maze_walls(n, rng, n_walls=n_walls)
    F[wall] = 0.0
    free = np.flatnonzero(~wall.reshape(-1))
    pick = rng.choice(free, size=n_src, replace=False)
    sj, si = np.divmod(pick, n)
    return Instance(n, n, h, F, si.astype(np.int32), sj.astype(np.int32),
                    np.zeros(n_src), name=f"checkermaze{n}_s{seed}")


def block_field(n: int, rng: np.random.Generator, B: int, lo: float = 0.5,
                hi: float = 2.0) -> np.ndarray:
    nb = -(-n // B)
    vals = rng.uniform(lo, hi, size=(nb, nb))
    idx = np.arange(n) // B
    return vals[idx[:, None], idx[None, :]].astype(np.float64)


def random_instance(rng: np.random.Generator, n_lo: int, n_hi: int,
                    kinds=("sin", "blocks")) -> Instance:
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    n = max(n, 2)
    h, _ = _grid(n)
    kind = kinds[int(rng.integers(0, len(kinds)))]
    if kind == "sin":
        F = sin_field(n, float(rng.uniform(2.0, 30.0)), 0.5)
    elif kind == "blocks":
        F = block_field(n, rng, int(rng.integers(4, 65)))
    elif kind == "checkermaze":
        F = checker_field(n)
        F[maze_walls(n, rng, n_walls=max(1, n // 128))] = 0.0
    else:
        raise ValueError(kind)
    ns = int(rng.integers(1, 9))
    cand = np.flatnonzero(F.reshape(-1) > 0)
    pick = rng.choice(cand, size=min(ns, cand.size), replace=False)
    sj, si = np.divmod(pick, n)
    return Instance(n, n, h, F, si.astype(np.int32), sj.astype(np.int32),
                    np.zeros(pick.size), name=f"{kind}{n}")


def batch_mix(count: int = 512, seed: int = 1, n_lo: int = 65, n_hi: int = 1025):
    rng = np.random.default_rng(seed)
    return [random_instance(rng, n_lo, n_hi) for _ in range(count)]


def poisson_stream(count: int, rate_per_s: float, seed: int = 1, n_lo: int = 129,
                   n_hi: int = 2049):
    """(arrival_time_s, Instance) pairs; speed types as in the sin, block and
    checker-maze workloads in equal shares."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
    kinds = ("sin", "blocks", "checkermaze")
    return [(float(t[i]), random_instance(rng, n_lo, n_hi, kinds)) for i in range(count)]


def tiny_random(rng: np.random.Generator, n_max: int = 17, obstacle_frac: float = 0.1):
    """Tiny random grid for brute-force cross-checks: F uniform in [0.5, 2]
    with some obstacles, 1-3 sources with random q in [0, 0.1]."""
    nx = int(rng.integers(2, n_max + 1))
    ny = int(rng.integers(2, n_max + 1))
    F = rng.uniform(0.5, 2.0, size=(ny, nx))
    F[rng.random((ny, nx)) < obstacle_frac] = 0.0
    ns = int(rng.integers(1, 4))
    pick = rng.choice(nx * ny, size=min(ns, nx * ny), replace=False)
    sj, si = np.divmod(pick, nx)
    sq = rng.uniform(0.0, 0.1, size=pick.size)
    return Instance(nx, ny, 1.0 / (max(nx, ny) - 1), F, si.astype(np.int32),
                    sj.astype(np.int32), sq, name=f"tiny{nx}x{ny}")
