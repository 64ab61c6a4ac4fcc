"""ctypes wrapper over ``eik_oracle.c`` (plain C, FP64, -O2 -ffp-contract=off).

TEST INFRASTRUCTURE ONLY: the product path never imports this module.

Functions follow the paper (Chacon & Vladimirsky, "Fast two-scale methods for
Eikonal equations"):
  * ``fmm``      -- Alg. FMM (Sec. 3.1), binary heap;
  * ``fsm``      -- Algs. FSM_order / FSM (Sec. 3.2), Gauss-Seidel in 4 directions;
  * ``lsm``      -- the Locking Sweeping Method (Remark locking_FSM);
  * ``cells``    -- the Heap-Cell Methods HCM / FHCM (Secs. 4.2, 4.3), HCM also
    with locking inside cells;
  * ``fmsm``     -- the Fast Marching-Sweeping Method (Sec. 4.1, Alg. FMSM);
  * ``jacobi``   -- value iteration from +inf (eq. generic_value_it) on eq. Eik_discr;
  * ``apply_T``  -- one application of the local update operator of eq. Eik_discr;
  * ``node_update`` -- the local update at one node (eqs. one_sided_update,
    two_sided_update, min over the four quadrants).

Arrays are ``(ny, nx)`` float64, node (i, j) at ``[j, i]`` (x fastest in memory).
Sources are given as integer arrays ``si``, ``sj`` and float ``sq``.

``Oracle.from_source(text)`` compiles a modified copy of the C source; the
test-suite uses it to plant mistakes in the oracle and check that the pins
catch them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "eik_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC", "-shared"]
_lock = threading.Lock()
_default = None


class OracleError(RuntimeError):
    pass


def _compile(src_path: str, out_path: str) -> None:
    tmp = out_path + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", *_CFLAGS, "-o", tmp, src_path, "-lm"], check=True)
    os.replace(tmp, out_path)


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, no GPU needed)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(SOURCE)):
        return _LIB
    _compile(SOURCE, _LIB)
    return _LIB


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _args(F, h, si, sj, sq):
    F = np.ascontiguousarray(F, dtype=np.float64)
    if F.ndim != 2:
        raise ValueError("F must be 2-D (ny, nx)")
    ny, nx = F.shape
    si = np.ascontiguousarray(np.atleast_1d(si), dtype=np.int32)
    sj = np.ascontiguousarray(np.atleast_1d(sj), dtype=np.int32)
    sq = np.ascontiguousarray(np.atleast_1d(sq), dtype=np.float64)
    if not (si.shape == sj.shape == sq.shape):
        raise ValueError("si, sj, sq must have the same length")
    keep = (F, si, sj, sq)
    args = [nx, ny, float(h), _ptr(F, ctypes.c_double), int(si.size),
            _ptr(si, ctypes.c_int32), _ptr(sj, ctypes.c_int32),
            _ptr(sq, ctypes.c_double)]
    return keep, args, (ny, nx)


def _check(rc, what):
    if rc == -6:
        raise OracleError(f"{what}: did not converge")
    if rc != 0:
        raise OracleError(f"{what}: error {rc}")


class Oracle:
    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        P = ctypes.POINTER
        common = [ctypes.c_int, ctypes.c_int, d, P(d), ctypes.c_int, P(i32), P(i32), P(d)]
        lib.orc_fmm.argtypes = common + [P(d), P(i64)]
        lib.orc_fsm.argtypes = common + [P(d), i32, P(i32)]
        lib.orc_lsm.argtypes = common + [P(d), i32, P(i32), P(i64)]
        lib.orc_jacobi.argtypes = common + [P(d), i32, P(i32)]
        lib.orc_apply_T.argtypes = common + [P(d), P(d)]
        lib.orc_node_update.argtypes = [d, d, d, d, d]
        lib.orc_node_update.restype = d
        lib.orc_cells.argtypes = common + [ctypes.c_int, ctypes.c_int, P(d), P(i64)]
        lib.orc_fmsm.argtypes = common + [ctypes.c_int, P(d), P(d), P(i32), P(i32), P(i64)]
        for fn in (lib.orc_fmm, lib.orc_fsm, lib.orc_lsm, lib.orc_jacobi, lib.orc_apply_T, lib.orc_cells, lib.orc_fmsm):
            fn.restype = ctypes.c_int
        self.lib = lib
        self.path = lib_path

    @classmethod
    def from_source(cls, text: str) -> "Oracle":
        """Compile a (modified) copy of the oracle source into a private
        library; used only to plant mistakes in tests."""
        tmpdir = tempfile.mkdtemp(prefix="orc_variant_")
        src = os.path.join(tmpdir, "variant.c")
        with open(src, "w") as fh:
            fh.write(text)
        out = os.path.join(tmpdir, "variant.so")
        _compile(src, out)
        return cls(out)

    def fmm(self, F, h, si, sj, sq, return_count=False):
        """Fast Marching (Alg. FMM).  Returns U (ny, nx)."""
        keep, args, shape = _args(F, h, si, sj, sq)
        U = np.empty(shape, dtype=np.float64)
        n_acc = ctypes.c_int64(0)
        _check(self.lib.orc_fmm(*args, _ptr(U, ctypes.c_double), ctypes.byref(n_acc)), "fmm")
        del keep
        return (U, n_acc.value) if return_count else U

    def fsm(self, F, h, si, sj, sq, max_sweeps=100000, return_sweeps=False):
        """Fast Sweeping (Algs. FSM_order, FSM).  Returns U (and the sweep
        count, which includes the final sweep that changed nothing)."""
        keep, args, shape = _args(F, h, si, sj, sq)
        U = np.empty(shape, dtype=np.float64)
        ns = ctypes.c_int32(0)
        _check(self.lib.orc_fsm(*args, _ptr(U, ctypes.c_double), int(max_sweeps),
                                ctypes.byref(ns)), "fsm")
        del keep
        return (U, ns.value) if return_sweeps else U

    def lsm(self, F, h, si, sj, sq, max_sweeps=100000):
        """Locking Sweeping (Remark locking_FSM).  Returns U and
        {'sweeps', 'evals' (local updates computed)}."""
        keep, args, shape = _args(F, h, si, sj, sq)
        U = np.empty(shape, dtype=np.float64)
        ns, ne = ctypes.c_int32(0), ctypes.c_int64(0)
        _check(self.lib.orc_lsm(*args, _ptr(U, ctypes.c_double), int(max_sweeps), ctypes.byref(ns),
                                ctypes.byref(ne)), "lsm")
        del keep
        return U, {"sweeps": ns.value, "evals": ne.value}

    def cells(self, F, h, si, sj, sq, k, fast=False, lsm=False):
        """Heap-Cell Method (Sec. 4.2; exact) on k x k cells, its cells
        swept with locking flags (lsm=True; the same values), or the Fast
        Heap-Cell Method (Sec. 4.3, Alg. FHCM; fast=True, inexact).  Returns U
        and {'avhr', 'avs', 'mon_pct', 'removals', 'sweeps', 'evals'}."""
        if fast and lsm:
            raise ValueError("fast and lsm exclude each other")
        keep, args, shape = _args(F, h, si, sj, sq)
        U = np.empty(shape, dtype=np.float64)
        st = np.zeros(5, dtype=np.int64)
        method = 1 if fast else 2 if lsm else 0
        _check(self.lib.orc_cells(*args, int(k), method, _ptr(U, ctypes.c_double),
                                  _ptr(st, ctypes.c_int64)), "cells")
        del keep
        ny, nx = shape
        J = ((nx + k - 1) // k) * ((ny + k - 1) // k)
        return U, {"removals": int(st[0]), "sweeps": int(st[1]), "avhr": st[0] / J, "avs": st[1] / J,
                   "mon_pct": 100.0 * st[2] / st[3] if st[3] else 100.0, "evals": int(st[4])}

    def fmsm(self, F, h, si, sj, sq, k):
        """Fast Marching-Sweeping Method (Sec. 4.1, Alg. FMSM) on k x k cells
        (inexact).  Returns U and {'avs', 'sweeps', 'cells', 'accepted',
        'order' (cell indices in processing order), 'Uc' (coarse values,
        (cyn, cxn)), 'dirs' (per cell the sweep directions, bit d for
        direction d of Alg. FSM_order, 16 for a cell swept by Alg. FSM)}."""
        keep, args, shape = _args(F, h, si, sj, sq)
        ny, nx = shape
        cxn, cyn = (nx + k - 1) // k, (ny + k - 1) // k
        U = np.empty(shape, dtype=np.float64)
        Uc = np.empty((cyn, cxn), dtype=np.float64)
        order = np.empty(cxn * cyn, dtype=np.int32)
        dirs = np.zeros((cyn, cxn), dtype=np.int32)
        st = np.zeros(3, dtype=np.int64)
        _check(self.lib.orc_fmsm(*args, int(k), _ptr(U, ctypes.c_double), _ptr(Uc, ctypes.c_double),
                                 _ptr(order, ctypes.c_int32), _ptr(dirs, ctypes.c_int32),
                                 _ptr(st, ctypes.c_int64)), "fmsm")
        del keep
        return U, {"cells": int(st[0]), "sweeps": int(st[1]), "avs": st[1] / max(int(st[0]), 1),
                   "accepted": int(st[2]), "order": order, "Uc": Uc, "dirs": dirs}

    def jacobi(self, F, h, si, sj, sq, max_iters=1_000_000, return_iters=False):
        """Jacobi value iteration from +inf; only sensible on tiny grids."""
        keep, args, shape = _args(F, h, si, sj, sq)
        U = np.empty(shape, dtype=np.float64)
        it = ctypes.c_int32(0)
        _check(self.lib.orc_jacobi(*args, _ptr(U, ctypes.c_double), int(max_iters),
                                   ctypes.byref(it)), "jacobi")
        del keep
        return (U, it.value) if return_iters else U

    def apply_T(self, F, h, si, sj, sq, V):
        """One application of the update operator T: (T V) = q on sources,
        the local update from V's neighbours elsewhere."""
        keep, args, shape = _args(F, h, si, sj, sq)
        V = np.ascontiguousarray(V, dtype=np.float64)
        if V.shape != shape:
            raise ValueError("V shape mismatch")
        TV = np.empty(shape, dtype=np.float64)
        _check(self.lib.orc_apply_T(*args, _ptr(V, ctypes.c_double),
                                    _ptr(TV, ctypes.c_double)), "apply_T")
        del keep
        return TV

    def node_update(self, ue, uw, un, us, f):
        """The local update at one node from its E, W, N, S neighbour values."""
        return self.lib.orc_node_update(float(ue), float(uw), float(un), float(us), float(f))


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def fmm(*a, **k):
    return default().fmm(*a, **k)


def fsm(*a, **k):
    return default().fsm(*a, **k)


def lsm(*a, **k):
    return default().lsm(*a, **k)


def fmsm(*a, **k):
    return default().fmsm(*a, **k)


def jacobi(*a, **k):
    return default().jacobi(*a, **k)


def cells(*a, **k):
    return default().cells(*a, **k)


def apply_T(*a, **k):
    return default().apply_T(*a, **k)


def node_update(*a, **k):
    return default().node_update(*a, **k)
