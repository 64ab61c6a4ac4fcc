"""ctypes binding of ``libeik.so`` (the C ABI declared in ``include/eik.h``).

Argument marshalling only: every step of the solve runs in the CUDA library.
Importing this module loads the library and raises ``ImportError`` if it has
not been built (``python -m paper_1110_6220_gb300.build``) -- there is no CPU
fallback.

Arrays may be NumPy arrays (host memory) or torch tensors (CPU or CUDA); the
library detects device pointers itself.  Grid arrays are (ny, nx) float64,
C-contiguous, node (i, j) at [j, i].
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeik.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libeik.so not built ({LIB_PATH}); run python -m paper_1110_6220_gb300.build")
_lib = ctypes.CDLL(LIB_PATH)

# ------------------------------------------------------------------ constants
EIK_OK = 0
EIK_EINVAL = -1
EIK_ENOMEM = -2
EIK_EBUSY = -3
EIK_EAGAIN = -4
EIK_ETIMEDOUT = -5
EIK_ENOTCONVERGED = -6
EIK_ECUDA = -7
EIK_FP64 = 0
EIK_FP32_REFINE = 1
EIK_METHOD_HCM = 0
EIK_METHOD_FHCM = 1
EIK_METHOD_FMSM = 2
EIK_METHOD_HCM_LSM = 3
EIK_SCHED_AUTO = 0
EIK_SCHED_ROUNDS = 1
EIK_SCHED_FIFO = 2
EIK_SCHED_ORDERED = 3
EIK_NOALLOC_SCRATCH_BYTES = 32 << 20
EIK_NOALLOC_MAX_SOURCES = 256


class eik_plan_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("h", ctypes.c_double),
                ("cell_k", ctypes.c_int32), ("bucket_width", ctypes.c_double),
                ("precision", ctypes.c_int32), ("tol", ctypes.c_double),
                ("deadline_ns", ctypes.c_int64), ("method", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("window", ctypes.c_int32)]


class eik_instance(ctypes.Structure):
    _fields_ = [("F", ctypes.c_void_p), ("src_ij", ctypes.c_void_p), ("src_q", ctypes.c_void_p),
                ("nsrc", ctypes.c_int32), ("U", ctypes.c_void_p)]


class eik_stats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("mpts_per_s", ctypes.c_double),
                ("updates_per_pt", ctypes.c_double), ("avhr", ctypes.c_double),
                ("avs", ctypes.c_double), ("max_residual", ctypes.c_double),
                ("err_bound", ctypes.c_double), ("bucket_width", ctypes.c_double),
                ("cell_visits", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("buckets", ctypes.c_int64), ("pass_ms", ctypes.c_double * 2),
                ("launches", ctypes.c_int32), ("cell_k", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("status", ctypes.c_int32),
                ("mono_pct", ctypes.c_double), ("queue_left", ctypes.c_int64)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["pass_ms"] = list(self.pass_ms)
        return d


class eik_tune_result(ctypes.Structure):
    _fields_ = [("cell_k", ctypes.c_int32), ("bucket_first", ctypes.c_double),
                ("bucket_main", ctypes.c_double), ("async_first", ctypes.c_int32),
                ("async_main", ctypes.c_int32), ("one_pass", ctypes.c_int32),
                ("hold_ns", ctypes.c_int32), ("ms", ctypes.c_double),
                ("ms_before", ctypes.c_double), ("trials", ctypes.c_int32),
                ("ordered", ctypes.c_int32), ("window", ctypes.c_int32)]


eik_plan = ctypes.c_void_p
eik_server = ctypes.c_void_p
eik_batch = ctypes.c_void_p
_P = ctypes.POINTER

_lib.eik_strerror.argtypes = [ctypes.c_int]
_lib.eik_strerror.restype = ctypes.c_char_p
_lib.eik_plan_create.argtypes = [_P(eik_plan), _P(eik_plan_desc), ctypes.c_void_p]
_lib.eik_plan_create.restype = ctypes.c_int
_lib.eik_plan_destroy.argtypes = [eik_plan]
_lib.eik_plan_destroy.restype = None
_lib.eik_plan_workspace_bytes.argtypes = [_P(eik_plan_desc)]
_lib.eik_plan_workspace_bytes.restype = ctypes.c_size_t
_lib.eik_solve.argtypes = [eik_plan, _P(eik_instance), _P(eik_stats)]
_lib.eik_solve.restype = ctypes.c_int
_lib.eik_solve_noalloc.argtypes = [_P(eik_plan_desc), _P(eik_instance), _P(eik_stats),
                                   ctypes.c_void_p]
_lib.eik_solve_noalloc.restype = ctypes.c_int
_lib.eik_solve_batch.argtypes = [_P(eik_plan_desc), _P(eik_instance), ctypes.c_int32,
                                 _P(eik_stats), ctypes.c_void_p]
_lib.eik_solve_batch.restype = ctypes.c_int
_lib.eik_batch_create.argtypes = [_P(eik_batch), _P(eik_plan_desc), _P(eik_instance), ctypes.c_int32,
                                  ctypes.c_void_p]
_lib.eik_batch_create.restype = ctypes.c_int
_lib.eik_batch_run.argtypes = [eik_batch, _P(eik_stats)]
_lib.eik_batch_run.restype = ctypes.c_int
_lib.eik_batch_destroy.argtypes = [eik_batch]
_lib.eik_batch_destroy.restype = None
_lib.eik_tune.argtypes = [_P(eik_plan_desc), _P(eik_instance), ctypes.c_int32, ctypes.c_void_p,
                          _P(eik_tune_result)]
_lib.eik_tune.restype = ctypes.c_int
_lib.eik_tune_save.argtypes = [ctypes.c_char_p]
_lib.eik_tune_save.restype = ctypes.c_int
_lib.eik_tune_load.argtypes = [ctypes.c_char_p]
_lib.eik_tune_load.restype = ctypes.c_int
_lib.eik_tune_reset.argtypes = []
_lib.eik_tune_reset.restype = None
_lib.eik_server_create.argtypes = [_P(eik_server), ctypes.c_size_t, ctypes.c_int32,
                                   ctypes.c_void_p]
_lib.eik_server_create.restype = ctypes.c_int
_lib.eik_submit.argtypes = [eik_server, _P(eik_plan_desc), _P(eik_instance), _P(ctypes.c_uint64)]
_lib.eik_submit.restype = ctypes.c_int
_lib.eik_poll.argtypes = [eik_server, ctypes.c_uint64, _P(eik_stats)]
_lib.eik_poll.restype = ctypes.c_int
_lib.eik_server_destroy.argtypes = [eik_server]
_lib.eik_server_destroy.restype = None

SYMBOLS = ["eik_strerror", "eik_plan_create", "eik_plan_destroy", "eik_plan_workspace_bytes",
           "eik_solve", "eik_solve_noalloc", "eik_solve_batch", "eik_batch_create", "eik_batch_run",
           "eik_batch_destroy", "eik_tune", "eik_tune_save",
           "eik_tune_load", "eik_tune_reset", "eik_server_create", "eik_submit", "eik_poll",
           "eik_server_destroy"]


class EikError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {eik_strerror(code)} ({code})" if what else eik_strerror(code))


# ------------------------------------------------------------------ C names
def eik_strerror(code: int) -> str:
    return _lib.eik_strerror(int(code)).decode()


def eik_plan_create(desc: eik_plan_desc, cuda_stream=None) -> eik_plan:
    p = eik_plan()
    rc = _lib.eik_plan_create(ctypes.byref(p), ctypes.byref(desc), _stream_ptr(cuda_stream))
    if rc:
        raise EikError(rc, "eik_plan_create")
    return p


def eik_plan_destroy(plan: eik_plan) -> None:
    _lib.eik_plan_destroy(plan)


def eik_plan_workspace_bytes(desc: eik_plan_desc) -> int:
    return int(_lib.eik_plan_workspace_bytes(ctypes.byref(desc)))


def eik_solve(plan: eik_plan, inst: eik_instance) -> tuple[int, eik_stats]:
    st = eik_stats()
    rc = _lib.eik_solve(plan, ctypes.byref(inst), ctypes.byref(st))
    return rc, st


def eik_solve_noalloc(desc: eik_plan_desc, inst: eik_instance, cuda_stream=None):
    """FP64 solve that allocates nothing (fixed in-library device scratch);
    F and U must be device tensors.  Returns (status, eik_stats)."""
    st = eik_stats()
    rc = _lib.eik_solve_noalloc(ctypes.byref(desc), ctypes.byref(inst), ctypes.byref(st),
                                _stream_ptr(cuda_stream))
    return rc, st


def eik_solve_batch(descs, insts, cuda_stream=None):
    n = len(descs)
    D = (eik_plan_desc * n)(*descs)
    I = (eik_instance * n)(*insts)
    S = (eik_stats * n)()
    rc = _lib.eik_solve_batch(D, I, n, S, _stream_ptr(cuda_stream))
    return rc, list(S)


def eik_batch_create(descs, insts, cuda_stream=None) -> eik_batch:
    n = len(descs)
    D = (eik_plan_desc * n)(*descs)
    I = (eik_instance * n)(*insts)
    b = eik_batch()
    rc = _lib.eik_batch_create(ctypes.byref(b), D, I, n, _stream_ptr(cuda_stream))
    if rc:
        raise EikError(rc, "eik_batch_create")
    b.n_inst = n
    return b


def eik_batch_run(batch: eik_batch, n_inst: int = None):
    n = n_inst if n_inst is not None else batch.n_inst
    S = (eik_stats * n)()
    rc = _lib.eik_batch_run(batch, S)
    return rc, list(S)


def eik_batch_destroy(batch: eik_batch) -> None:
    _lib.eik_batch_destroy(batch)


def eik_tune(descs, insts, cuda_stream=None):
    n = len(descs)
    D = (eik_plan_desc * n)(*descs)
    I = (eik_instance * n)(*insts)
    r = eik_tune_result()
    rc = _lib.eik_tune(D, I, n, _stream_ptr(cuda_stream), ctypes.byref(r))
    return rc, r


def eik_tune_save(path) -> int:
    return _lib.eik_tune_save(os.fsencode(path))


def eik_tune_load(path) -> int:
    return _lib.eik_tune_load(os.fsencode(path))


def eik_tune_reset() -> None:
    _lib.eik_tune_reset()


def eik_server_create(hbm_budget_bytes: int, max_inflight: int = 0, cuda_stream=None) -> eik_server:
    s = eik_server()
    rc = _lib.eik_server_create(ctypes.byref(s), int(hbm_budget_bytes), int(max_inflight),
                                _stream_ptr(cuda_stream))
    if rc:
        raise EikError(rc, "eik_server_create")
    return s


def eik_submit(server: eik_server, desc: eik_plan_desc, inst: eik_instance) -> tuple[int, int]:
    t = ctypes.c_uint64(0)
    rc = _lib.eik_submit(server, ctypes.byref(desc), ctypes.byref(inst), ctypes.byref(t))
    return rc, t.value


def eik_poll(server: eik_server, ticket: int) -> tuple[int, eik_stats]:
    st = eik_stats()
    rc = _lib.eik_poll(server, ctypes.c_uint64(ticket), ctypes.byref(st))
    return rc, st


def eik_server_destroy(server: eik_server) -> None:
    _lib.eik_server_destroy(server)


# ------------------------------------------------------------------ marshalling
def _stream_ptr(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(int(s.cuda_stream))  # torch.cuda.Stream


def _ptr(a, dtype):
    """Data pointer of a C-contiguous NumPy array or torch tensor of `dtype`."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return ctypes.c_void_p(a.data_ptr()) if a.numel() else None
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"array must be a C-contiguous {np.dtype(dtype)} ndarray")
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def make_desc(nx, ny, h, cell_k=8, precision=EIK_FP64, bucket_width=0.0, tol=0.0,
              deadline_ns=0, method=0, schedule=EIK_SCHED_AUTO, window=0) -> eik_plan_desc:
    return eik_plan_desc(int(nx), int(ny), float(h), int(cell_k), float(bucket_width),
                         int(precision), float(tol), int(deadline_ns), int(method), int(schedule),
                         int(window))


def make_instance(F, src_ij, src_q, U) -> eik_instance:
    n = int(src_q.shape[0])
    return eik_instance(_ptr(F, np.float64), _ptr(src_ij, np.int32), _ptr(src_q, np.float64), n,
                        _ptr(U, np.float64))


class Plan:
    """Owns an ``eik_plan`` for one grid shape."""

    def __init__(self, nx, ny, h, cell_k=8, precision=EIK_FP64, bucket_width=0.0, tol=0.0,
                 deadline_ns=0, stream=None, method=EIK_METHOD_HCM, schedule=EIK_SCHED_AUTO, window=0):
        self.desc = make_desc(nx, ny, h, cell_k, precision, bucket_width, tol, deadline_ns, method,
                              schedule, window)
        self.handle = eik_plan_create(self.desc, stream)

    def solve(self, F, src_ij, src_q, U):
        """Solve into U (same kind of memory as the caller chose); returns
        (status, eik_stats).  Keeps every array alive for the call."""
        inst = make_instance(F, src_ij, src_q, U)
        return eik_solve(self.handle, inst)

    def close(self):
        if self.handle:
            eik_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(F, h, si, sj, sq, cell_k=8, precision=EIK_FP64, bucket_width=0.0, tol=0.0,
          deadline_ns=0, method=EIK_METHOD_HCM, schedule=EIK_SCHED_AUTO, window=0):
    """Convenience: host arrays in, host U out, (U, stats); raises on error."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    ny, nx = F.shape
    src_ij = np.ascontiguousarray(np.stack([np.atleast_1d(si), np.atleast_1d(sj)], axis=1)
                                  .reshape(-1), dtype=np.int32)
    sq = np.ascontiguousarray(np.atleast_1d(sq), dtype=np.float64)
    U = np.empty((ny, nx), dtype=np.float64)
    with Plan(nx, ny, h, cell_k, precision, bucket_width, tol, deadline_ns, method=method,
              schedule=schedule, window=window) as p:
        rc, st = p.solve(F, src_ij, sq, U)
    if rc:
        raise EikError(rc, "eik_solve")
    return U, st
