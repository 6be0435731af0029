"""Python binding of the GB300 ASRAL library (liblbdd.so, C ABI in include/lbdd.h).

Argument marshalling only: every step of the solver runs in the CUDA kernels
of ``csrc/``.  There is no CPU fallback -- if the library cannot be built or
loaded, or no compute-capability-10.3 GPU is present, calls raise.

Names follow the C ABI (``lbdd_create`` -> :func:`create`, ...).  Device
buffers may be passed as ``torch.Tensor`` (CUDA) or raw integer pointers;
host buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = [
    "load", "LbddError", "Solver", "create", "create_strict", "set_penalty_table", "road_cm", "solve", "reset", "insert", "solve_batch", "objective",
    "assignment", "loads", "rounds_done", "get_stats", "best_transfer_table",
    "best_transfer", "best_transfer_workspace", "cm_pitch", "strerror", "destroy",
    "Batch", "autotune", "tune_get", "tune_clear", "Server", "RequestInfo", "ServerStats",
]

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_INVARIANT, ERR_STATE, ERR_NODEV, ERR_BUDGET = \
    -1, -2, -3, -4, -5, -6, -7, -8
CM_I32, CM_I16 = 0, 1
OPT_CLUSTER, OPT_NCYC_SKIP, OPT_NPATH_REUSE, OPT_TC_SMEM, OPT_PHASE_TIMERS = 1, 2, 3, 4, 5
TINF = 2**31 - 1

_lib = None


class LbddError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {strerror(code)} ({code})"
        if code == ERR_CUDA and _lib is not None:
            msg += f" [{_lib.lbdd_last_cuda_error().decode()}]"
        super().__init__(msg)


_STAT_FIELDS = (
    "rounds", "cycles_applied", "paths_applied", "bf_calls", "bf_sweeps", "bf_max_sweeps",
    "moves", "ncyc_skipped", "rows_scanned", "cm_elem_bytes", "cluster_size",
    "prologue_ns", "rounds_ns", "merge_ns", "relax_ns", "sync_ns", "gather_ns", "apply_ns",
    "rescan_ns", "relax_loop_ns", "relax_reduce_ns", "cost_slice_in_smem", "npath_reused",
    "col_rows", "front_sum")


class _Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in _STAT_FIELDS] + [("front_hist", ctypes.c_int64 * 6)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("quantum_us", ctypes.c_int64), ("cluster_size", ctypes.c_int)]


class _RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("objective", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("submit_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64)]


_SERVER_STAT_FIELDS = ("passes", "admitted", "completed", "failed", "queued", "bytes_in_use",
                       "peak_bytes", "busy_ns", "uptime_ns", "peak_active", "launches")


class _ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in _SERVER_STAT_FIELDS]


def load():
    """Build (if stale) and load liblbdd.so; raises on any failure."""
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P, i32, i64, c_int, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int,
                                  ctypes.c_size_t)
        lib.lbdd_create.argtypes = [ctypes.POINTER(P), i32, i32, P, c_int, c_int, P, P, P]
        lib.lbdd_set_option.argtypes = [P, c_int, i64]
        lib.lbdd_create_strict.argtypes = [ctypes.POINTER(P), i32, i32, P, c_int, c_int, P, P]
        lib.lbdd_set_penalty_table.argtypes = [P, P, i32]
        lib.lbdd_road_cm.argtypes = [i32, P, P, P, i32, P, i32, P, P, i64, P]
        lib.lbdd_solve.argtypes = [P, i64]
        lib.lbdd_reset.argtypes = [P]
        lib.lbdd_insert.argtypes = [P, P, c_int, ctypes.POINTER(i32)]
        lib.lbdd_solve_batch.argtypes = [ctypes.POINTER(P), c_int, i64, c_int, c_int, P]
        lib.lbdd_objective.argtypes = [P, ctypes.POINTER(i64)]
        lib.lbdd_assignment.argtypes = [P, P, c_int]
        lib.lbdd_loads.argtypes = [P, P]
        lib.lbdd_rounds_done.argtypes = [P, ctypes.POINTER(i64)]
        lib.lbdd_get_stats.argtypes = [P, ctypes.POINTER(_Stats)]
        lib.lbdd_best_transfer_table.argtypes = [P, P, P, c_int]
        lib.lbdd_destroy.argtypes = [P]
        lib.lbdd_destroy.restype = None
        lib.lbdd_strerror.argtypes = [c_int]
        lib.lbdd_strerror.restype = ctypes.c_char_p
        lib.lbdd_last_cuda_error.argtypes = []
        lib.lbdd_last_cuda_error.restype = ctypes.c_char_p
        lib.lbdd_best_transfer_workspace.argtypes = [i32, i32]
        lib.lbdd_best_transfer_workspace.restype = sz
        lib.lbdd_best_transfer.argtypes = [i32, i32, P, c_int, i64, P, P, P, P, sz, P]
        lib.lbdd_cm_pitch.argtypes = [i32, c_int]
        lib.lbdd_max_centers.argtypes = []
        lib.lbdd_max_centers.restype = i32
        lib.lbdd_cm_pitch.restype = i64
        lib.lbdd_solver_cm.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(c_int),
                                       ctypes.POINTER(i64)]
        PI32 = ctypes.POINTER(i32)
        lib.lbdd_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), c_int, c_int,
                                          c_int, P]
        lib.lbdd_batch_run.argtypes = [P, i64]
        lib.lbdd_batch_plan.argtypes = [P, PI32, PI32, PI32, PI32, PI32, c_int]
        lib.lbdd_batch_destroy.argtypes = [P]
        lib.lbdd_batch_destroy.restype = None
        lib.lbdd_autotune.argtypes = [ctypes.POINTER(P), c_int, c_int, P]
        lib.lbdd_tune_get.argtypes = [c_int, i32, c_int, ctypes.POINTER(ctypes.c_double)]
        lib.lbdd_tune_clear.argtypes = []
        lib.lbdd_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_ServerConfig)]
        lib.lbdd_server_submit.argtypes = [P, i32, i32, P, c_int, P, P, P, ctypes.POINTER(i64)]
        lib.lbdd_server_submit_ex.argtypes = [P, i32, i32, P, c_int, c_int, P, P, P,
                                              ctypes.POINTER(i64)]
        lib.lbdd_server_poll.argtypes = [P, i64, i64, ctypes.POINTER(_RequestInfo)]
        lib.lbdd_server_release.argtypes = [P, i64]
        lib.lbdd_server_get_stats.argtypes = [P, ctypes.POINTER(_ServerStats)]
        lib.lbdd_server_destroy.argtypes = [P]
        lib.lbdd_server_destroy.restype = None
        _lib = lib
    return _lib


def strerror(code: int) -> str:
    return load().lbdd_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise LbddError(rc, what)


def _dptr(x) -> int:
    """Device pointer of a CUDA tensor or an int."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("expected a contiguous CUDA tensor")
        return x.data_ptr()
    raise TypeError(type(x))


def _host_vec(a, length: int, what: str) -> np.ndarray:
    """Contiguous int32 host copy of a length-`length` vector (the C side reads
    exactly that many entries)."""
    v = np.ascontiguousarray(a, dtype=np.int32)
    if v.shape != (length,):
        raise ValueError(f"{what}: expected {length} entries, got shape {v.shape}")
    return v


def _numel(x) -> int:
    return int(x.numel()) if hasattr(x, "numel") else int(np.asarray(x).size)


def _need(x, count: int, what: str):
    """A device tensor argument holds at least `count` elements (raw ints are
    taken as they are)."""
    if not isinstance(x, int) and _numel(x) < count:
        raise ValueError(f"{what}: needs at least {count} elements, has {_numel(x)}")


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class Stats:
    rounds: int
    cycles_applied: int
    paths_applied: int
    bf_calls: int
    bf_sweeps: int
    bf_max_sweeps: int
    moves: int
    ncyc_skipped: int
    rows_scanned: int
    cm_elem_bytes: int
    cluster_size: int
    prologue_ns: int
    rounds_ns: int
    merge_ns: int
    relax_ns: int
    sync_ns: int
    gather_ns: int
    apply_ns: int
    rescan_ns: int
    relax_loop_ns: int
    relax_reduce_ns: int
    cost_slice_in_smem: int
    npath_reused: int
    col_rows: int
    front_sum: int
    front_hist: tuple


def create(n, k, cm, cap, pen, stream=None, cm_dtype=None):
    """lbdd_create.  cm: numpy (n, k) int32/int16 (host) or a CUDA tensor."""
    lib = load()
    cap = _host_vec(cap, int(k), "cap")
    pen = _host_vec(pen, int(k), "pen")
    if isinstance(cm, np.ndarray):
        cm = np.ascontiguousarray(cm)
        if cm.size != int(n) * int(k):
            raise ValueError(f"cm: expected {n} x {k} entries, got shape {cm.shape}")
        dt = {np.dtype(np.int32): CM_I32, np.dtype(np.int16): CM_I16}[cm.dtype]
        ptr, is_dev = cm.ctypes.data, 0
    else:
        import torch
        dt = {torch.int32: CM_I32, torch.int16: CM_I16}[cm.dtype] if cm_dtype is None else cm_dtype
        _need(cm, int(n) * int(k), "cm")
        ptr, is_dev = _dptr(cm), 1
    h = ctypes.c_void_p()
    _check(lib.lbdd_create(ctypes.byref(h), int(n), int(k), ptr, dt, is_dev, cap.ctypes.data,
                           pen.ctypes.data, _stream_handle(stream)), "lbdd_create")
    return h


def create_strict(n, k, cm, cap, stream=None):
    """lbdd_create_strict (Alg. 5).  cm: numpy (n, k) int32/int16 (host)."""
    lib = load()
    cap = _host_vec(cap, int(k), "cap")
    cm = np.ascontiguousarray(cm)
    if cm.size != int(n) * int(k):
        raise ValueError(f"cm: expected {n} x {k} entries, got shape {cm.shape}")
    dt = {np.dtype(np.int32): CM_I32, np.dtype(np.int16): CM_I16}[cm.dtype]
    h = ctypes.c_void_p()
    _check(lib.lbdd_create_strict(ctypes.byref(h), int(n), int(k), cm.ctypes.data, dt, 0,
                                  cap.ctypes.data, _stream_handle(stream)), "lbdd_create_strict")
    return h


def road_cm(row_ptr, col, w, centers, demand, out, ld=None, stream=None):
    """lbdd_road_cm on device tensors (int32); out: device int32 (n, ld)."""
    n, k = len(demand), len(centers)
    ld = int(ld if ld is not None else k)
    if len(col) != len(w):
        raise ValueError("col and w must have one entry per road")
    _need(out, n * ld, "out")
    _check(load().lbdd_road_cm(int(len(row_ptr) - 1), _dptr(row_ptr), _dptr(col), _dptr(w),
                               int(k), _dptr(centers), int(n), _dptr(demand), _dptr(out),
                               ld, _stream_handle(stream)),
           "lbdd_road_cm")
    return out


def set_penalty_table(h, qtab, k: int = None):
    """lbdd_set_penalty_table: qtab (k, Q) int32, q_s(j) = qtab[s, min(j, Q) - 1]."""
    q = np.ascontiguousarray(qtab, dtype=np.int32)
    if q.ndim != 2 or q.shape[1] < 1 or (k is not None and q.shape[0] != k):
        raise ValueError(f"qtab: expected a (k, Q) table, got shape {q.shape}")
    _check(load().lbdd_set_penalty_table(h, q.ctypes.data, int(q.shape[1])),
           "lbdd_set_penalty_table")


def set_option(h, option: int, value: int):
    _check(load().lbdd_set_option(h, option, value), "lbdd_set_option")


def solve(h, max_rounds: int = -1):
    _check(load().lbdd_solve(h, int(max_rounds)), "lbdd_solve")


def reset(h):
    _check(load().lbdd_reset(h), "lbdd_reset")


def insert(h, row, k: int) -> int:
    """lbdd_insert: one more demand unit with costs `row` (k entries, int32 or
    int16); returns its index."""
    r = np.ascontiguousarray(row)
    if r.dtype not in (np.int32, np.int16):
        r = r.astype(np.int32)
    if r.shape != (int(k),):
        raise ValueError(f"row: expected {k} entries, got shape {r.shape}")
    dt = CM_I16 if r.dtype == np.int16 else CM_I32
    u = ctypes.c_int32()
    _check(load().lbdd_insert(h, r.ctypes.data, dt, ctypes.byref(u)), "lbdd_insert")
    return u.value


def solve_batch(handles, max_rounds: int = -1, cluster_size: int = 0, max_clusters: int = 0,
                stream=None):
    arr = _handles(handles)
    _check(load().lbdd_solve_batch(arr, len(handles), int(max_rounds), cluster_size, max_clusters,
                                   _stream_handle(stream)), "lbdd_solve_batch")


def objective(h) -> int:
    v = ctypes.c_int64()
    _check(load().lbdd_objective(h, ctypes.byref(v)), "lbdd_objective")
    return v.value


def rounds_done(h) -> int:
    v = ctypes.c_int64()
    _check(load().lbdd_rounds_done(h, ctypes.byref(v)), "lbdd_rounds_done")
    return v.value


def assignment(h, n: int, out=None):
    """Host numpy copy (default) or into a CUDA int32 tensor `out`."""
    if out is None:
        a = np.empty(n, np.int32)
        _check(load().lbdd_assignment(h, a.ctypes.data, 0), "lbdd_assignment")
        return a
    _need(out, n, "out")
    _check(load().lbdd_assignment(h, _dptr(out), 1), "lbdd_assignment")
    return out


def loads(h, k: int):
    a = np.empty(k, np.int32)
    _check(load().lbdd_loads(h, a.ctypes.data), "lbdd_loads")
    return a


def get_stats(h) -> Stats:
    s = _Stats()
    _check(load().lbdd_get_stats(h, ctypes.byref(s)), "lbdd_get_stats")
    d = {f: getattr(s, f) for f in _STAT_FIELDS}
    d["front_hist"] = tuple(s.front_hist)
    return Stats(**d)


def best_transfer_table(h, k: int):
    tc = np.empty((k, k), np.int32)
    td = np.empty((k, k), np.int32)
    _check(load().lbdd_best_transfer_table(h, tc.ctypes.data, td.ctypes.data, 0),
           "lbdd_best_transfer_table")
    return tc, td


def solver_cm(h):
    p, dt, ld = ctypes.c_void_p(), ctypes.c_int(), ctypes.c_int64()
    _check(load().lbdd_solver_cm(h, ctypes.byref(p), ctypes.byref(dt), ctypes.byref(ld)),
           "lbdd_solver_cm")
    return p.value, dt.value, ld.value


def cm_pitch(k: int, cm_dtype: int) -> int:
    return int(load().lbdd_cm_pitch(k, cm_dtype))


def max_centers() -> int:
    """lbdd_max_centers: the largest k a solver accepts."""
    return int(load().lbdd_max_centers())


def best_transfer_workspace(n: int, k: int) -> int:
    return int(load().lbdd_best_transfer_workspace(n, k))


def best_transfer(n, k, cm_dev, cm_dtype, ld, assign_dev, tc_dev, td_dev, workspace,
                  workspace_bytes, stream=None):
    """lbdd_best_transfer (asynchronous on `stream`)."""
    _need(cm_dev, int(n) * int(ld), "cm")
    _need(assign_dev, int(n), "assign")
    _need(tc_dev, int(k) * int(k), "tc")
    _need(td_dev, int(k) * int(k), "td")
    if not isinstance(workspace, int) and \
            _numel(workspace) * workspace.element_size() < int(workspace_bytes):
        raise ValueError(f"workspace: smaller than workspace_bytes = {workspace_bytes}")
    _check(load().lbdd_best_transfer(int(n), int(k), _dptr(cm_dev), int(cm_dtype), int(ld),
                                     _dptr(assign_dev), _dptr(tc_dev), _dptr(td_dev),
                                     _dptr(workspace), int(workspace_bytes),
                                     _stream_handle(stream)), "lbdd_best_transfer")


def destroy(h):
    if h is not None and (not hasattr(h, "value") or h.value):
        load().lbdd_destroy(h)


class Solver:
    """RAII wrapper around one lbdd_solver handle (strict=True: Alg. 5, no
    penalties; the instance gains a dummy center when capacity is short)."""

    def __init__(self, cm, cap, pen, stream=None, cluster: int = 0, ncyc_skip: bool = True,
                 npath_reuse: bool = True, phase_timers: bool = False, strict: bool = False,
                 qtab=None, tc_smem: bool = True):
        if isinstance(cm, np.ndarray):
            n, k = cm.shape
        else:
            n, k = int(cm.shape[0]), int(cm.shape[1])
        self.n, self.k = int(n), int(k)
        if strict:
            self.h = create_strict(self.n, self.k, cm, cap, stream=stream)
            if int(np.sum(np.asarray(cap, dtype=np.int64))) < self.n:
                self.k += 1
        else:
            self.h = create(self.n, self.k, cm, cap, pen, stream=stream)
        if cluster:
            set_option(self.h, OPT_CLUSTER, cluster)
        if not ncyc_skip:
            set_option(self.h, OPT_NCYC_SKIP, 0)
        if not npath_reuse:
            set_option(self.h, OPT_NPATH_REUSE, 0)
        if phase_timers:
            set_option(self.h, OPT_PHASE_TIMERS, 1)
        if not tc_smem:
            set_option(self.h, OPT_TC_SMEM, 0)
        if qtab is not None:
            set_penalty_table(self.h, qtab, self.k)

    def solve(self, max_rounds: int = -1):
        solve(self.h, max_rounds)
        return self

    def reset(self):
        reset(self.h)
        return self

    def insert(self, row) -> int:
        """Append one demand unit (lbdd_insert); returns its index."""
        u = insert(self.h, row, self.k)
        self.n += 1
        return u

    @property
    def objective(self) -> int:
        return objective(self.h)

    @property
    def rounds(self) -> int:
        return rounds_done(self.h)

    def assignment(self, out=None):
        return assignment(self.h, self.n, out)

    def loads(self):
        return loads(self.h, self.k)

    def stats(self) -> Stats:
        return get_stats(self.h)

    def table(self):
        return best_transfer_table(self.h, self.k)

    def close(self):
        if self.h is not None:
            destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _handles(handles):
    return (ctypes.c_void_p * len(handles))(
        *[h.h.value if isinstance(h, Solver) else (h.value if hasattr(h, "value") else h)
          for h in handles])


class Batch:
    """lbdd_batch: a planned, graph-captured batch of solvers (Solver objects
    or handles, which must outlive the batch)."""

    def __init__(self, solvers, cluster_size: int = 0, max_clusters: int = 0, stream=None):
        self.m = len(solvers)
        self._keep = list(solvers)
        h = ctypes.c_void_p()
        _check(load().lbdd_batch_create(ctypes.byref(h), _handles(solvers), self.m, cluster_size,
                                        max_clusters, _stream_handle(stream)),
               "lbdd_batch_create")
        self.h = h

    def run(self, max_rounds: int = -1):
        _check(load().lbdd_batch_run(self.h, int(max_rounds)), "lbdd_batch_run")

    def plan(self):
        """(cluster size per instance, [(cluster size, clusters, instances) per group])."""
        m = self.m
        cl = (ctypes.c_int32 * m)()
        ng = ctypes.c_int32()
        gc, gn, gs = (ctypes.c_int32 * 16)(), (ctypes.c_int32 * 16)(), (ctypes.c_int32 * 16)()
        _check(load().lbdd_batch_plan(self.h, cl, ctypes.byref(ng), gc, gn, gs, 16),
               "lbdd_batch_plan")
        return list(cl), [(gc[g], gn[g], gs[g]) for g in range(ng.value)]

    def close(self):
        if self.h is not None:
            load().lbdd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(solvers, probe_rounds: int = 4096, stream=None):
    _check(load().lbdd_autotune(_handles(solvers), len(solvers), int(probe_rounds),
                                _stream_handle(stream)), "lbdd_autotune")


def tune_get(cm_dtype: int, k: int, cluster_size: int) -> float:
    v = ctypes.c_double()
    _check(load().lbdd_tune_get(cm_dtype, int(k), int(cluster_size), ctypes.byref(v)),
           "lbdd_tune_get")
    return v.value


def tune_clear():
    _check(load().lbdd_tune_clear(), "lbdd_tune_clear")


REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


@dataclass
class RequestInfo:
    state: int
    status: int
    objective: int
    rounds: int
    submit_ns: int
    admit_ns: int
    done_ns: int


@dataclass
class ServerStats:
    passes: int
    admitted: int
    completed: int
    failed: int
    queued: int
    bytes_in_use: int
    peak_bytes: int
    busy_ns: int
    uptime_ns: int
    peak_active: int
    launches: int


class Server:
    """lbdd_server: continuous-batching request server on the current device.

    submit() keeps references to the request's host arrays until the request
    is released (``result``/``release``)."""

    def __init__(self, budget_bytes: int, max_active: int = 0, quantum_us: int = 0,
                 cluster_size: int = 0):
        cfg = _ServerConfig(int(budget_bytes), int(max_active), int(quantum_us), int(cluster_size))
        h = ctypes.c_void_p()
        _check(load().lbdd_server_create(ctypes.byref(h), ctypes.byref(cfg)), "lbdd_server_create")
        self.h = h
        self._bufs = {}

    def submit(self, cm, cap, pen) -> int:
        """Queue a request; cm is a host (n, k) array (lbdd_server_submit) or
        a contiguous CUDA tensor whose values are ready (lbdd_server_submit_ex
        with a device CM).  The binding keeps cm alive until the result is
        taken."""
        if isinstance(cm, np.ndarray):
            cm = np.ascontiguousarray(cm)
            dt = {np.dtype(np.int32): CM_I32, np.dtype(np.int16): CM_I16}[cm.dtype]
            ptr, is_dev = cm.ctypes.data, 0
        else:
            import torch
            dt = {torch.int32: CM_I32, torch.int16: CM_I16}[cm.dtype]
            ptr, is_dev = _dptr(cm), 1
        if cm.ndim != 2:
            raise ValueError(f"cm: expected an (n, k) matrix, got shape {tuple(cm.shape)}")
        n, k = (int(x) for x in cm.shape)
        cap = _host_vec(cap, k, "cap")
        pen = _host_vec(pen, k, "pen")
        out = np.empty(n, np.int32)
        t = ctypes.c_int64()
        _check(load().lbdd_server_submit_ex(self.h, n, k, ptr, dt, is_dev, cap.ctypes.data,
                                            pen.ctypes.data, out.ctypes.data, ctypes.byref(t)),
               "lbdd_server_submit_ex")
        self._bufs[t.value] = (cm, out)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """RequestInfo, or None if the request has not ended within timeout_ms."""
        info = _RequestInfo()
        rc = load().lbdd_server_poll(self.h, int(ticket), int(timeout_ms), ctypes.byref(info))
        if rc == ERR_TIMEOUT:
            return None
        _check(rc, "lbdd_server_poll")
        return RequestInfo(*[getattr(info, f) for f, _ in _RequestInfo._fields_])

    def result(self, ticket: int, timeout_ms: int = -1):
        """(RequestInfo, allotment) once the request ended; releases it."""
        info = self.poll(ticket, timeout_ms)
        if info is None:
            return None
        _, out = self._bufs.pop(ticket)
        _check(load().lbdd_server_release(self.h, int(ticket)), "lbdd_server_release")
        return info, out

    def stats(self) -> ServerStats:
        s = _ServerStats()
        _check(load().lbdd_server_get_stats(self.h, ctypes.byref(s)), "lbdd_server_get_stats")
        return ServerStats(*[getattr(s, f) for f in _SERVER_STAT_FIELDS])

    def close(self):
        if self.h is not None:
            load().lbdd_server_destroy(self.h)
            self.h = None
            self._bufs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
