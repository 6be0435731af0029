"""CPU oracle for ASRAL -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the C-ABI library
and its Python binding) never imports, links or executes anything here.

The arithmetic lives in ``asral_oracle.c`` (plain single-threaded C, built to
``_oracle.so`` by :func:`build`); this module only marshals numpy arrays.
Exact reference solvers used to pin the oracle live in :mod:`oracle.exact`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None

OK, ERR_ARG, ERR_OOM, ERR_INVARIANT = 0, -1, -2, -5
INF = 1 << 62
MODE_DEFINITION, MODE_HEAP = 0, 1


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "asral_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", src, "-o", _SO + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


class _Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "rounds", "cycles_applied", "paths_applied", "bf_calls", "bf_sweeps",
        "bf_max_sweeps", "moves")]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_objective.argtypes = [i64, i64, P, P, P, P]
        lib.oracle_objective.restype = i64
        lib.oracle_smin_order.argtypes = [i64, i64, P, P, P]
        lib.oracle_best_transfer.argtypes = [i64, i64, P, P, P, P]
        lib.oracle_bf.argtypes = [i64, i64, P, P, P, P]
        lib.oracle_has_negative_cycle.argtypes = [i64, P]
        lib.oracle_asral.argtypes = [i64, i64, P, P, P, c_int, i64, c_int, P, P, P, P]
        lib.oracle_asral_q.argtypes = [i64, i64, P, P, P, i64, c_int, i64, c_int, P, P, P, P]
        lib.oracle_asral_order.argtypes = [i64, i64, P, P, P, i64, c_int, i64, c_int, P, P, P, P,
                                           P]
        lib.oracle_road_cm.argtypes = [i64, P, P, P, i64, P, i64, P, P]
        lib.oracle_objective_q.argtypes = [i64, i64, P, P, P, i64, P]
        lib.oracle_objective_q.restype = i64
        lib.oracle_strict.argtypes = [i64, i64, P, P, P, P, P]
        _lib = lib
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _p(a):
    return a.ctypes.data


@dataclass
class Result:
    assign: np.ndarray      # (n,) int32, -1 = not allotted
    load: np.ndarray        # (k,) int64
    delta: int              # tracked objective (Eq. 1)
    stats: dict
    rc: int


def smin_order(cm):
    cm = _c(cm, np.int32)
    n, k = cm.shape
    smin = np.empty(n, np.int32)
    order = np.empty(n, np.int32)
    rc = _load().oracle_smin_order(n, k, _p(cm), _p(smin), _p(order))
    assert rc == OK, rc
    return smin, order


def best_transfer(cm, assign):
    """Best-transfer table by definition: (tc int64 with INF, td int32)."""
    cm = _c(cm, np.int32)
    n, k = cm.shape
    assign = _c(assign, np.int32)
    tc = np.empty((k, k), np.int64)
    td = np.empty((k, k), np.int32)
    rc = _load().oracle_best_transfer(n, k, _p(cm), _p(assign), _p(tc), _p(td))
    assert rc == OK, rc
    return tc, td


def bellman_ford(W, src):
    """Canonical synchronous Bellman-Ford on an (N, N) int64 matrix with INF
    for absent edges.  Returns (rc, dist, par, sweeps)."""
    W = _c(W, np.int64)
    N = W.shape[0]
    dist = np.empty(N, np.int64)
    par = np.empty(N, np.int32)
    sw = ctypes.c_int64(0)
    rc = _load().oracle_bf(N, src, _p(W), _p(dist), _p(par), ctypes.byref(sw))
    return rc, dist, par, sw.value


def has_negative_cycle(tc) -> bool:
    tc = _c(tc, np.int64)
    r = _load().oracle_has_negative_cycle(tc.shape[0], _p(tc))
    assert r in (0, 1)
    return bool(r)


def objective(cm, cap, pen, assign) -> int:
    cm = _c(cm, np.int32)
    n, k = cm.shape
    return int(_load().oracle_objective(n, k, _p(cm), _p(_c(cap, np.int32)),
                                         _p(_c(pen, np.int32)), _p(_c(assign, np.int32))))


def asral(cm, cap, pen, mode=MODE_HEAP, max_rounds=-1, check=False, order=None) -> Result:
    """Alg. 2 on the instance; see asral_oracle.c for the exact reading.
    order: the units' extraction order (default: the MinDistance order)."""
    cm = _c(cm, np.int32)
    n, k = cm.shape
    cap = _c(cap, np.int32)
    pen = _c(pen, np.int32)
    assign = np.empty(n, np.int32)
    load = np.empty(k, np.int64)
    delta = ctypes.c_int64(0)
    st = _Stats()
    if order is None:
        rc = _load().oracle_asral(n, k, _p(cm), _p(cap), _p(pen), int(mode), int(max_rounds),
                                  int(bool(check)), _p(assign), _p(load), ctypes.byref(delta),
                                  ctypes.byref(st))
    else:
        order = _c(order, np.int32)
        if order.shape != (n,):
            raise ValueError(f"order: expected {n} entries, got shape {order.shape}")
        rc = _load().oracle_asral_order(n, k, _p(cm), _p(cap), _p(pen), 1, int(mode),
                                        int(max_rounds), int(bool(check)), _p(order), _p(assign),
                                        _p(load), ctypes.byref(delta), ctypes.byref(st))
    stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
    return Result(assign=assign, load=load, delta=int(delta.value), stats=stats, rc=rc)


def insertion_order(cm, n0: int) -> np.ndarray:
    """Extraction order of a solve of the first n0 units (their MinDistance
    order) followed by the units n0..n-1 inserted afterwards, in index order
    (each insertion is one more iteration of Alg. 2)."""
    cm = _c(cm, np.int32)
    n = cm.shape[0]
    if not 1 <= n0 <= n:
        raise ValueError(f"n0 = {n0} outside [1, {n}]")
    _, order0 = smin_order(cm[:n0])
    return np.concatenate([order0, np.arange(n0, n, dtype=np.int32)])


def objective_q(cm, cap, qtab, assign) -> int:
    """Eq. (1) with penalty tables qtab (k x Q): q_s(j) = qtab[s, min(j, Q) - 1]."""
    cm = _c(cm, np.int32)
    n, k = cm.shape
    qtab = _c(qtab, np.int32)
    return int(_load().oracle_objective_q(n, k, _p(cm), _p(_c(cap, np.int32)), _p(qtab),
                                          qtab.shape[1], _p(_c(assign, np.int32))))


def asral_q(cm, cap, qtab, mode=MODE_HEAP, max_rounds=-1, check=False, order=None) -> Result:
    """Alg. 2 with general penalty functions (Def. 4) given as tables (k x Q).
    order: the units' extraction order (default: the MinDistance order)."""
    cm = _c(cm, np.int32)
    n, k = cm.shape
    cap = _c(cap, np.int32)
    qtab = _c(qtab, np.int32)
    assert qtab.ndim == 2 and qtab.shape[0] == k
    if order is not None:
        order = _c(order, np.int32)
        if order.shape != (n,):
            raise ValueError(f"order: expected {n} entries, got shape {order.shape}")
    assign = np.empty(n, np.int32)
    load = np.empty(k, np.int64)
    delta = ctypes.c_int64(0)
    st = _Stats()
    rc = _load().oracle_asral_order(n, k, _p(cm), _p(cap), _p(qtab), qtab.shape[1], int(mode),
                                    int(max_rounds), int(bool(check)),
                                    None if order is None else _p(order), _p(assign), _p(load),
                                    ctypes.byref(delta), ctypes.byref(st))
    stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
    return Result(assign=assign, load=load, delta=int(delta.value), stats=stats, rc=rc)


def road_cm(row_ptr, col, w, centers, demand):
    """CM from shortest paths on a road network (Section 3.4): (rc, CM n x k)."""
    row_ptr, col, w = _c(row_ptr, np.int32), _c(col, np.int32), _c(w, np.int32)
    centers, demand = _c(centers, np.int32), _c(demand, np.int32)
    V, k, n = len(row_ptr) - 1, len(centers), len(demand)
    cm = np.zeros((n, k), np.int32)
    rc = _load().oracle_road_cm(V, _p(row_ptr), _p(col), _p(w), k, _p(centers), n, _p(demand),
                                _p(cm))
    return rc, cm


def strict(cm, cap):
    """Appendix B (Alg. 5).  Returns (rc, assign over the extended centers,
    extended cost, stats)."""
    cm = _c(cm, np.int32)
    n, k = cm.shape
    cap = _c(cap, np.int32)
    assign = np.empty(n, np.int32)
    cost = ctypes.c_int64(0)
    st = _Stats()
    rc = _load().oracle_strict(n, k, _p(cm), _p(cap), _p(assign), ctypes.byref(cost),
                               ctypes.byref(st))
    stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
    return rc, assign, int(cost.value), stats
