"""Seeded synthetic LBDD instances shared by the CPU oracle and the CUDA path.

This package holds no part of the solver: it only synthesises the inputs of
the problem statement (Section 2.1): the demand-service cost matrix CM
(n x k, demand-major, positive integers), the capacity c_s of every service
center and, per center, a constant per-unit overload penalty (the form used in
the paper's experiments, Section 5).

Named workloads (see ``CONFIGS``) reproduce the shape of the paper's
city-scale experiments with synthetic points because the New Delhi road
network is not available: unit demand, random center placement, total
capacity theta*n < n split at random, and penalties drawn from a range.

The numeric kernels live in ``gen.c`` (compiled to ``_gen.so`` by
:func:`build`); they are bit-reproducible across x86-64 and aarch64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_gen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into _gen.so (no fused multiply-add, OpenMP threads)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", src, "-o", _SO + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64, u64, u32, f64, i32 = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_double, ctypes.c_int32)
        lib.lbdd_gen_u64.argtypes = [u64, u32, u64]
        lib.lbdd_gen_u64.restype = u64
        lib.lbdd_gen_u01.argtypes = [u64, u32, u64]
        lib.lbdd_gen_u01.restype = f64
        lib.lbdd_gen_log.argtypes = [f64]
        lib.lbdd_gen_log.restype = f64
        lib.lbdd_gen_exp.argtypes = [f64]
        lib.lbdd_gen_exp.restype = f64
        lib.lbdd_gen_points_uniform.argtypes = [u64, u32, i64, P]
        lib.lbdd_gen_points_gmm.argtypes = [u64, i64, ctypes.c_int, f64, f64, P]
        lib.lbdd_gen_cm.argtypes = [i64, i64, P, P, f64, f64, f64, u64, ctypes.c_int, P]
        lib.lbdd_gen_cm_sample.argtypes = [i64, P, i64, P, P, f64, f64, f64, u64, P]
        lib.lbdd_gen_caps_uniform.argtypes = [u64, i64, i64, P]
        lib.lbdd_gen_caps_zipf.argtypes = [u64, i64, i64, f64, P]
        lib.lbdd_gen_pens.argtypes = [u64, i64, i32, i32, P]
        lib.lbdd_gen_logu_size.argtypes = [u64, u64, f64, f64]
        lib.lbdd_gen_logu_size.restype = i64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


# Stream ids of the point sets (must match the enum in gen.c).
_ST_DEMAND_XY, _ST_CENTER_XY = 1, 2


@dataclass
class Recipe:
    """Parameters of one synthetic instance."""
    n: int
    k: int
    seed: int
    layout: str = "uniform"          # "uniform" or "gmm" demand points
    ncomp: int = 30                  # mixture components for "gmm"
    sigma: tuple = (0.02, 0.08)      # component sigma range for "gmm"
    scale: float = 100.0             # CM = max(1, floor(scale*dist*rf + 0.5))
    road: tuple = (1.0, 1.0)         # road-factor range per (d, s) pair
    cap_frac: float = 0.9            # total capacity = floor(cap_frac * n)
    cap_dist: str = "uniform"        # "uniform" or "zipf"
    zipf: float = 1.2
    pen: tuple = (50, 500)           # per-unit penalty range, inclusive
    name: str = ""


@dataclass
class Instance:
    n: int
    k: int
    cm: np.ndarray                   # (n, k) int32 or int16, demand-major
    cap: np.ndarray                  # (k,) int32
    pen: np.ndarray                  # (k,) int32
    recipe: Recipe = field(repr=False, default=None)
    dxy: np.ndarray = field(repr=False, default=None)
    sxy: np.ndarray = field(repr=False, default=None)

    def cm_sample(self, pairs: np.ndarray) -> np.ndarray:
        """Regenerate CM[d, s] for an (m, 2) array of (d, s) pairs."""
        lib = _load()
        r = self.recipe
        pairs = np.ascontiguousarray(pairs, dtype=np.int64)
        out = np.empty(len(pairs), dtype=np.int64)
        _check(lib.lbdd_gen_cm_sample(len(pairs), _ptr(pairs), self.k, _ptr(self.dxy),
                                      _ptr(self.sxy), r.scale, r.road[0], r.road[1],
                                      r.seed, _ptr(out)), "cm_sample")
        return out


# Workloads.  "tiny" is the small single instance (2,000 x 20); "city" the
# city-scale single solve (200,000 x 500, clustered demand, road factors,
# Zipf capacities); "large" the HBM-bound solve (2,000,000 x 2,000); "wide"
# a test instance with the large one's k and tight capacity.
CONFIGS = {
    "tiny": Recipe(n=2000, k=20, seed=1, layout="uniform", scale=100.0, cap_frac=0.9,
                   cap_dist="uniform", pen=(50, 500), name="tiny"),
    "city": Recipe(n=200_000, k=500, seed=2, layout="gmm", scale=1000.0, road=(1.0, 1.5),
                   cap_frac=0.8, cap_dist="zipf", zipf=1.2, pen=(200, 2000), name="city"),
    "large": Recipe(n=2_000_000, k=2000, seed=3, layout="gmm", scale=1000.0, road=(1.0, 1.5),
                    cap_frac=0.85, cap_dist="zipf", zipf=1.2, pen=(100, 5000), name="large"),
    # as "large" but with 20,000 units and total capacity 0.3 n: a solver
    # whose k x k table does not fit a cluster's shared memory applies
    # refinements from the first few hundred rounds on
    "wide": Recipe(n=20_000, k=2000, seed=7, layout="gmm", scale=1000.0, road=(1.0, 1.5),
                   cap_frac=0.3, cap_dist="uniform", pen=(100, 5000), name="wide"),
}

BATCH_SEED0 = 1000      # batched mix: instance i uses seed 1000 + i
SERVE_SEED0 = 100000    # serving stream: request i uses seed 100000 + i


def _mix_recipe(seed: int, name: str, n_range, k_range) -> Recipe:
    lib = _load()
    n = int(lib.lbdd_gen_logu_size(seed, 0, n_range[0], n_range[1]))
    k = int(lib.lbdd_gen_logu_size(seed, 1, k_range[0], k_range[1]))
    return Recipe(n=n, k=k, seed=seed, layout="uniform", scale=100.0, cap_frac=0.9,
                  cap_dist="uniform", pen=(50, 500), name=name)


def batch_recipe(i: int, n_range=(3.0, 5.0), k_range=(1.0, 2.6020599913279625)) -> Recipe:
    """Instance i of the batched mix: n log-uniform in [10^3, 10^5), k
    log-uniform in [10, 400), otherwise generated like "tiny"."""
    return _mix_recipe(BATCH_SEED0 + i, f"batch{i}", n_range, k_range)


SERVE_LARGE = (1_000_000, 1000)   # size of the serving stream's large requests


def serve_recipe(i: int, large_frac: float = 0.05, large=SERVE_LARGE):
    """Request i of the serving stream and whether it is a large one.

    With probability large_frac (one draw of the counter stream of seed
    100000 + i) the request is large: n x k = `large`, clustered demand,
    road factors and Zipf capacities like the city-scale instance.  Otherwise
    it is sized and generated like the batched mix."""
    lib = _load()
    seed = SERVE_SEED0 + i
    if lib.lbdd_gen_u01(seed, 40, 0) < large_frac:
        n, k = large
        return Recipe(n=int(n), k=int(k), seed=seed, layout="gmm", scale=1000.0, road=(1.0, 1.5),
                      cap_frac=0.85, cap_dist="zipf", zipf=1.2, pen=(100, 5000),
                      name=f"serve{i}L"), True
    return _mix_recipe(seed, f"serve{i}", (3.0, 5.0), (1.0, 2.6020599913279625)), False


def arrival_times(count: int, rate: float) -> np.ndarray:
    """Poisson arrivals of the serving stream (seconds from the first):
    exponential gaps -ln(1 - U) / rate, U from the counter stream of seed
    100000; arrival 0 is at time 0."""
    lib = _load()
    gaps = np.array([-np.log1p(-lib.lbdd_gen_u01(SERVE_SEED0, 41, i)) for i in range(count)])
    gaps[0] = 0.0
    return np.cumsum(gaps) / rate


def make(recipe: Recipe, dtype: str = "i32", points_only: bool = False) -> Instance:
    """Synthesise one instance.  dtype: "i32" or "i16" (raises if a cost
    does not fit int16)."""
    lib = _load()
    r = recipe
    n, k = int(r.n), int(r.k)
    dxy = np.empty((n, 2), dtype=np.float64)
    sxy = np.empty((k, 2), dtype=np.float64)
    if r.layout == "uniform":
        _check(lib.lbdd_gen_points_uniform(r.seed, _ST_DEMAND_XY, n, _ptr(dxy)), "points")
    elif r.layout == "gmm":
        _check(lib.lbdd_gen_points_gmm(r.seed, n, r.ncomp, r.sigma[0], r.sigma[1], _ptr(dxy)),
               "gmm")
    else:
        raise ValueError(r.layout)
    _check(lib.lbdd_gen_points_uniform(r.seed, _ST_CENTER_XY, k, _ptr(sxy)), "centers")
    cap = np.empty(k, dtype=np.int32)
    total = int(np.floor(r.cap_frac * n))
    if r.cap_dist == "uniform":
        _check(lib.lbdd_gen_caps_uniform(r.seed, k, total, _ptr(cap)), "caps")
    elif r.cap_dist == "zipf":
        _check(lib.lbdd_gen_caps_zipf(r.seed, k, total, r.zipf, _ptr(cap)), "caps")
    else:
        raise ValueError(r.cap_dist)
    pen = np.empty(k, dtype=np.int32)
    _check(lib.lbdd_gen_pens(r.seed, k, r.pen[0], r.pen[1], _ptr(pen)), "pens")
    if points_only:
        cm = None
    else:
        np_dt = {"i32": np.int32, "i16": np.int16}[dtype]
        cm = np.empty((n, k), dtype=np_dt)
        _check(lib.lbdd_gen_cm(n, k, _ptr(dxy), _ptr(sxy), r.scale, r.road[0], r.road[1],
                               r.seed, np.dtype(np_dt).itemsize, _ptr(cm)), "cm")
    return Instance(n=n, k=k, cm=cm, cap=cap, pen=pen, recipe=r, dxy=dxy, sxy=sxy)


def make_named(name: str, dtype: str = "i32", **overrides) -> Instance:
    base = CONFIGS[name]
    r = Recipe(**{**base.__dict__, **overrides})
    return make(r, dtype=dtype)


@dataclass
class RoadNetwork:
    """Directed CSR graph (both directions of every road), node coordinates,
    and the centers / demand nodes chosen on it."""
    V: int
    row_ptr: np.ndarray      # (V + 1,) int32
    col: np.ndarray          # (E,) int32
    w: np.ndarray            # (E,) int32, >= 1
    xy: np.ndarray           # (V, 2) float64
    centers: np.ndarray      # (k,) int32 node ids
    demand: np.ndarray       # (n,) int32 node ids (every other node)


def road_network(seed: int, W: int, H: int, k: int, diag_frac: float = 0.15) -> RoadNetwork:
    """Synthetic road network standing in for the paper's New Delhi graph
    (Section 5): a W x H grid of intersections (jittered positions) with
    4-neighbour roads plus a fraction of diagonal roads; road length =
    floor(100 * euclidean * rf + 0.5) with rf in [1, 1.5] per road, at least
    1.  k distinct nodes become service centers, every other node is one
    unit of demand.  All draws come from the counter stream of `seed`."""
    lib = _load()
    V = W * H
    u01 = lambda st, i: lib.lbdd_gen_u01(seed, st, i)
    xy = np.empty((V, 2), np.float64)
    for v in range(V):
        x, y = v % W, v // W
        xy[v, 0] = (x + 0.35 * (u01(70, 2 * v) - 0.5)) / W
        xy[v, 1] = (y + 0.35 * (u01(70, 2 * v + 1) - 0.5)) / H
    roads = []
    for v in range(V):
        x, y = v % W, v // W
        if x + 1 < W:
            roads.append((v, v + 1))
        if y + 1 < H:
            roads.append((v, v + W))
        if x + 1 < W and y + 1 < H and u01(71, v) < diag_frac:
            roads.append((v, v + W + 1))
    adj = [[] for _ in range(V)]
    for i, (a, b) in enumerate(roads):
        dx, dy = xy[a] - xy[b]
        rf = 1.0 + 0.5 * u01(72, i)
        wt = max(1, int(np.floor(100.0 * np.sqrt(dx * dx + dy * dy) * W * rf + 0.5)))
        adj[a].append((b, wt))
        adj[b].append((a, wt))
    row_ptr = np.zeros(V + 1, np.int32)
    for v in range(V):
        row_ptr[v + 1] = row_ptr[v] + len(adj[v])
    col = np.empty(row_ptr[-1], np.int32)
    w = np.empty(row_ptr[-1], np.int32)
    for v in range(V):
        for i, (b, wt) in enumerate(sorted(adj[v])):
            col[row_ptr[v] + i] = b
            w[row_ptr[v] + i] = wt
    # k distinct centers by a seeded partial shuffle
    perm = np.arange(V, dtype=np.int64)
    for i in range(k):
        j = i + int(lib.lbdd_gen_u64(seed, 73, i) % (V - i))
        perm[i], perm[j] = perm[j], perm[i]
    centers = np.sort(perm[:k]).astype(np.int32)
    is_c = np.zeros(V, bool)
    is_c[centers] = True
    demand = np.nonzero(~is_c)[0].astype(np.int32)
    return RoadNetwork(V=V, row_ptr=row_ptr, col=col, w=w, xy=xy, centers=centers, demand=demand)


def penalty_table(seed: int, k: int, Q: int, base=(1, 30), step=(0, 10)) -> np.ndarray:
    """General penalty functions (Def. 4) as a k x Q table: q_s(j) for the
    j-th allotment beyond capacity, j = 1..Q (the last value repeats).
    q_s(1) uniform in `base`, then non-decreasing by steps uniform in `step`;
    drawn from the counter stream of `seed`."""
    lib = _load()
    q = np.empty((k, Q), dtype=np.int32)
    for s in range(k):
        v = base[0] + int(lib.lbdd_gen_u64(seed, 60, s) % (base[1] - base[0] + 1))
        for j in range(Q):
            if j:
                v += step[0] + int(lib.lbdd_gen_u64(seed, 61, s * Q + j) % (step[1] - step[0] + 1))
            q[s, j] = v
    return q


def random_small(seed: int, n: int, k: int, cm_max: int = 20, cap_frac: float = 0.7,
                 pen=(1, 30)) -> Instance:
    """Tiny instance with CM uniform in [1, cm_max] drawn from the counter
    stream (many ties on purpose), for exhaustive and exact-solver checks."""
    lib = _load()
    cm = np.empty((n, k), dtype=np.int32)
    for d in range(n):
        for s in range(k):
            cm[d, s] = 1 + lib.lbdd_gen_u64(seed, 11, d * k + s) % cm_max
    cap = np.empty(k, dtype=np.int32)
    total = max(k, int(np.floor(cap_frac * n)))
    _check(lib.lbdd_gen_caps_uniform(seed, k, total, _ptr(cap)), "caps")
    p = np.empty(k, dtype=np.int32)
    _check(lib.lbdd_gen_pens(seed, k, pen[0], pen[1], _ptr(p)), "pens")
    r = Recipe(n=n, k=k, seed=seed, name=f"small{seed}")
    return Instance(n=n, k=k, cm=cm, cap=cap, pen=p, recipe=r)
