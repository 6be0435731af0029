"""The seeded input generator: determinism, ranges and the stated recipe."""
import hashlib
import json
import os

import numpy as np
import pytest

import lbdd_inputs as L

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_counter_stream_is_pure():
    lib = L._load()
    a = [lib.lbdd_gen_u64(7, 3, i) for i in range(100)]
    b = [lib.lbdd_gen_u64(7, 3, i) for i in reversed(range(100))][::-1]
    assert a == b
    assert len(set(a)) == 100
    assert lib.lbdd_gen_u64(7, 3, 5) != lib.lbdd_gen_u64(7, 4, 5)
    assert lib.lbdd_gen_u64(7, 3, 5) != lib.lbdd_gen_u64(8, 3, 5)


def test_deterministic_log_exp_close_to_libm():
    lib = L._load()
    import math
    for x in [1e-12, 1e-3, 0.3, 0.5, 0.7071, 1.0, 1.5, 2.0, 10.0, 1e6]:
        assert abs(lib.lbdd_gen_log(x) - math.log(x)) <= 4e-15 * max(1.0, abs(math.log(x)))
    for x in [-30.0, -1.0, -0.2, 0.0, 0.3, 1.0, 5.0, 11.5]:
        assert abs(lib.lbdd_gen_exp(x) / math.exp(x) - 1.0) < 1e-14


def test_tiny_recipe_shape_and_bytes():
    inst = L.make_named("tiny")
    assert inst.cm.shape == (2000, 20) and inst.cm.dtype == np.int32
    assert inst.cm.min() >= 1
    assert int(inst.cap.sum()) == 1800 and inst.cap.min() >= 1      # 0.9 * n
    assert inst.pen.min() >= 50 and inst.pen.max() <= 500
    # CM entry = max(1, round(100 * Euclidean distance)) on the unit square
    d = np.sqrt(((inst.dxy[:, None, :] - inst.sxy[None, :, :]) ** 2).sum(-1))
    approx = np.maximum(1, np.floor(100 * d + 0.5))
    assert np.abs(approx - inst.cm).max() <= 1
    # the stored digest catches drift of the generator across machines
    with open(os.path.join(GOLD, "tiny_oracle.json")) as f:
        gold = json.load(f)
    assert hashlib.sha256(inst.cm.tobytes()).hexdigest() == gold["cm_sha256"]


def test_int16_matches_int32():
    r = L.Recipe(n=3000, k=50, seed=9, layout="gmm", scale=1000.0, road=(1.0, 1.5),
                 cap_frac=0.8, cap_dist="zipf", pen=(200, 2000))
    a = L.make(r, "i32")
    b = L.make(r, "i16")
    assert np.array_equal(a.cm, b.cm.astype(np.int32))
    assert int(a.cap.sum()) == int(np.floor(0.8 * 3000))


def test_int16_range_error():
    r = L.Recipe(n=10, k=3, seed=1, scale=1e6)
    with pytest.raises(RuntimeError):
        L.make(r, "i16")


def test_cm_sample_regenerates_entries():
    r = L.Recipe(n=500, k=40, seed=5, layout="gmm", scale=1000.0, road=(1.0, 1.5))
    inst = L.make(r)
    rng = np.random.default_rng(0)
    pairs = np.stack([rng.integers(0, 500, 64), rng.integers(0, 40, 64)], 1)
    assert np.array_equal(inst.cm_sample(pairs), inst.cm[pairs[:, 0], pairs[:, 1]])


def test_zipf_caps_are_skewed_and_exact():
    r = L.CONFIGS["city"]
    pts = L.make(r, points_only=True)
    caps = np.sort(pts.cap)[::-1]
    assert int(caps.sum()) == 160000 and caps.min() >= 1
    # rank-1 / rank-10 ratio of r^-1.2 weights is 10^1.2 ~ 15.8
    assert 12 < caps[0] / caps[9] < 20


def test_batch_sizes_log_uniform():
    ns, ks = [], []
    for i in range(256):
        r = L.batch_recipe(i)
        assert 1000 <= r.n < 100000 and 10 <= r.k < 400
        ns.append(r.n)
        ks.append(r.k)
    # log-uniform: roughly half below the geometric midpoint
    assert 0.35 < np.mean(np.array(ns) < 10000) < 0.65
    assert 0.35 < np.mean(np.array(ks) < 63) < 0.65


def test_road_network_structure():
    """Two-way roads (the CSR holds both directions with equal lengths),
    lengths >= 1, a connected grid, k distinct centers and every other node
    one unit of demand; the same seed gives the same network."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    g = L.road_network(5, 20, 13, 9)
    assert g.V == 260 and len(g.row_ptr) == g.V + 1 and g.row_ptr[0] == 0
    assert (np.diff(g.row_ptr) >= 2).all() and (g.w >= 1).all()
    A = csr_matrix((g.w, g.col, g.row_ptr), shape=(g.V, g.V))
    assert (A != A.T).nnz == 0
    assert connected_components(A, directed=False)[0] == 1
    assert len(np.unique(g.centers)) == 9
    assert np.array_equal(np.sort(np.concatenate([g.centers, g.demand])), np.arange(g.V))
    h = L.road_network(5, 20, 13, 9)
    assert np.array_equal(g.w, h.w) and np.array_equal(g.centers, h.centers)


def test_penalty_table_is_positive_and_non_decreasing():
    q = L.penalty_table(3, 50, 12, base=(1, 40), step=(0, 15))
    assert q.shape == (50, 12) and (q >= 1).all() and (np.diff(q, axis=1) >= 0).all()
    assert (q[:, 0] <= 40).all() and (np.diff(q, axis=1) <= 15).all()
    assert np.array_equal(q, L.penalty_table(3, 50, 12, base=(1, 40), step=(0, 15)))
