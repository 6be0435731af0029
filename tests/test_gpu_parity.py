"""GPU parity: the CUDA solver (through the C ABI) against the CPU oracle.

All integer: the allotment vector, the tracked objective, the loads and the
best-transfer table must match the oracle bit for bit.  Oracle inputs and
expected values come only from the seeded generator and the oracle (or the
stored oracle goldens under tests/golden/).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import lbdd_inputs as L
import oracle

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def run_gpu(lb, cm, cap, pen, rounds=-1, cluster=0, ncyc_skip=True, npath_reuse=True):
    with lb.Solver(cm, cap, pen, cluster=cluster, ncyc_skip=ncyc_skip,
                   npath_reuse=npath_reuse) as s:
        s.solve(rounds)
        return s.assignment(), s.objective, s.loads(), s.stats(), s.table()


def assert_same(gpu, ref, k):
    assign, delta, loads, stats, _ = gpu
    assert delta == ref.delta
    assert np.array_equal(assign, ref.assign)
    assert np.array_equal(loads.astype(np.int64), ref.load)


@pytest.mark.parametrize("cluster", [0, 1, 2, 4])
def test_tiny_matches_golden(gpu_lib, cluster):
    inst = L.make_named("tiny")
    with open(os.path.join(GOLD, "tiny_oracle.json")) as f:
        gold = json.load(f)
    assign, delta, loads, st, _ = run_gpu(gpu_lib, inst.cm, inst.cap, inst.pen, cluster=cluster)
    assert delta == gold["delta"]
    assert sha(assign.astype(np.int32)) == gold["assign_sha256"]
    assert st.rounds == inst.n
    assert st.cycles_applied == gold["stats"]["cycles_applied"]
    assert st.paths_applied == gold["stats"]["paths_applied"]
    assert st.moves == gold["stats"]["moves"]


def test_phase_timers_change_nothing_but_stats(gpu_lib):
    inst = L.make_named("tiny")
    with open(os.path.join(GOLD, "tiny_oracle.json")) as f:
        gold = json.load(f)
    for timers in (False, True):
        with gpu_lib.Solver(inst.cm, inst.cap, inst.pen, phase_timers=timers) as s:
            s.solve()
            st = s.stats()
            assert s.objective == gold["delta"]
            assert sha(s.assignment().astype(np.int32)) == gold["assign_sha256"]
            assert st.rounds_ns > 0
            assert (st.relax_ns > 0) == timers and (st.front_sum > 0) == timers


def test_tiny_without_skip_and_int32_storage(gpu_lib):
    inst = L.make_named("tiny")
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    out = run_gpu(gpu_lib, inst.cm, inst.cap, inst.pen, ncyc_skip=False, npath_reuse=False)
    assert_same(out, ref, inst.k)
    # every Alg. 1 and Alg. 4 call ran Bellman-Ford: same call count as the oracle
    assert out[3].bf_calls == ref.stats["bf_calls"]
    assert out[3].ncyc_skipped == 0 and out[3].npath_reused == 0
    # a CM too wide for int16 stays int32 and gives the same result
    cm = inst.cm.astype(np.int32) + 40000
    ref2 = oracle.asral(cm, inst.cap, inst.pen)
    out2 = run_gpu(gpu_lib, cm, inst.cap, inst.pen)
    assert out2[3].cm_elem_bytes == 4
    assert_same(out2, ref2, inst.k)


@pytest.mark.parametrize("seed", range(24))
def test_random_small_instances(gpu_lib, seed):
    """Many ties (CM in [1, cm_max]) exercise every tie-break rule."""
    n = [30, 120, 257, 600][seed % 4]
    k = [2, 5, 9, 17, 33, 70][seed % 6]
    inst = L.random_small(5000 + seed, n=n, k=k, cm_max=[3, 12, 50][seed % 3],
                          cap_frac=[0.3, 0.7, 0.95][(seed // 3) % 3],
                          pen=[(1, 4), (1, 40), (20, 300)][(seed // 2) % 3])
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    assert ref.rc == 0
    for cluster in (1, 2, 4) if k >= 4 else (1,):
        out = run_gpu(gpu_lib, inst.cm, inst.cap, inst.pen, cluster=cluster)
        assert_same(out, ref, k)
        tc_ref, td_ref = oracle.best_transfer(inst.cm, ref.assign)
        tc, td = out[4]
        tc_ref = np.where(tc_ref >= oracle.INF, 2**31 - 1, tc_ref)
        assert np.array_equal(tc, tc_ref) and np.array_equal(td, td_ref)


@pytest.mark.parametrize("seed", range(6))
def test_shortcuts_do_not_change_results(gpu_lib, seed):
    """Skipping Alg. 1 when T is unchanged and answering Alg. 4 from Alg. 1's
    labels must give exactly the same allotment as running every
    Bellman-Ford (and as the oracle)."""
    inst = L.random_small(6100 + seed, n=400, k=[6, 23, 40][seed % 3], cm_max=[6, 40][seed % 2],
                          cap_frac=0.6, pen=(1, 30))
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    outs = [run_gpu(gpu_lib, inst.cm, inst.cap, inst.pen, cluster=c, ncyc_skip=a, npath_reuse=b)
            for c in (1, 2) for a in (True, False) for b in (True, False)]
    for out in outs:
        assert_same(out, ref, inst.k)
    assert outs[0][3].npath_reused > 0


def test_single_center_and_ample_capacity(gpu_lib):
    inst = L.random_small(77, n=300, k=1, cm_max=30)
    cap, pen = np.array([100], np.int32), np.array([9], np.int32)
    out = run_gpu(gpu_lib, inst.cm, cap, pen)
    assert out[1] == int(inst.cm.sum()) + 9 * 200
    inst = L.random_small(78, n=500, k=12, cm_max=30)
    cap = np.full(12, 500, np.int32)
    out = run_gpu(gpu_lib, inst.cm, cap, inst.pen)
    assert out[1] == int(inst.cm.min(axis=1).sum()) and out[3].moves == 0


def test_resume_is_exact(gpu_lib):
    inst = L.make_named("tiny")
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    with gpu_lib.Solver(inst.cm, inst.cap, inst.pen) as s:
        for chunk in (1, 699, 300, 1000):
            s.solve(chunk)
        assert s.rounds == 2000
        assert s.objective == ref.delta
        assert np.array_equal(s.assignment(), ref.assign)
        part = oracle.asral(inst.cm, inst.cap, inst.pen, max_rounds=0)
        assert part.delta == 0


def test_truncated_prefix_matches_oracle(gpu_lib):
    inst = L.make_named("tiny")
    for R in (1, 17, 555):
        ref = oracle.asral(inst.cm, inst.cap, inst.pen, max_rounds=R)
        out = run_gpu(gpu_lib, inst.cm, inst.cap, inst.pen, rounds=R)
        assert_same(out, ref, inst.k)


def test_batch_matches_individual(gpu_lib):
    insts = [L.make(L.batch_recipe(i, n_range=(2.5, 3.3), k_range=(0.5, 1.9)), dtype="i16")
             for i in range(12)]
    refs = [oracle.asral(x.cm, x.cap, x.pen) for x in insts]
    solvers = [gpu_lib.Solver(x.cm, x.cap, x.pen) for x in insts]
    try:
        gpu_lib.solve_batch([s.h for s in solvers])
        for s, ref in zip(solvers, refs):
            assert s.objective == ref.delta
            assert np.array_equal(s.assignment(), ref.assign)
    finally:
        for s in solvers:
            s.close()


def test_city_prefix_matches_golden(gpu_lib):
    """City-scale instance (200,000 x 500), first 3,000 rounds, against the
    stored oracle result; the best-transfer table must also equal the
    oracle's table for the oracle's own allotment at that point."""
    inst = L.make_named("city", dtype="i16")
    with open(os.path.join(GOLD, "city_r3000_oracle.json")) as f:
        gold = json.load(f)
    assert sha(inst.cm.astype(np.int32)) == gold["cm_sha256"]
    assign, delta, loads, st, (tc, td) = run_gpu(gpu_lib, inst.cm, inst.cap, inst.pen,
                                                 rounds=3000)
    assert delta == gold["delta"]
    assert sha(assign.astype(np.int32)) == gold["assign_sha256"]
    assert sha(loads.astype(np.int64)) == gold["load_sha256"]
    assert st.moves == gold["stats"]["moves"] > 0
    # the allotment is the oracle's (digest above), so the oracle's table of
    # it (Defs. 8-10, by definition) is the expected incremental table
    rtc, rtd = oracle.best_transfer(inst.cm, assign)
    assert np.array_equal(tc, np.where(rtc >= oracle.INF, 2**31 - 1, rtc))
    assert np.array_equal(td, rtd)


def test_rejects_bad_input(gpu_lib):
    cm = np.ones((4, 3), np.int32)
    cap = np.ones(3, np.int32)
    pen = np.ones(3, np.int32)
    bad = cm.copy()
    bad[2, 1] = 0
    with pytest.raises(gpu_lib.LbddError) as e:
        gpu_lib.Solver(bad, cap, pen)
    assert e.value.code == gpu_lib.ERR_ARG
    with pytest.raises(gpu_lib.LbddError):
        gpu_lib.Solver(cm, np.array([1, 0, 1], np.int32), pen)
    with pytest.raises(gpu_lib.LbddError):
        gpu_lib.Solver(cm, cap, np.array([1, 1, -2], np.int32))


def test_city_full_solve_matches_golden(gpu_lib):
    """The whole city-scale solve (200,000 x 500, every round) against the
    stored oracle result."""
    inst = L.make_named("city", dtype="i16")
    with open(os.path.join(GOLD, "city_oracle.json")) as f:
        gold = json.load(f)
    assert sha(inst.cm.astype(np.int32)) == gold["cm_sha256"]
    with gpu_lib.Solver(inst.cm, inst.cap, inst.pen) as s:
        s.solve()
        assert s.rounds == inst.n
        assert s.objective == gold["delta"]
        assert sha(s.assignment().astype(np.int32)) == gold["assign_sha256"]
        assert sha(s.loads().astype(np.int64)) == gold["load_sha256"]
        st = s.stats()
        assert st.cycles_applied == gold["stats"]["cycles_applied"]
        assert st.paths_applied == gold["stats"]["paths_applied"]
        assert st.moves == gold["stats"]["moves"]


def test_large_prefix_matches_golden(gpu_lib):
    """The 2,000,000 x 2,000 instance (CM 8 GB as int16): prologue over the
    whole CM and the first 200 rounds against the stored oracle result."""
    inst = L.make_named("large", dtype="i16")
    with open(os.path.join(GOLD, "large_r200_oracle.json")) as f:
        gold = json.load(f)
    assert (inst.n, inst.k, inst.recipe.seed) == (gold["n"], gold["k"], gold["seed"])
    with gpu_lib.Solver(inst.cm, inst.cap, inst.pen) as s:
        s.solve(gold["rounds"])
        assert s.objective == gold["delta"]
        assert sha(s.assignment().astype(np.int32)) == gold["assign_sha256"]
        assert sha(s.loads().astype(np.int64)) == gold["load_sha256"]


def test_largest_k(gpu_lib):
    """k = lbdd_max_centers(), the most centers a 16-CTA cluster's shared
    memory holds (slack and penalty replicas of every center, the path
    buffers, and the double-buffered Bellman-Ford messages of all 16 CTAs):
    a prefix of the solve and the best-transfer table after it equal the
    oracle's; one more center is refused at creation."""
    k = gpu_lib.max_centers()
    assert k == 5376
    inst = L.make(L.Recipe(n=5500, k=k, seed=4826, cap_frac=0.99, pen=(1, 30), name="maxk"))
    R = 12
    ref = oracle.asral(inst.cm, inst.cap, inst.pen, max_rounds=R)
    assert ref.rc == 0
    assign, delta, loads, st, (tc, td) = run_gpu(gpu_lib, inst.cm, inst.cap, inst.pen, rounds=R)
    assert st.cluster_size == 16
    assert_same((assign, delta, loads, st, None), ref, k)
    tc_ref, td_ref = oracle.best_transfer(inst.cm, ref.assign)
    tc_ref = np.where(tc_ref >= oracle.INF, 2**31 - 1, tc_ref)
    assert np.array_equal(tc, tc_ref) and np.array_equal(td, td_ref)
    wide = np.ones((8, k + 1), np.int32)
    with pytest.raises(gpu_lib.LbddError) as e:
        gpu_lib.Solver(wide, np.ones(k + 1, np.int32), np.ones(k + 1, np.int32))
    assert e.value.code == gpu_lib.ERR_ARG


@pytest.mark.parametrize("n,k,cm_max,cap_frac", [
    (1, 1, 5, 0.5),      # one unit, one center
    (1, 7, 9, 0.5),      # one unit: Delta is its cheapest cost
    (40, 1, 9, 0.1),     # one center, overloaded from the fifth unit on
    (200, 9, 1, 0.5),    # every cost equal: only the tie-break rules decide
    (64, 64, 2, 1.0),    # capacity exactly n, one slot per center
    (129, 33, 4, 0.2),   # ragged: 33 columns over 1, 2 and 4 CTAs
])
def test_degenerate_instances(gpu_lib, n, k, cm_max, cap_frac):
    inst = L.random_small(9100 + n + k, n=n, k=k, cm_max=cm_max, cap_frac=cap_frac, pen=(1, 9))
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    assert ref.rc == 0
    assert ref.delta == oracle.objective(inst.cm, inst.cap, inst.pen, ref.assign)
    for cluster in sorted({1, min(2, k), min(4, k)}):
        out = run_gpu(gpu_lib, inst.cm, inst.cap, inst.pen, cluster=cluster)
        assert_same(out, ref, k)
