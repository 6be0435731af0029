"""GPU parity of batched solves (lbdd_batch_*, lbdd_solve_batch, lbdd_autotune).

A batch only schedules independent runs of Alg. 2, so every instance must
end with exactly the oracle's allotment and objective, whatever its cluster
size, group, queue position or how its rounds are split between passes.
"""
import numpy as np
import pytest

import lbdd_inputs as L
import oracle

pytestmark = pytest.mark.gpu


def mix(count, seed0=0, n_range=(2.3, 3.2), k_range=(0.4, 2.2)):
    """Small instances of the batched mix (n ~ 200..1600, k ~ 2..160)."""
    return [L.make(L.batch_recipe(seed0 + i, n_range=n_range, k_range=k_range), dtype="i16")
            for i in range(count)]


@pytest.fixture(scope="module")
def small_mix():
    insts = mix(16)
    refs = [oracle.asral(x.cm, x.cap, x.pen) for x in insts]
    return insts, refs


def check(solvers, refs):
    for s, ref in zip(solvers, refs):
        assert s.rounds == len(ref.assign)
        assert s.objective == ref.delta
        assert np.array_equal(s.assignment(), ref.assign)
        assert np.array_equal(s.loads().astype(np.int64), ref.load)


def test_graph_batch_matches_oracle(gpu_lib, small_mix):
    insts, refs = small_mix
    solvers = [gpu_lib.Solver(x.cm, x.cap, x.pen) for x in insts]
    try:
        b = gpu_lib.Batch(solvers)
        cl, groups = b.plan()
        assert len(cl) == len(insts) and all(c in (1, 2, 4, 8, 16) for c in cl)
        assert sum(g[2] for g in groups) == len(insts)
        b.run()
        check(solvers, refs)
        b.run()                      # nothing left: a no-op
        check(solvers, refs)
        b.close()
    finally:
        for s in solvers:
            s.close()


def test_graph_batch_in_slices(gpu_lib, small_mix):
    """Replaying the graph with a round limit resumes every instance where
    it stopped."""
    insts, refs = small_mix
    solvers = [gpu_lib.Solver(x.cm, x.cap, x.pen) for x in insts]
    try:
        b = gpu_lib.Batch(solvers)
        for _ in range(200):
            b.run(97)
            if all(s.rounds == s.n for s in solvers):
                break
        check(solvers, refs)
        b.close()
    finally:
        for s in solvers:
            s.close()


@pytest.mark.parametrize("cluster", [1, 2])
def test_forced_cluster_and_cap(gpu_lib, small_mix, cluster):
    insts, refs = small_mix
    solvers = [gpu_lib.Solver(x.cm, x.cap, x.pen) for x in insts]
    try:
        gpu_lib.solve_batch([s.h for s in solvers], cluster_size=cluster, max_clusters=3)
        check(solvers, refs)
    finally:
        for s in solvers:
            s.close()


def test_resume_on_another_cluster_size(gpu_lib):
    """Solver state lives in device memory: a solve may continue on a
    different cluster size."""
    inst = L.make_named("tiny")
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    with gpu_lib.Solver(inst.cm, inst.cap, inst.pen, cluster=1) as s:
        s.solve(700)
        gpu_lib.set_option(s.h, gpu_lib.OPT_CLUSTER, 4)
        s.solve(600)
        gpu_lib.set_option(s.h, gpu_lib.OPT_CLUSTER, 2)
        s.solve()
        assert s.objective == ref.delta
        assert np.array_equal(s.assignment(), ref.assign)


def test_autotune_then_plan(gpu_lib):
    insts = mix(10, seed0=40, n_range=(2.5, 3.0), k_range=(0.5, 2.3))
    refs = [oracle.asral(x.cm, x.cap, x.pen) for x in insts]
    solvers = [gpu_lib.Solver(x.cm, x.cap, x.pen) for x in insts]
    try:
        gpu_lib.tune_clear()
        gpu_lib.autotune(solvers, probe_rounds=64)
        for s in solvers:
            assert s.rounds == 0          # autotuning works on clones
            assert gpu_lib.tune_get(gpu_lib.CM_I16, s.k, 1) > 0
        b = gpu_lib.Batch(solvers)
        cl, groups = b.plan()
        import torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert sum(c * n for c, n, _ in groups) <= sms
        b.run()
        check(solvers, refs)
        b.close()
    finally:
        gpu_lib.tune_clear()
        for s in solvers:
            s.close()


def test_batch_rejects_bad_arguments(gpu_lib):
    inst = L.random_small(5, n=30, k=4)
    with gpu_lib.Solver(inst.cm, inst.cap, inst.pen) as s:
        with pytest.raises(gpu_lib.LbddError):
            gpu_lib.Batch([s], cluster_size=3)
        with pytest.raises(gpu_lib.LbddError):
            gpu_lib.solve_batch([s], cluster_size=32)
        for C in (3, 6, 17):             # single solves take the batch sizes too
            with pytest.raises(gpu_lib.LbddError):
                gpu_lib.set_option(s.h, gpu_lib.OPT_CLUSTER, C)


def test_full_batched_mix_matches_oracle_golden(gpu_lib):
    """The 256-instance batched mix (n log-uniform in [1e3, 1e5), k in
    [10, 400)), one graph replay, against the stored oracle results."""
    import hashlib
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "batch256_oracle.json")))["instances"]
    insts = [L.make(L.batch_recipe(i), dtype="i16") for i in range(len(gold))]
    solvers = [gpu_lib.Solver(x.cm, x.cap, x.pen) for x in insts]
    try:
        b = gpu_lib.Batch(solvers)
        b.run()
        for g, x, s in zip(gold, insts, solvers):
            assert (g["n"], g["k"]) == (x.n, x.k)
            assert s.objective == g["delta"], g["i"]
            a = s.assignment().astype(np.int32)
            assert hashlib.sha256(a.tobytes()).hexdigest() == g["assign_sha256"], g["i"]
        b.close()
    finally:
        for s in solvers:
            s.close()


def test_mixed_variants_in_one_batch(gpu_lib):
    """Strict-LBDD solvers (their own launch group), solvers with penalty
    tables and plain solvers in one batch, in slices: each ends with its own
    oracle's result."""
    plain = mix(4, seed0=40)
    strict = [L.random_small(9700 + i, n=[60, 150][i % 2], k=[5, 12][i % 2], cm_max=25,
                             cap_frac=[0.7, 1.3][i % 2]) for i in range(3)]
    tabled = [L.random_small(9800 + i, n=120, k=[6, 17][i % 2], cm_max=30, cap_frac=0.5)
              for i in range(3)]
    qs = [L.penalty_table(9800 + i, x.k, 7, base=(1, 40), step=(0, 15)) for i, x in enumerate(tabled)]
    solvers, expect = [], []
    try:
        for x in plain:
            ref = oracle.asral(x.cm, x.cap, x.pen)
            solvers.append(gpu_lib.Solver(x.cm, x.cap, x.pen))
            expect.append((ref.delta, ref.assign))
        for x in strict:
            rc, a, cost, _ = oracle.strict(x.cm, x.cap)
            assert rc == 0
            solvers.append(gpu_lib.Solver(x.cm, x.cap, None, strict=True))
            expect.append((cost, a))
        for x, q in zip(tabled, qs):
            ref = oracle.asral_q(x.cm, x.cap, q)
            solvers.append(gpu_lib.Solver(x.cm, x.cap, x.pen, qtab=q))
            expect.append((ref.delta, ref.assign))
        order = [solvers[i] for i in (4, 0, 7, 1, 5, 9, 2, 8, 3, 6)]   # interleaved
        b = gpu_lib.Batch(order)
        for _ in range(3):
            b.run(40)
        b.run()
        b.close()
        for s, (delta, assign) in zip(solvers, expect):
            assert s.objective == delta
            assert np.array_equal(s.assignment(), assign)
    finally:
        for s in solvers:
            s.close()
