"""GPU parity on the solver code paths that the full-size workloads take.

* Bellman-Ford relaxations that read the owned cost slice of the
  best-transfer table from global memory.  Every solver whose slice does not
  fit shared memory takes this path (2,000 centers on a 16-CTA cluster, for
  example); here it is forced on small instances with the cost-slice option
  off, on clusters of 1, 2, 4 and 16 CTAs.
* The int32 solver: costs of 32768 and more are not narrowed to int16, so the
  int32 kernel (four costs per 16-byte vector, int32 slices, 64-bit labels)
  runs, on clusters of 2, 4 and 16 CTAs, with the slice in shared memory and
  in global memory.
* A 20,000 x 2,000 instance with total capacity 0.3 n: its slice misses
  shared memory, and its first 1,000 rounds apply cycles and paths.
* The 2,000,000 x 2,000 instance over its first 9,000 rounds, which include
  the first overloaded centers and the paths applied there.

Each case compares the allotment, the tracked objective (Eq. 1), the loads,
the refinement counts and the best-transfer table (Defs. 8-10) with the CPU
oracle, bit for bit, and checks that the case really applied refinements.
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
TINF = 2**31 - 1


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def solve(lb, inst, cluster, tc_smem=True, rounds=-1, **kw):
    with lb.Solver(inst.cm, inst.cap, inst.pen, cluster=cluster, tc_smem=tc_smem, **kw) as s:
        s.solve(rounds)
        return s.assignment(), s.objective, s.loads(), s.stats(), s.table()


def check(out, ref, cm):
    assign, delta, loads, st, (tc, td) = out
    assert delta == ref.delta
    assert np.array_equal(assign, ref.assign)
    assert np.array_equal(loads.astype(np.int64), ref.load)
    assert st.cycles_applied == ref.stats["cycles_applied"]
    assert st.paths_applied == ref.stats["paths_applied"]
    assert st.moves == ref.stats["moves"]
    rtc, rtd = oracle.best_transfer(cm, ref.assign)
    assert np.array_equal(tc, np.where(rtc >= oracle.INF, TINF, rtc))
    assert np.array_equal(td, rtd)


def clusters_for(k, sizes):
    return [c for c in sizes if c <= k]


GLOBAL_CASES = [  # (n, k, cm_max, cap_frac, pen)
    (120, 5, 12, 0.3, (1, 40)),
    (257, 17, 3, 0.7, (20, 300)),
    (600, 33, 50, 0.3, (1, 4)),
    (400, 70, 12, 0.5, (1, 30)),
    (300, 21, 6, 0.95, (20, 300)),
    (500, 40, 40, 0.2, (1, 40)),
    (129, 33, 4, 0.2, (1, 9)),
    (200, 9, 1, 0.5, (1, 9)),
    (64, 64, 2, 1.0, (1, 9)),
    (40, 1, 9, 0.1, (1, 9)),
]


@pytest.mark.parametrize("case", range(len(GLOBAL_CASES)))
def test_global_memory_relaxation(gpu_lib, case):
    """Cost slice forced out of shared memory: every relaxation reads the
    table column from global memory."""
    n, k, cm_max, cap_frac, pen = GLOBAL_CASES[case]
    inst = L.random_small(7300 + case, n=n, k=k, cm_max=cm_max, cap_frac=cap_frac, pen=pen)
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    assert ref.rc == 0
    for cluster in clusters_for(k, (1, 2, 4, 16)):
        out = solve(gpu_lib, inst, cluster, tc_smem=False)
        assert out[3].cost_slice_in_smem == 0 and out[3].cluster_size == cluster
        check(out, ref, inst.cm)


def test_global_memory_relaxation_applies_refinements(gpu_lib):
    """The cases above include instances where cycles and paths are applied."""
    moved = 0
    for case, (n, k, cm_max, cap_frac, pen) in enumerate(GLOBAL_CASES):
        inst = L.random_small(7300 + case, n=n, k=k, cm_max=cm_max, cap_frac=cap_frac, pen=pen)
        ref = oracle.asral(inst.cm, inst.cap, inst.pen)
        moved += ref.stats["cycles_applied"] > 0 and ref.stats["paths_applied"] > 0
    assert moved >= 4


INT32_CASES = [  # (n, k, cm_max, offset, cap_frac, pen)
    (300, 17, 100000, 0, 0.5, (1, 40000)),
    (600, 40, 12, 40000, 0.3, (1, 30)),
    (257, 33, 3, 40000, 0.7, (20, 300)),
    (500, 70, 70000, 0, 0.2, (1000, 90000)),
    (400, 16, 50, 40000, 0.95, (1, 4)),
    (200, 23, 2000000, 0, 0.6, (1, 3000000)),
]


@pytest.mark.parametrize("case", range(len(INT32_CASES)))
def test_int32_solver(gpu_lib, case):
    """CM with costs of 32768 and more stays int32 (no narrowing)."""
    n, k, cm_max, off, cap_frac, pen = INT32_CASES[case]
    inst = L.random_small(7400 + case, n=n, k=k, cm_max=cm_max, cap_frac=cap_frac, pen=pen)
    inst.cm = inst.cm + np.int32(off)
    assert inst.cm.max() >= 32768
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    assert ref.rc == 0 and ref.stats["moves"] > 0
    for cluster in clusters_for(k, (2, 4, 16)):
        for tc_smem in (True, False):
            out = solve(gpu_lib, inst, cluster, tc_smem=tc_smem)
            assert out[3].cm_elem_bytes == 4 and out[3].cluster_size == cluster
            check(out, ref, inst.cm)


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _check_golden(out, gold):
    assign, delta, loads, st, (tc, td) = out
    assert delta == gold["delta"]
    assert sha(assign.astype(np.int32)) == gold["assign_sha256"]
    assert sha(loads.astype(np.int64)) == gold["load_sha256"]
    for f in ("cycles_applied", "paths_applied", "moves"):
        assert getattr(st, f) == gold["stats"][f], f
    assert sha(tc.astype(np.int32)) == gold["table_tc_sha256"]
    assert sha(td.astype(np.int32)) == gold["table_td_sha256"]


@pytest.mark.parametrize("cluster", [16, 8])
def test_wide_prefix_global_slice_matches_golden(gpu_lib, cluster):
    """20,000 x 2,000 with tight capacity: the owned cost slice cannot sit in
    shared memory at 8 or 16 CTAs, and the 1,000-round prefix applies cycles
    and paths (stored oracle result)."""
    gold = _golden("wide_r1000_oracle.json")
    assert gold["stats"]["moves"] > 0 and gold["stats"]["paths_applied"] > 0
    inst = L.make_named("wide", dtype="i16")
    assert (inst.n, inst.k, inst.recipe.seed) == (gold["n"], gold["k"], gold["seed"])
    out = solve(gpu_lib, inst, cluster, rounds=gold["rounds"])
    assert out[3].cost_slice_in_smem == 0 and out[3].cluster_size == cluster
    _check_golden(out, gold)


def test_large_prefix_with_refinements_matches_golden(gpu_lib):
    """2,000,000 x 2,000 (CM 8 GB as int16), first 9,000 rounds: the first
    overloaded center appears at round 8,325, and the paths applied after it
    run on the global-memory slice path of a 16-CTA cluster."""
    gold = _golden("large_r9000_oracle.json")
    assert gold["stats"]["moves"] > 0 and gold["stats"]["paths_applied"] > 0
    inst = L.make_named("large", dtype="i16")
    assert (inst.n, inst.k, inst.recipe.seed) == (gold["n"], gold["k"], gold["seed"])
    out = solve(gpu_lib, inst, 0, rounds=gold["rounds"])
    assert out[3].cost_slice_in_smem == 0 and out[3].cluster_size == 16
    _check_golden(out, gold)
