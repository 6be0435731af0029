"""GPU parity of strict-LBDD (Appendix B, Alg. 5) against the oracle, and
its optimality (Theorem 2) against the exact assignment optimum."""
import numpy as np
import pytest

import lbdd_inputs as L
import oracle
from oracle import exact

pytestmark = pytest.mark.gpu


def solve_strict(lb, inst, cluster=0, ncyc_skip=True):
    with lb.Solver(inst.cm, inst.cap, None, strict=True, cluster=cluster,
                   ncyc_skip=ncyc_skip) as s:
        s.solve()
        return s.assignment(), s.objective, s.loads(), s.stats()


@pytest.mark.parametrize("seed", range(16))
def test_strict_random_small(gpu_lib, seed):
    n = [20, 60, 150, 300][seed % 4]
    k = [2, 3, 7, 12, 30][seed % 5]
    inst = L.random_small(9100 + seed, n=n, k=k, cm_max=[4, 15, 60][seed % 3],
                          cap_frac=[0.5, 0.9, 1.4][(seed // 2) % 3])
    rc, ref_assign, ref_cost, ref_st = oracle.strict(inst.cm, inst.cap)
    assert rc == 0
    for cluster in (1, 2) if k >= 4 else (1,):
        for skip in (True, False):
            a, obj, loads, st = solve_strict(gpu_lib, inst, cluster, skip)
            assert obj == ref_cost
            assert np.array_equal(a, ref_assign)
            assert st.cycles_applied == ref_st["cycles_applied"]
            assert st.moves == ref_st["moves"]
            # capacities are never exceeded
            K = len(loads)
            capx = list(inst.cap) + ([n - int(np.sum(inst.cap))] if K > k else [])
            assert np.all(loads <= np.asarray(capx))
            assert np.array_equal(np.bincount(a, minlength=K), loads)


@pytest.mark.parametrize("seed", range(6))
def test_strict_is_optimal(gpu_lib, seed):
    """Theorem 2: Alg. 5 reaches the minimum over capacity-respecting
    allotments (min-cost assignment on slot-expanded centers)."""
    inst = L.random_small(9300 + seed, n=[12, 40, 90][seed % 3], k=[3, 5][seed % 2], cm_max=30,
                          cap_frac=[0.6, 1.2][seed % 2])
    a, obj, _, _ = solve_strict(gpu_lib, inst)
    assert obj == exact.strict_optimum(inst.cm, inst.cap)


def test_strict_tiny_named(gpu_lib):
    inst = L.make_named("tiny")
    rc, ref_assign, ref_cost, _ = oracle.strict(inst.cm, inst.cap)
    assert rc == 0
    a, obj, _, _ = solve_strict(gpu_lib, inst)
    assert obj == ref_cost and np.array_equal(a, ref_assign)
