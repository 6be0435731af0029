"""GPU parity with general penalty functions (Def. 4, per-center tables)
against the oracle's Alg. 2 with the same tables."""
import numpy as np
import pytest

import lbdd_inputs as L
import oracle

pytestmark = pytest.mark.gpu


def run(lb, inst, q, cluster=0, ncyc_skip=True, npath_reuse=True):
    with lb.Solver(inst.cm, inst.cap, inst.pen, cluster=cluster, ncyc_skip=ncyc_skip,
                   npath_reuse=npath_reuse, qtab=q) as s:
        s.solve()
        return s.assignment(), s.objective, s.loads()


@pytest.mark.parametrize("seed", range(14))
def test_penalty_tables_random_small(gpu_lib, seed):
    n = [40, 150, 400][seed % 3]
    k = [3, 6, 17, 40][seed % 4]
    Q = [2, 5, 9, 30][seed % 4]
    inst = L.random_small(9500 + seed, n=n, k=k, cm_max=[5, 30, 90][seed % 3],
                          cap_frac=[0.3, 0.6, 0.9][(seed // 2) % 3])
    q = L.penalty_table(9500 + seed, k, Q, base=(1, 40), step=(0, 15))
    ref = oracle.asral_q(inst.cm, inst.cap, q)
    assert ref.rc == 0
    for cluster in (1, 2, 4) if k >= 4 else (1,):
        for skip, reuse in ((True, True), (False, False)):
            a, obj, loads = run(gpu_lib, inst, q, cluster, skip, reuse)
            assert obj == ref.delta
            assert np.array_equal(a, ref.assign)
            assert np.array_equal(loads.astype(np.int64), ref.load)


def test_penalty_table_tiny_named(gpu_lib):
    inst = L.make_named("tiny")
    q = L.penalty_table(1, inst.k, 16, base=(50, 500), step=(0, 60))
    ref = oracle.asral_q(inst.cm, inst.cap, q)
    a, obj, _ = run(gpu_lib, inst, q)
    assert obj == ref.delta and np.array_equal(a, ref.assign)


def test_one_column_table_is_the_constant_penalty(gpu_lib):
    inst = L.make_named("tiny")
    ref = oracle.asral(inst.cm, inst.cap, inst.pen)
    a, obj, _ = run(gpu_lib, inst, inst.pen[:, None])
    assert obj == ref.delta and np.array_equal(a, ref.assign)


def test_penalty_table_rules(gpu_lib):
    inst = L.random_small(9700, n=50, k=4)
    with gpu_lib.Solver(inst.cm, inst.cap, inst.pen) as s:
        with pytest.raises(gpu_lib.LbddError):
            gpu_lib.set_penalty_table(s.h, np.array([[3, 2]] * 4, np.int32))   # decreasing
        s.solve(10)
        with pytest.raises(gpu_lib.LbddError):                                  # rounds already run
            gpu_lib.set_penalty_table(s.h, np.ones((4, 2), np.int32))
        s.reset()
        gpu_lib.set_penalty_table(s.h, np.ones((4, 2), np.int32))
