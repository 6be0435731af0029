"""GPU parity of demand-unit insertion (lbdd_insert) with the CPU oracle.

The paper's proof sketch of its dynamic-update theorem: adding a demand unit
is one more iteration of the loop of Alg. 2.  The oracle runs that loop with
the inserted units extracted after the solved ones, in insertion order
(oracle.insertion_order), and is pinned to the exact optimum after every
insert.  Here the solver is created with the first n0 units, solved, then
given the remaining units one by one through the C ABI; the allotment, the
tracked objective (Eq. 1), the loads and the best-transfer table must equal
the oracle's bit for bit, across several growths of the device arrays.
"""
import numpy as np
import pytest

import lbdd_inputs as L
import oracle

pytestmark = pytest.mark.gpu

TINF = 2**31 - 1


def check(s, ref, cm):
    assert s.objective == ref.delta
    assert np.array_equal(s.assignment(), ref.assign)
    assert np.array_equal(s.loads().astype(np.int64), ref.load)
    tc, td = s.table()
    rtc, rtd = oracle.best_transfer(cm, ref.assign)
    assert np.array_equal(tc, np.where(rtc >= oracle.INF, TINF, rtc))
    assert np.array_equal(td, rtd)


@pytest.mark.parametrize("cluster", [1, 2, 4, 16])
def test_insert_one_by_one_after_a_solve(gpu_lib, cluster):
    """100 units solved, 400 inserted (several growths of the arrays and the
    page pool), a solve after each insert; the state equals the oracle's
    after every 50 inserts and at the end."""
    J = L.random_small(8100 + cluster, n=500, k=24, cm_max=40, cap_frac=0.6, pen=(5, 60))
    n0 = 100
    order = oracle.insertion_order(J.cm, n0)
    with gpu_lib.Solver(J.cm[:n0], J.cap, J.pen, cluster=cluster) as s:
        s.solve()
        for d in range(n0, J.n):
            assert s.insert(J.cm[d]) == d
            s.solve()
            if (d + 1) % 50 == 0 or d + 1 == J.n:
                ref = oracle.asral(J.cm[:d + 1], J.cap, J.pen, order=order[:d + 1])
                assert ref.rc == 0
                check(s, ref, J.cm[:d + 1])
        assert s.rounds == J.n and s.stats().moves > 0


def test_inserts_then_one_solve_and_int16_rows(gpu_lib):
    """Several units inserted before one solve are extracted in insertion
    order; rows may come as int16."""
    J = L.random_small(8200, n=300, k=40, cm_max=25, cap_frac=0.5, pen=(1, 30))
    n0 = 120
    with gpu_lib.Solver(J.cm[:n0], J.cap, J.pen) as s:
        s.solve()
        for d in range(n0, J.n):
            s.insert(J.cm[d].astype(np.int16) if d % 2 else J.cm[d])
        s.solve()
        ref = oracle.asral(J.cm, J.cap, J.pen, order=oracle.insertion_order(J.cm, n0))
        check(s, ref, J.cm)


def test_insert_before_the_first_round_and_reset(gpu_lib):
    """Units inserted before any round join the instance (the first solve
    orders all units); lbdd_reset re-solves all units in the MinDistance
    order."""
    J = L.random_small(8300, n=400, k=30, cm_max=30, cap_frac=0.7, pen=(1, 40))
    ref = oracle.asral(J.cm, J.cap, J.pen)
    with gpu_lib.Solver(J.cm[:150], J.cap, J.pen) as s:
        for d in range(150, J.n):
            s.insert(J.cm[d])
        s.solve()
        check(s, ref, J.cm)
    with gpu_lib.Solver(J.cm[:150], J.cap, J.pen) as s:
        s.solve()
        for d in range(150, J.n):
            s.insert(J.cm[d])
        s.solve()
        s.reset()
        s.solve()
        check(s, ref, J.cm)


def test_insert_into_int32_and_penalty_table_solvers(gpu_lib):
    J = L.random_small(8400, n=260, k=20, cm_max=90000, cap_frac=0.5, pen=(100, 5000))
    order = oracle.insertion_order(J.cm, 60)
    with gpu_lib.Solver(J.cm[:60], J.cap, J.pen, cluster=4) as s:
        assert s.stats().cm_elem_bytes == 4
        s.solve()
        for d in range(60, J.n):
            s.insert(J.cm[d])
            if d % 3 == 0:
                s.solve()
        s.solve()
        check(s, oracle.asral(J.cm, J.cap, J.pen, order=order), J.cm)
    J = L.random_small(8401, n=240, k=16, cm_max=30, cap_frac=0.4, pen=(1, 9))
    qtab = L.penalty_table(8401, 16, 4, base=(1, 12), step=(0, 9))
    order = oracle.insertion_order(J.cm, 80)
    ref = oracle.asral_q(J.cm, J.cap, qtab, order=order)
    with gpu_lib.Solver(J.cm[:80], J.cap, J.pen, qtab=qtab) as s:
        s.solve()
        for d in range(80, J.n):
            s.insert(J.cm[d])
        s.solve()
        assert s.objective == ref.delta and np.array_equal(s.assignment(), ref.assign)


def test_insert_refusals(gpu_lib):
    J = L.random_small(8500, n=50, k=6, cm_max=9)
    with gpu_lib.Solver(J.cm, J.cap, J.pen) as s:       # stored as int16
        s.solve()
        for bad in (np.full(6, 40000, np.int32), np.array([1, 2, 0, 4, 5, 6], np.int32)):
            with pytest.raises(gpu_lib.LbddError) as e:
                s.insert(bad)
            assert e.value.code == gpu_lib.ERR_ARG
        with pytest.raises(ValueError):
            s.insert(np.ones(5, np.int32))
        b = gpu_lib.Batch([s])
        with pytest.raises(gpu_lib.LbddError) as e:
            gpu_lib.insert(s.h, np.ones(6, np.int32), 6)
        assert e.value.code == gpu_lib.ERR_STATE
        b.close()
        assert s.insert(np.ones(6, np.int32)) == 50     # allowed again once the batch is gone
    with gpu_lib.Solver(J.cm, J.cap, J.pen, strict=True) as s:
        with pytest.raises(gpu_lib.LbddError) as e:
            gpu_lib.insert(s.h, np.ones(s.k, np.int32), s.k)
        assert e.value.code == gpu_lib.ERR_STATE
