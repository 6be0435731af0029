"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each check is an exact
solver (brute force, the paper's min-cost-matching reduction), a closed
form, a library routine (scipy Bellman-Ford / negative-cycle detection), a
theorem of the paper (Lemmas 1-2, Theorem 2), or an independent data
structure (the BestTransHeaps vs. the table recomputed by definition).
The last test plants typical mistakes in a copy of the oracle and checks that
at least one pin fails for each.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import lbdd_inputs as L
import oracle
from oracle import exact


def small(seed, n, k, **kw):
    return L.random_small(seed, n=n, k=k, **kw)


# ---------------------------------------------------------------- exact ---

def test_brute_force_equals_matching_reduction():
    """The min-cost-matching reduction (Section 1) solves Eq. (1) exactly."""
    for s in range(25):
        J = small(100 + s, 7, 3, cm_max=9, cap_frac=0.5, pen=(1, 6))
        assert exact.brute_force(J.cm, J.cap, J.pen) == exact.matching_optimum(J.cm, J.cap, J.pen)


@pytest.mark.parametrize("mode", [oracle.MODE_DEFINITION, oracle.MODE_HEAP])
def test_asral_never_below_optimum_and_reaches_it(mode):
    """ASRAL's objective is a feasible value, so never below the optimum.
    With constant per-unit penalties every refinement is a shortest
    augmenting path of a convex-cost flow, and on all seeded instances here
    the value equals the optimum; a dropped term, a sign or index slip in the
    graphs of Defs. 9/10 breaks the equality."""
    for s in range(40):
        n = [8, 20, 45][s % 3]
        k = [2, 3, 5, 7][s % 4]
        J = small(300 + s, n, k, cm_max=[4, 15, 60][s % 3], cap_frac=[0.3, 0.6, 0.95][s % 3],
                  pen=[(1, 5), (1, 40), (10, 100)][(s // 3) % 3])
        r = oracle.asral(J.cm, J.cap, J.pen, mode=mode, check=True)
        assert r.rc == oracle.OK
        opt = exact.matching_optimum(J.cm, J.cap, J.pen)
        assert r.delta >= opt
        assert r.delta == opt, (s, r.delta, opt)


def test_brute_force_bound_on_tiny():
    for s in range(20):
        J = small(700 + s, 8, 3, cm_max=6, cap_frac=0.5, pen=(1, 4))
        r = oracle.asral(J.cm, J.cap, J.pen)
        assert r.rc == 0 and r.delta >= exact.brute_force(J.cm, J.cap, J.pen)


# ----------------------------------------------------------- invariants ---

def test_incremental_objective_equals_eq1_and_allotment_complete():
    inst = L.make_named("tiny")
    r = oracle.asral(inst.cm, inst.cap, inst.pen)
    assert r.rc == 0
    assert (r.assign >= 0).all() and (r.assign < inst.k).all()      # each unit once
    assert np.array_equal(np.bincount(r.assign, minlength=inst.k), r.load)
    assert r.delta == exact.eq1_objective(inst.cm, inst.cap, inst.pen, r.assign)
    assert r.delta == oracle.objective(inst.cm, inst.cap, inst.pen, r.assign)


def test_lemmas_hold_every_round():
    """Lemmas 1 and 2: Gamma has no negative cycle after every round (the
    oracle's check mode runs the test after each round and also compares
    the tracked objective with Eq. (1))."""
    for s in range(30):
        J = small(900 + s, 30, 5, cm_max=25, cap_frac=0.5, pen=(1, 30))
        assert oracle.asral(J.cm, J.cap, J.pen, check=True).rc == oracle.OK
    inst = L.make(L.Recipe(n=400, k=12, seed=17, scale=100.0, cap_frac=0.8, pen=(20, 200)))
    assert oracle.asral(inst.cm, inst.cap, inst.pen, check=True).rc == oracle.OK


def test_heap_mode_equals_definition_mode():
    """BestTransHeaps (Section 3.4) and the table by definition agree."""
    for s in range(15):
        J = small(1200 + s, 60, 6, cm_max=8, cap_frac=0.6, pen=(1, 9))   # many ties
        a = oracle.asral(J.cm, J.cap, J.pen, mode=oracle.MODE_DEFINITION)
        b = oracle.asral(J.cm, J.cap, J.pen, mode=oracle.MODE_HEAP)
        assert a.rc == b.rc == 0
        assert np.array_equal(a.assign, b.assign) and a.delta == b.delta
        assert a.stats == b.stats
    inst = L.make_named("tiny")
    a = oracle.asral(inst.cm, inst.cap, inst.pen, mode=oracle.MODE_DEFINITION)
    b = oracle.asral(inst.cm, inst.cap, inst.pen, mode=oracle.MODE_HEAP)
    assert np.array_equal(a.assign, b.assign) and a.delta == b.delta


def test_truncated_rounds_are_a_prefix():
    inst = L.make_named("tiny")
    full = oracle.asral(inst.cm, inst.cap, inst.pen)
    part = oracle.asral(inst.cm, inst.cap, inst.pen, max_rounds=700)
    assert part.stats["rounds"] == 700
    assert (part.assign >= 0).sum() == 700
    assert part.delta == oracle.objective(inst.cm, inst.cap, inst.pen, part.assign)
    assert full.delta != part.delta


# --------------------------------------------------------- closed forms ---

def test_ample_capacity_gives_row_minima():
    """cap_s >= n for all s: nothing is ever overloaded, every unit sits at a
    row minimum and Delta = sum_d min_s CM(d, s)."""
    for s in range(10):
        J = small(1500 + s, 50, 6, cm_max=30)
        cap = np.full(J.k, J.n, np.int32)
        r = oracle.asral(J.cm, cap, J.pen)
        assert r.rc == 0 and r.delta == int(J.cm.min(axis=1).sum())
        assert r.stats["moves"] == 0


def test_single_center_closed_form():
    for s in range(5):
        J = small(1600 + s, 40, 1, cm_max=30)
        cap, pen = np.array([13], np.int32), np.array([7], np.int32)
        r = oracle.asral(J.cm, cap, pen)
        assert r.delta == int(J.cm.sum()) + 7 * (40 - 13)


def test_smin_and_order_definition():
    """Alg. 2, first step: lowest-index row minimum; order (cost, d) ascending,
    checked against numpy's argmin (first occurrence) and lexsort."""
    J = small(1700, 500, 9, cm_max=5)
    smin, order = oracle.smin_order(J.cm)
    assert np.array_equal(smin, np.argmin(J.cm, axis=1))
    cost = J.cm[np.arange(J.n), smin]
    assert np.array_equal(order, np.lexsort((np.arange(J.n), cost)))


# ---------------------------------------------------- best transfers -----

def _best_transfer_certificate(cm, assign, tc, td):
    """The facts that fix the table of Defs. 8-10 uniquely, checked as a
    certificate rather than recomputed: every finite entry (u, v) names a
    unit d allotted to u whose transfer cost CM(d, v) - CM(d, u) is the
    entry (attained), no unit of u transfers to v for less (minimal), no unit
    of u with a lower index transfers for the same cost (lowest d on ties);
    a center without units, and the diagonal, have no entries."""
    k = cm.shape[1]
    cm = cm.astype(np.int64)
    for u in range(k):
        members = np.nonzero(assign == u)[0]
        for v in range(k):
            if u == v or len(members) == 0:
                assert tc[u, v] >= oracle.INF and td[u, v] == -1
                continue
            d = int(td[u, v])
            assert assign[d] == u and tc[u, v] == cm[d, v] - cm[d, u]
            t = cm[members, v] - cm[members, u]
            assert (t >= tc[u, v]).all()
            assert not (members[t == tc[u, v]] < d).any()


@pytest.mark.parametrize("seed", range(4))
def test_best_transfer_table_certificate(seed):
    J = small(1750 + seed, [60, 200, 31, 120][seed], [4, 9, 13, 6][seed],
              cm_max=[3, 20, 7, 50][seed])
    rng = np.random.default_rng(seed)
    assign = rng.integers(-1, J.k, J.n).astype(np.int32)     # -1: not allotted yet
    assign[assign == 1] = 0                                  # center 1 holds nothing
    tc, td = oracle.best_transfer(J.cm, assign)
    _best_transfer_certificate(J.cm, assign, tc, td)


def test_best_transfer_certificate_rejects_plausible_mistakes():
    """The certificate fails for a transposed table, a flipped sign and the
    highest instead of the lowest d on ties."""
    J = small(1760, 150, 7, cm_max=4)
    assign = np.argmin(J.cm, axis=1).astype(np.int32)
    tc, td = oracle.best_transfer(J.cm, assign)
    _best_transfer_certificate(J.cm, assign, tc, td)
    cm = J.cm.astype(np.int64)
    k = J.k
    flipped = tc.copy()
    fin = td >= 0
    u, v = np.nonzero(fin)
    flipped[u, v] = cm[td[u, v], u] - cm[td[u, v], v]
    last = td.copy()
    for a in range(k):
        members = np.nonzero(assign == a)[0]
        for b in range(k):
            if a != b and len(members):
                t = cm[members, b] - cm[members, a]
                last[a, b] = members[np.nonzero(t == t.min())[0][-1]]
    for bad_tc, bad_td in ((tc.T.copy(), td.T.copy()), (flipped, td), (tc, last)):
        with pytest.raises(AssertionError):
            _best_transfer_certificate(J.cm, assign, bad_tc, bad_td)


def test_best_transfer_at_smin_is_nonnegative():
    """With every unit at its most suitable center (Alg. 2, first step), no
    transfer lowers a unit's cost: every finite entry is >= 0, and a 0
    entry means a tie between the two centers' costs."""
    J = small(1770, 400, 11, cm_max=6)
    smin, _ = oracle.smin_order(J.cm)
    tc, td = oracle.best_transfer(J.cm, smin)
    fin = td >= 0
    assert (tc[fin] >= 0).all() and (tc[fin] == 0).any()


# ------------------------------------------------------- Bellman-Ford -----

def _random_potential_graph(rng, N, density):
    W = np.full((N, N), oracle.INF, np.int64)
    pot = rng.integers(0, 30, N)
    for u in range(N):
        for v in range(N):
            if u != v and rng.random() < density:
                W[u, v] = int(rng.integers(0, 6)) + pot[v] - pot[u]   # no negative cycle
    return W


def test_bellman_ford_matches_scipy_and_paths_are_tight():
    import scipy.sparse as sp
    from scipy.sparse.csgraph import bellman_ford
    rng = np.random.default_rng(1)
    for t in range(60):
        N = int(rng.integers(2, 12))
        W = _random_potential_graph(rng, N, 0.5)
        src = int(rng.integers(0, N))
        rc, dist, par, sweeps = oracle.bellman_ford(W, src)
        assert rc == 0 and sweeps <= N
        mask = W < oracle.INF
        G = sp.csr_matrix((W[mask].astype(float), np.nonzero(mask)), shape=(N, N))
        ref = bellman_ford(G, indices=src)
        for v in range(N):
            if np.isinf(ref[v]):
                assert dist[v] >= oracle.INF and par[v] == -1
            else:
                assert dist[v] == ref[v]
                if v != src:   # parent edge is tight, parent is lowest such index
                    u = par[v]
                    assert dist[u] + W[u, v] == dist[v]


def _canonical_parent_violations(bf, trials=80, seed=11):
    """Count graphs where `bf`'s parent differs from the closed form: hop(v),
    the sweep of v's last change, is the fewest edges among shortest paths to
    v (levels of a breadth-first search over the tight edges
    dist[u] + W[u][v] = dist[v], distances from scipy), and par[v] is the
    lowest u with a tight edge and hop(u) = hop(v) - 1."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import bellman_ford
    rng = np.random.default_rng(seed)
    bad = 0
    for t in range(trials):
        N = int(rng.integers(3, 14))
        W = _random_potential_graph(rng, N, [0.3, 0.6, 0.9][t % 3])
        src = int(rng.integers(0, N))
        rc, dist, par = bf(W, src)
        if rc != 0:              # no negative cycle here: any error is a violation
            bad += 1
            continue
        mask = W < oracle.INF
        G = sp.csr_matrix((W[mask].astype(float), np.nonzero(mask)), shape=(N, N))
        ref = bellman_ford(G, indices=src)
        reach = ~np.isinf(ref)
        d = np.where(reach, ref, 0).astype(np.int64)
        tight = mask & reach[:, None] & reach[None, :] & \
            (d[:, None] + np.where(mask, W, 0) == d[None, :])
        hop = np.full(N, -1)
        hop[src] = 0
        level = [src]
        while level:
            nxt = []
            for u in level:
                for v in np.nonzero(tight[u])[0]:
                    if hop[v] < 0:
                        hop[v] = hop[u] + 1
                        nxt.append(int(v))
            level = nxt
        for v in range(N):
            if v != src and reach[v]:
                cands = [u for u in range(N) if tight[u, v] and hop[u] == hop[v] - 1]
                if par[v] != min(cands):
                    bad += 1
                    break
    return bad


def test_bellman_ford_parent_is_the_canonical_closed_form():
    """Zero-cost edges of the random graphs make many ties."""
    def bf(W, src):
        rc, dist, par, _ = oracle.bellman_ford(W, src)
        return rc, dist, par
    assert _canonical_parent_violations(bf) == 0


BF_MUTATIONS = {
    "highest_predecessor_on_ties": ("if (c < best) { best = c; bu = (int32_t)u; }",
                                    "if (c <= best) { best = c; bu = (int32_t)u; }"),
    "update_on_equal_label": ("if (best < prev[v]) {", "if (best <= prev[v] && best < OR_INF) {"),
    "in_place_sweep": ("int64_t c = prev[u] + w;", "int64_t c = (dist[u] < prev[u] ? dist[u] : prev[u]) + w;"),
}


@pytest.mark.parametrize("name", sorted(BF_MUTATIONS))
def test_planted_bellman_ford_mistake_is_caught(name, tmp_path):
    """Tie and sweep-order mistakes planted in a copy of the oracle's
    Bellman-Ford break the canonical parents (or, updating on equal labels,
    never converge)."""
    old, new = BF_MUTATIONS[name]
    src_text = open(_SRC).read()
    assert src_text.count(old) == 1, name
    mutated = tmp_path / "mut.c"
    mutated.write_text(src_text.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", str(mutated), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    P, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.oracle_bf.argtypes = [i64, i64, P, P, P, P]

    def bf(W, src):
        W = np.ascontiguousarray(W, np.int64)
        N = W.shape[0]
        dist = np.empty(N, np.int64)
        par = np.empty(N, np.int32)
        rc = lib.oracle_bf(N, src, W.ctypes.data, dist.ctypes.data, par.ctypes.data, None)
        return rc, dist, par
    assert _canonical_parent_violations(bf) > 0


def test_bellman_ford_reports_negative_cycle():
    W = np.full((4, 4), oracle.INF, np.int64)
    W[0, 1], W[1, 2], W[2, 1], W[2, 3] = 1, -3, 1, 0
    rc, *_ = oracle.bellman_ford(W, 0)
    assert rc == oracle.ERR_INVARIANT


def test_negative_cycle_checker_matches_scipy():
    import scipy.sparse as sp
    from scipy.sparse.csgraph import NegativeCycleError, bellman_ford
    rng = np.random.default_rng(2)
    for t in range(80):
        k = int(rng.integers(2, 8))
        tc = np.where(rng.random((k, k)) < 0.6, rng.integers(-6, 10, (k, k)), oracle.INF)
        np.fill_diagonal(tc, oracle.INF)
        mask = tc < oracle.INF
        G = sp.csr_matrix((tc[mask].astype(float), np.nonzero(mask)), shape=(k, k))
        try:
            bellman_ford(G)
            ref = False
        except NegativeCycleError:
            ref = True
        assert oracle.has_negative_cycle(tc) == ref


# -------------------------------------------------------- strict-LBDD -----

def test_strict_lbdd_is_optimal():
    """Theorem 2 + Alg. 5: the NegCycle-only variant with dummy units is
    optimal for hard capacities; checked against the assignment reduction,
    with and without excess demand."""
    for s in range(30):
        n, k = [10, 30, 60][s % 3], [2, 4, 6][s % 3]
        J = small(1800 + s, n, k, cm_max=[6, 25, 40][s % 3], cap_frac=[0.6, 1.0, 1.4][s % 3])
        rc, assign, cost, st = oracle.strict(J.cm, J.cap)
        assert rc == 0
        assert cost == exact.strict_optimum(J.cm, J.cap)
        k_ext = k + (1 if J.cap.sum() < n else 0)
        load = np.bincount(assign, minlength=k_ext)
        assert (load[:k] <= J.cap).all()


# ------------------------------------------------------ planted mistakes --

_SRC = os.path.join(os.path.dirname(oracle.__file__), "asral_oracle.c")

MUTATIONS = {
    "dropped_penalty_term": ("int64_t q = over ? q_of(qtab, Q, j, S.load[j] - cap[j] + 1) : 0;",
                             "int64_t q = 0;"),
    "transfer_sign": ("int64_t t = (int64_t)cm[d * k + v] - (int64_t)cm[d * k + u];",
                      "int64_t t = (int64_t)cm[d * k + u] - (int64_t)cm[d * k + v];"),
    "penalty_edge_sign": ("S->W[u * N + k] = qu - q_of(S->qtab, S->Q, j, S->load[j] - S->cap[j]);",
                          "S->W[u * N + k] = q_of(S->qtab, S->Q, j, S->load[j] - S->cap[j]) - qu;"),
    "transposed_sink_edge": ("if (u != j) S->W[u * N + k] = S->tc[u * k + j];",
                             "if (u != j) S->W[u * N + k] = S->tc[j * k + u];"),
    "wrong_vacancy_test": ("int over = S.load[j] >= cap[j];", "int over = S.load[j] > cap[j];"),
    "terminal_load_not_moved": ("S->load[term] += 1;", "S->load[j] += 0;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(_SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", str(mutated), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    P, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.oracle_asral.argtypes = [i64, i64, P, P, P, c_int, i64, c_int, P, P, P, P]
    def run(J, mode):
        cm = np.ascontiguousarray(J.cm, np.int32)
        assign = np.empty(J.n, np.int32)
        load = np.empty(J.k, np.int64)
        delta = ctypes.c_int64(0)
        st = oracle._Stats()
        rc = lib.oracle_asral(J.n, J.k, cm.ctypes.data, J.cap.ctypes.data, J.pen.ctypes.data,
                              mode, -1, 0, assign.ctypes.data, load.ctypes.data,
                              ctypes.byref(delta), ctypes.byref(st))
        return rc, assign, load, delta.value

    caught = False
    for s in range(12):
        J = small(2100 + s, 24, 4, cm_max=20, cap_frac=0.5, pen=(1, 25))
        opt = exact.matching_optimum(J.cm, J.cap, J.pen)
        results = [run(J, mode) for mode in (oracle.MODE_DEFINITION, oracle.MODE_HEAP)]
        for rc, assign, load, delta in results:
            if rc != 0 or delta != opt or \
                    delta != exact.eq1_objective(J.cm, J.cap, J.pen, assign) or \
                    not np.array_equal(np.bincount(assign, minlength=J.k), load):
                caught = True
        if results[0][3] != results[1][3] or not np.array_equal(results[0][1], results[1][1]):
            caught = True
        if caught:
            break
    assert caught, f"mutation {name} escaped every pin"


# ------------------------------------------- general penalty functions --

def _qinst(seed, n, k, Q, **kw):
    J = small(seed, n, k, **kw)
    return J, L.penalty_table(seed, k, Q, base=(1, 12), step=(0, 9))


def test_penalty_table_brute_force_equals_matching_reduction():
    """The slot reduction with the j-th overload slot at CM + q_s(j) solves
    Eq. (1) exactly for non-decreasing q (Def. 4)."""
    for s in range(20):
        J, q = _qinst(3100 + s, 7, 3, 4, cm_max=9, cap_frac=0.4)
        assert exact.brute_force_q(J.cm, J.cap, q) == exact.matching_optimum_q(J.cm, J.cap, q)


@pytest.mark.parametrize("mode", [oracle.MODE_DEFINITION, oracle.MODE_HEAP])
def test_asral_with_penalty_tables_against_optimum(mode):
    """ASRAL with increasing penalties: a feasible value (never below the
    optimum), the incremental objective equals Eq. (1) and Lemmas 1/2 hold
    every round (check mode), and the value equals the optimum on every
    seeded instance here (the penalties are convex)."""
    for s in range(30):
        n = [10, 24, 50][s % 3]
        k = [2, 3, 5][s % 3]
        J, q = _qinst(3300 + s, n, k, [2, 5, 9][s % 3], cm_max=[6, 25][s % 2],
                      cap_frac=[0.3, 0.6][s % 2])
        r = oracle.asral_q(J.cm, J.cap, q, mode=mode, check=True)
        assert r.rc == oracle.OK
        assert r.delta == exact.eq1_objective_q(J.cm, J.cap, q, r.assign)
        opt = exact.matching_optimum_q(J.cm, J.cap, q)
        assert r.delta >= opt
        assert r.delta == opt, (s, r.delta, opt)


def test_constant_table_equals_constant_penalty():
    for s in range(8):
        J = small(3500 + s, 40, 4, cm_max=15, cap_frac=0.5, pen=(1, 30))
        q = np.repeat(J.pen[:, None], 3, axis=1)
        a, b = oracle.asral(J.cm, J.cap, J.pen), oracle.asral_q(J.cm, J.cap, q)
        assert a.delta == b.delta and np.array_equal(a.assign, b.assign)


def test_penalty_table_rejects_decreasing_or_nonpositive():
    J = small(3600, 10, 2)
    bad = np.array([[5, 4], [1, 1]], np.int32)
    assert oracle.asral_q(J.cm, J.cap, bad).rc == oracle.ERR_ARG
    assert oracle.asral_q(J.cm, J.cap, np.array([[1, 2], [0, 1]], np.int32)).rc == oracle.ERR_ARG


Q_MUTATIONS = {
    # the allotment pays the penalty of the previous overload unit
    "allot_penalty_index": ("int64_t q = over ? q_of(qtab, Q, j, S.load[j] - cap[j] + 1) : 0;",
                            "int64_t q = over ? q_of(qtab, Q, j, S.load[j] - cap[j] + (S.load[j] > cap[j] ? 0 : 1)) : 0;"),
    # the penalty edge saves the anchor's next unit instead of its last one
    "anchor_penalty_index": ("qu - q_of(S->qtab, S->Q, j, S->load[j] - S->cap[j]);",
                             "qu - q_of(S->qtab, S->Q, j, S->load[j] - S->cap[j] + 1);"),
    # Eq. (1) charges every overload unit the first table value
    "objective_flat_table": ("total += q_of(qtab, Q, s, j);", "total += q_of(qtab, Q, s, 1);"),
}


@pytest.mark.parametrize("name", sorted(Q_MUTATIONS))
def test_planted_penalty_table_mistake_is_caught(name, tmp_path):
    old, new = Q_MUTATIONS[name]
    src = open(_SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", str(mutated), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    P, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.oracle_asral_q.argtypes = [i64, i64, P, P, P, i64, c_int, i64, c_int, P, P, P, P]
    caught = False
    for s in range(12):
        J, q = _qinst(3700 + s, 24, 4, 6, cm_max=20, cap_frac=0.4)
        cm = np.ascontiguousarray(J.cm, np.int32)
        qq = np.ascontiguousarray(q, np.int32)
        assign = np.empty(J.n, np.int32)
        load = np.empty(J.k, np.int64)
        delta = ctypes.c_int64(0)
        st = oracle._Stats()
        rc = lib.oracle_asral_q(J.n, J.k, cm.ctypes.data, J.cap.ctypes.data, qq.ctypes.data,
                                q.shape[1], oracle.MODE_HEAP, -1, 1, assign.ctypes.data,
                                load.ctypes.data, ctypes.byref(delta), ctypes.byref(st))
        opt = exact.matching_optimum_q(J.cm, J.cap, q)
        if rc != 0 or delta.value != opt or \
                delta.value != exact.eq1_objective_q(J.cm, J.cap, q, assign):
            caught = True
            break
    assert caught, f"mutation {name} escaped every pin"


# ------------------------------------------------ road-network cost matrix --

def _grid_csr(W, H, weight=1):
    adj = [[] for _ in range(W * H)]
    for v in range(W * H):
        x, y = v % W, v // W
        for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= x + dx < W and 0 <= y + dy < H:
                adj[v].append(v + dx + dy * W)
    row_ptr = np.zeros(W * H + 1, np.int32)
    for v in range(W * H):
        row_ptr[v + 1] = row_ptr[v] + len(adj[v])
    col = np.array([b for a in adj for b in sorted(a)], np.int32)
    return row_ptr, col, np.full(len(col), weight, np.int32)


def test_road_cm_unit_grid_is_manhattan():
    """On a unit-length grid the shortest path is the Manhattan distance."""
    W, H = 13, 9
    row_ptr, col, w = _grid_csr(W, H, weight=3)
    centers = np.array([0, 17, 60, 116], np.int32)
    demand = np.array([v for v in range(W * H) if v not in set(centers)], np.int32)
    rc, cm = oracle.road_cm(row_ptr, col, w, centers, demand)
    assert rc == 0
    for d, v in enumerate(demand):
        for s, c in enumerate(centers):
            assert cm[d, s] == 3 * (abs(v % W - c % W) + abs(v // W - c // W))


def test_road_cm_equals_scipy_dijkstra():
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    g = L.road_network(11, 24, 17, 6)
    rc, cm = oracle.road_cm(g.row_ptr, g.col, g.w, g.centers, g.demand)
    assert rc == 0
    A = csr_matrix((g.w.astype(np.float64), g.col, g.row_ptr), shape=(g.V, g.V))
    D = dijkstra(A, directed=True, indices=g.centers)
    assert np.array_equal(cm, D[:, g.demand].T.astype(np.int64))


def _csr_min(a, b, wts, V):
    """Directed CSR of the roads a -> b; of parallel roads the shortest is kept."""
    best = {}
    for u, v, c in zip(a.tolist(), b.tolist(), wts.tolist()):
        best[(u, v)] = min(best.get((u, v), c), c)
    keys = sorted(best)
    row_ptr = np.zeros(V + 1, np.int32)
    np.add.at(row_ptr, np.array([u for u, _ in keys]) + 1, 1)
    return (np.cumsum(row_ptr).astype(np.int32), np.array([v for _, v in keys], np.int32),
            np.array([best[x] for x in keys], np.int32))


def test_road_cm_one_way_roads_follow_the_direction():
    """Directed roads: CM[d][s] is the length of the shortest path from
    center s to demand node d (scipy Dijkstra from the centers), in the
    graph as given and with every road reversed."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    rng = np.random.default_rng(7)
    V = 300
    src = np.concatenate([np.arange(V), rng.integers(0, V, 4 * V)])
    dst = np.concatenate([(np.arange(V) + 1) % V, rng.integers(0, V, 4 * V)])   # a ring: connected
    keep = src != dst
    src, dst = src[keep], dst[keep]
    wts = rng.integers(1, 50, len(src))
    centers = np.array([3, 77, 150, 299], np.int32)
    demand = np.setdiff1d(np.arange(V), centers).astype(np.int32)
    cms = []
    for a, b in ((src, dst), (dst, src)):
        row_ptr, col, w = _csr_min(a, b, wts, V)
        rc, cm = oracle.road_cm(row_ptr, col, w, centers, demand)
        assert rc == 0
        D = dijkstra(csr_matrix((w.astype(np.float64), col, row_ptr), shape=(V, V)),
                     directed=True, indices=centers)
        assert np.array_equal(cm, D[:, demand].T.astype(np.int64))
        cms.append(cm)
    assert not np.array_equal(cms[0], cms[1])           # one-way roads: direction matters
    # a demand node on a center's node would cost 0: refused (CM >= 1)
    assert oracle.road_cm(row_ptr, col, w, centers, np.array([3], np.int32))[0] == oracle.ERR_ARG


def test_road_cm_rejects_bad_graph():
    row_ptr, col, w = _grid_csr(4, 4)
    w[3] = 0
    assert oracle.road_cm(row_ptr, col, w, [0], [5])[0] == oracle.ERR_ARG
    # an isolated demand node is unreachable
    row_ptr2 = np.append(row_ptr, row_ptr[-1]).astype(np.int32)
    _, col2, w2 = _grid_csr(4, 4)
    assert oracle.road_cm(row_ptr2, col2, w2, [0], [16])[0] == oracle.ERR_ARG


BT_MUTATIONS = {
    "tie_takes_highest_unit": ("(t == tc[idx] && (int32_t)d < td[idx])",
                               "(t == tc[idx] && (int32_t)d > td[idx])"),
    "diagonal_kept": ("            if (v == u) continue;\n            int64_t t = (int64_t)cm[d * k + v]",
                      "            int64_t t = (int64_t)cm[d * k + v]"),
    "row_of_destination": ("int64_t idx = (int64_t)u * k + v;", "int64_t idx = v * k + u;"),
}


@pytest.mark.parametrize("name", sorted(BT_MUTATIONS))
def test_planted_best_transfer_mistake_is_caught(name, tmp_path):
    """Mistakes planted in a copy of the oracle's best-transfer table fail
    the certificate of Defs. 8-10."""
    old, new = BT_MUTATIONS[name]
    src = open(_SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", str(mutated), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    P, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.oracle_best_transfer.argtypes = [i64, i64, P, P, P, P]
    J = small(1780, 150, 7, cm_max=4)
    assign = np.argmin(J.cm, axis=1).astype(np.int32)
    cm = np.ascontiguousarray(J.cm, np.int32)
    tc = np.empty((J.k, J.k), np.int64)
    td = np.empty((J.k, J.k), np.int32)
    assert lib.oracle_best_transfer(J.n, J.k, cm.ctypes.data, assign.ctypes.data,
                                    tc.ctypes.data, td.ctypes.data) == 0
    with pytest.raises(AssertionError):
        _best_transfer_certificate(J.cm, assign, tc, td)


# ------------------------------------------- insertion of demand units --
# The paper's proof sketch of its dynamic-update theorem: adding a demand
# unit is one more iteration of the loop of Alg. 2.  The oracle runs the loop
# with the inserted units extracted after the solved ones.

def test_insertion_keeps_the_optimum_after_every_insert():
    """After the first n0 units are solved and each later unit inserted, the
    objective is the exact optimum of the units allotted so far (the
    slot-expanded matching of that sub-instance), the rest are unallotted,
    and Lemmas 1/2 and Eq. (1) hold after every round."""
    for s in range(10):
        n, k = [12, 18, 26][s % 3], [2, 3, 5][s % 3]
        J = small(3600 + s, n, k, cm_max=[5, 20, 60][s % 3], cap_frac=[0.4, 0.7, 0.9][s % 3],
                  pen=[(1, 6), (1, 30), (5, 80)][s % 3])
        n0 = n // 2
        order = oracle.insertion_order(J.cm, n0)
        assert np.array_equal(order[n0:], np.arange(n0, n))
        for m in range(n0, n + 1):
            r = oracle.asral(J.cm, J.cap, J.pen, order=order, max_rounds=m, check=True)
            assert r.rc == oracle.OK
            assert (r.assign[m:] == -1).all() and (r.assign[:m] >= 0).all()
            assert r.delta == exact.matching_optimum(J.cm[:m], J.cap, J.pen), (s, m)


def test_insertion_against_brute_force_on_tiny():
    for s in range(12):
        J = small(3700 + s, 8, 3, cm_max=7, cap_frac=0.5, pen=(1, 5))
        r = oracle.asral(J.cm, J.cap, J.pen, order=oracle.insertion_order(J.cm, 3))
        assert r.rc == 0 and r.delta == exact.brute_force(J.cm, J.cap, J.pen)


def test_units_already_last_in_the_order_insert_like_a_solve():
    """Inserting units whose (cost, index) keys already come last in the
    MinDistance order gives exactly the one-shot solve."""
    J = small(3800, 30, 4, cm_max=9, cap_frac=0.6, pen=(1, 20))
    _, order = oracle.smin_order(J.cm)
    last = order[-5:]
    perm = np.concatenate([np.setdiff1d(np.arange(30), last), last]).astype(np.int32)
    cm = J.cm[perm]                       # the five units become the last indices
    ref = oracle.asral(cm, J.cap, J.pen)
    ins = oracle.asral(cm, J.cap, J.pen, order=oracle.insertion_order(cm, 25))
    assert ins.delta == ref.delta and np.array_equal(ins.assign, ref.assign)


def test_order_must_be_a_permutation():
    J = small(3900, 10, 3)
    for bad in ([0] * 10, list(range(1, 11)), [-1] + list(range(1, 10))):
        assert oracle.asral(J.cm, J.cap, J.pen, order=np.array(bad, np.int32)).rc == oracle.ERR_ARG


def test_planted_insertion_mistake_is_caught(tmp_path):
    """An oracle that ignores the given extraction order fails the
    per-insert optimum pin."""
    src = open(_SRC).read()
    old = "else { seen[order_in[r]] = 1; order[r] = order_in[r]; }"
    assert src.count(old) == 1
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, "else { seen[order_in[r]] = 1; }"))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", str(mutated), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    P, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.oracle_asral_order.argtypes = [i64, i64, P, P, P, i64, c_int, i64, c_int, P, P, P, P, P]
    caught = False
    for s in range(10):
        J = small(3600 + s, 18, 3, cm_max=20, cap_frac=0.7, pen=(1, 30))
        order = oracle.insertion_order(J.cm, 9)
        cm = np.ascontiguousarray(J.cm, np.int32)
        assign = np.empty(J.n, np.int32)
        load = np.empty(J.k, np.int64)
        delta = ctypes.c_int64(0)
        st = oracle._Stats()
        rc = lib.oracle_asral_order(J.n, J.k, cm.ctypes.data, J.cap.ctypes.data,
                                    J.pen.ctypes.data, 1, oracle.MODE_HEAP, 9, 0,
                                    order.ctypes.data, assign.ctypes.data, load.ctypes.data,
                                    ctypes.byref(delta), ctypes.byref(st))
        if rc != 0 or (assign[9:] != -1).any() or \
                delta.value != exact.matching_optimum(J.cm[:9], J.cap, J.pen):
            caught = True
            break
    assert caught
