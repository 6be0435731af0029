"""Exact LBDD solvers used to pin the oracle (test infrastructure only).

These do not run ASRAL.  They solve the problem statement of Section 2.1
exactly on tiny instances so that the heuristic's objective can be bounded
from below:

* :func:`brute_force` enumerates all k**n complete allotments and evaluates
  Eq. (1) directly.
* :func:`matching_optimum` is the paper's reduction to min-cost bipartite
  matching (Section 1 "Challenges"; Section 5 "Min-Cost Bipartite
  Matching"): every center s is expanded into cap_s ordinary slots costing
  CM(d, s) and n overload slots costing CM(d, s) + pen_s, and the rectangular
  assignment problem is solved with scipy's ``linear_sum_assignment``.
* :func:`eq1_objective_q`, :func:`brute_force_q` and
  :func:`matching_optimum_q` are the same with a general penalty function
  (Def. 4) given as a table: q_s(j) = qtab[s][min(j, Q) - 1] is the extra
  cost of the j-th allotment beyond capacity.  In the matching, the j-th
  overload slot of s costs CM(d, s) + q_s(j); since q_s is non-decreasing
  an optimal matching never skips a cheaper overload slot of a center.
* :func:`strict_optimum` is the same reduction for strict-LBDD (Appendix B):
  only the cap_s ordinary slots, plus the dummy center's n - sum(cap) slots
  at max(CM) + 1 when demand exceeds capacity.
"""
from __future__ import annotations

import itertools

import numpy as np


def eq1_objective(cm, cap, pen, assign) -> int:
    """Eq. (1) with a constant per-unit penalty, in plain Python."""
    cm = np.asarray(cm)
    k = cm.shape[1]
    load = [0] * k
    total = 0
    for d, s in enumerate(assign):
        if s < 0:
            continue
        total += int(cm[d, s])
        load[s] += 1
    for s in range(k):
        total += int(pen[s]) * max(0, load[s] - int(cap[s]))
    return total


def q_value(qtab, s, j) -> int:
    row = qtab[s]
    return int(row[min(j, len(row)) - 1])


def eq1_objective_q(cm, cap, qtab, assign) -> int:
    """Eq. (1) with penalty tables, in plain Python."""
    cm = np.asarray(cm)
    k = cm.shape[1]
    load = [0] * k
    total = 0
    for d, s in enumerate(assign):
        if s < 0:
            continue
        total += int(cm[d, s])
        load[s] += 1
    for s in range(k):
        for j in range(1, load[s] - int(cap[s]) + 1):
            total += q_value(qtab, s, j)
    return total


def brute_force_q(cm, cap, qtab):
    cm = np.asarray(cm)
    n, k = cm.shape
    assert k ** n <= 20000, "brute force is for tiny instances only"
    return min(eq1_objective_q(cm, cap, qtab, a) for a in itertools.product(range(k), repeat=n))


def matching_optimum_q(cm, cap, qtab) -> int:
    from scipy.optimize import linear_sum_assignment
    cm = np.asarray(cm, dtype=np.int64)
    n, k = cm.shape
    cols = []
    for s in range(k):
        cols += [cm[:, s]] * int(min(cap[s], n))
        cols += [cm[:, s] + q_value(qtab, s, j) for j in range(1, n + 1)]
    C = np.stack(cols, axis=1)
    r, c = linear_sum_assignment(C)
    assert len(r) == n
    return int(C[r, c].sum())


def brute_force(cm, cap, pen):
    """Minimum of Eq. (1) over all k**n allotments (n <= 8, k <= 3)."""
    cm = np.asarray(cm)
    n, k = cm.shape
    assert k ** n <= 20000, "brute force is for tiny instances only"
    best = None
    for a in itertools.product(range(k), repeat=n):
        v = eq1_objective(cm, cap, pen, a)
        if best is None or v < best:
            best = v
    return best


def matching_optimum(cm, cap, pen) -> int:
    from scipy.optimize import linear_sum_assignment
    cm = np.asarray(cm, dtype=np.int64)
    n, k = cm.shape
    cols = []
    for s in range(k):
        cols += [cm[:, s]] * int(min(cap[s], n))
        cols += [cm[:, s] + int(pen[s])] * n
    C = np.stack(cols, axis=1)
    r, c = linear_sum_assignment(C)
    assert len(r) == n
    return int(C[r, c].sum())


def strict_optimum(cm, cap) -> int:
    from scipy.optimize import linear_sum_assignment
    cm = np.asarray(cm, dtype=np.int64)
    n, k = cm.shape
    capsum = int(np.sum(cap))
    cols = []
    for s in range(k):
        cols += [cm[:, s]] * int(min(cap[s], n))
    if capsum < n:
        cols += [np.full(n, int(cm.max()) + 1, dtype=np.int64)] * (n - capsum)
    C = np.stack(cols, axis=1)
    r, c = linear_sum_assignment(C)
    assert len(r) == n
    return int(C[r, c].sum())
