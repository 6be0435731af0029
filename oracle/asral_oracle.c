/*
 * CPU oracle for ASRAL (Ramnath et al., "Load Balanced Demand Distribution
 * under Overload Penalties", arXiv 2304.06543).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, single-threaded,
 * deliberately slow statement of what the GPU solver must compute.  It shares
 * no code, header or table with the CUDA path; only tests/, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.
 *
 * Everything is integer.  CM entries are positive integers (Table 1, Def. of
 * the cost matrix), capacities positive integers.  The penalty function of a
 * center (Def. 4) returns the extra cost of the j-th allotment beyond
 * capacity, q_s(j) > 0, non-decreasing in j.  It is given as a table of Q
 * values per center, q_s(j) = qtab[s*Q + min(j, Q) - 1] (the last value
 * repeats); Q = 1 is the constant per-unit form of the experiments
 * (Section 5), where pen[s] is the table.
 *
 * Readings where the paper is silent or loose:
 *  - "ties are broken arbitrarily" (Defs. 9 and 10): the best-transfer edge
 *    u->v is the lexicographic minimum of (transfer cost, demand index);
 *  - "most suitable" center (Section 3.1): lowest index among the minima;
 *    MinDistance heap order: (CM(d, s_min(d)), d) ascending;
 *  - Bellman-Ford (Sections 3.3/3.4, Alg. 3): synchronous sweeps over all
 *    nodes, a label changes only on strict improvement, the parent is the
 *    lowest-index predecessor achieving the new label, stop at the first
 *    sweep with no change; a change at sweep N (N = node count) means a
 *    negative cycle, i.e. a broken Lemma 1/2, reported as an error;
 *  - Def. 9 (d) "all other edges have 0 cost" adds no edge: the only pair it
 *    could concern that matters is anchor-out -> anchor-in, the empty cycle,
 *    whose cost 0 is rejected by the "< 0" test of Alg. 1;
 *  - the objective updates inside Alg. 1 and Alg. 4 (the in-loop comment and
 *    the extra "cost of last edge" update of Alg. 4): the objective changes by the
 *    path cost exactly once (transfer edges CM(new) - CM(old), plus the
 *    penalty edge for a negative path);
 *  - Def. 10 (c): q_u() is the penalty one more unit would pay at u, i.e.
 *    q_u(load_u - c_u + 1) when u is at or above capacity, else 0; q_{s*}()
 *    is the penalty the anchor's last unit beyond capacity paid,
 *    q_{s*}(load - c) (s* is over capacity whenever Alg. 4 runs).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_OOM (-2)
#define OR_ERR_INVARIANT (-5)

#define OR_INF ((int64_t)1 << 62) /* "no edge" / unreached */
#define OR_DUMMY_UNIT INT32_MAX    /* id of a dummy (zero-cost) unit, Appendix B */

enum { MODE_DEFINITION = 0, MODE_HEAP = 1 };

typedef struct {
    int64_t rounds;
    int64_t cycles_applied;
    int64_t paths_applied;
    int64_t bf_calls;
    int64_t bf_sweeps;
    int64_t bf_max_sweeps;
    int64_t moves;
} oracle_stats;

/* q_s(j), j >= 1: penalty of the j-th allotment beyond capacity (Def. 4). */
static int64_t q_of(const int32_t *qtab, int64_t Q, int64_t s, int64_t j) {
    return qtab[s * Q + (j < Q ? j : Q) - 1];
}

/* ------------------------------------------------------------------------
 * Objective, Eq. (1): sum of CM over the allotment plus the total penalty,
 * center s paying q_s(1) + ... + q_s(load - cap) when load > cap.
 * Units with assign[d] < 0 are not allotted and contribute nothing.
 */
int64_t oracle_objective_q(int64_t n, int64_t k, const int32_t *cm, const int32_t *cap,
                           const int32_t *qtab, int64_t Q, const int32_t *assign) {
    int64_t total = 0;
    int64_t *load = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    if (!load) return INT64_MIN;
    for (int64_t d = 0; d < n; ++d) {
        int32_t a = assign[d];
        if (a < 0) continue;
        total += cm[d * k + a];
        load[a] += 1;
    }
    for (int64_t s = 0; s < k; ++s)
        for (int64_t j = 1; j <= load[s] - cap[s]; ++j) total += q_of(qtab, Q, s, j);
    free(load);
    return total;
}

int64_t oracle_objective(int64_t n, int64_t k, const int32_t *cm, const int32_t *cap,
                         const int32_t *pen, const int32_t *assign) {
    return oracle_objective_q(n, k, cm, cap, pen, 1, assign);
}

/* ------------------------------------------------------------------------
 * Alg. 2, first step (and Section 3.1): the "most suitable" center of every unit
 * (lowest index among the minima of its CM row), and the MinDistance heap's
 * extraction order, realised as a sort of (CM(d, s_min), d) ascending.
 */
typedef struct { int64_t cost; int32_t d; } order_key;

static int order_cmp(const void *a, const void *b) {
    const order_key *x = (const order_key *)a, *y = (const order_key *)b;
    if (x->cost != y->cost) return x->cost < y->cost ? -1 : 1;
    return (x->d > y->d) - (x->d < y->d);
}

int oracle_smin_order(int64_t n, int64_t k, const int32_t *cm, int32_t *smin, int32_t *order) {
    if (n < 1 || k < 1 || !cm || !smin || !order) return OR_ERR_ARG;
    order_key *keys = (order_key *)malloc(sizeof(order_key) * (size_t)n);
    if (!keys) return OR_ERR_OOM;
    for (int64_t d = 0; d < n; ++d) {
        int32_t best = 0;
        for (int64_t s = 1; s < k; ++s)
            if (cm[d * k + s] < cm[d * k + best]) best = (int32_t)s;
        smin[d] = best;
        keys[d].cost = cm[d * k + best];
        keys[d].d = (int32_t)d;
    }
    qsort(keys, (size_t)n, sizeof(order_key), order_cmp);
    for (int64_t i = 0; i < n; ++i) order[i] = keys[i].d;
    free(keys);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Best-transfer table by definition (Def. 8 with the min taken per ordered
 * pair as in Defs. 9/10 (a)): for every ordered pair (u, v), u != v, the
 * lexicographically smallest (CM(d,v) - CM(d,u), d) over the units d
 * allotted to u.  tc = OR_INF and td = -1 when u has no unit.
 */
int oracle_best_transfer(int64_t n, int64_t k, const int32_t *cm, const int32_t *assign,
                         int64_t *tc, int32_t *td) {
    if (n < 1 || k < 1 || !cm || !assign || !tc || !td) return OR_ERR_ARG;
    for (int64_t i = 0; i < k * k; ++i) { tc[i] = OR_INF; td[i] = -1; }
    for (int64_t d = 0; d < n; ++d) {
        int32_t u = assign[d];
        if (u < 0) continue;
        for (int64_t v = 0; v < k; ++v) {
            if (v == u) continue;
            int64_t t = (int64_t)cm[d * k + v] - (int64_t)cm[d * k + u];
            int64_t idx = (int64_t)u * k + v;
            if (t < tc[idx] || (t == tc[idx] && (int32_t)d < td[idx])) {
                tc[idx] = t;
                td[idx] = (int32_t)d;
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Bellman-Ford label-correcting shortest paths (Sections 3.3/3.4; Alg. 3 is
 * the same relaxation with the sweep run on a GPU).  Synchronous form: each
 * sweep computes every label from the previous sweep's labels.
 *   W: N x N, W[u*N+v] = edge cost or OR_INF for "no edge".
 * Returns OR_OK, or OR_ERR_INVARIANT if sweep N still changes a label
 * (a negative cycle is reachable from src).
 */
int oracle_bf(int64_t N, int64_t src, const int64_t *W, int64_t *dist, int32_t *par,
              int64_t *sweeps_out) {
    if (N < 1 || src < 0 || src >= N || !W || !dist || !par) return OR_ERR_ARG;
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!prev) return OR_ERR_OOM;
    for (int64_t v = 0; v < N; ++v) { dist[v] = OR_INF; par[v] = -1; }
    dist[src] = 0;
    int64_t sweeps = 0;
    int rc = OR_OK;
    for (int64_t t = 1;; ++t) {
        memcpy(prev, dist, sizeof(int64_t) * (size_t)N);
        int changed = 0;
        for (int64_t v = 0; v < N; ++v) {
            if (v == src) continue;
            int64_t best = OR_INF;
            int32_t bu = -1;
            for (int64_t u = 0; u < N; ++u) {
                if (prev[u] >= OR_INF) continue;
                int64_t w = W[u * N + v];
                if (w >= OR_INF) continue;
                int64_t c = prev[u] + w;
                if (c < best) { best = c; bu = (int32_t)u; }
            }
            if (best < prev[v]) {
                dist[v] = best;
                par[v] = bu;
                changed = 1;
            }
        }
        sweeps = t;
        if (!changed) break;
        if (t >= N) { rc = OR_ERR_INVARIANT; break; }
    }
    free(prev);
    if (sweeps_out) *sweeps_out = sweeps;
    return rc;
}

/* ------------------------------------------------------------------------
 * BestTransHeap (Section 3.4, "Allotment subspace multi-graph
 * implementation"): one min-heap per ordered pair of centers, keyed on
 * (transfer cost, unit).  Removal is lazy: an entry (u, v, d) is live only
 * while d is still allotted to u.  A unit that leaves u and later returns
 * re-validates its old entries, which is harmless because the key depends
 * only on (d, u, v).
 */
typedef struct {
    uint64_t *a;
    int64_t size, cap;
} heap64;

static uint64_t pack_key(int64_t cost, int32_t d) {
    /* costs are differences of int32 CM entries: they fit in 33 bits */
    return ((uint64_t)(cost + ((int64_t)1 << 32)) << 31) | (uint64_t)(uint32_t)d;
}
static int64_t key_cost(uint64_t key) { return (int64_t)(key >> 31) - ((int64_t)1 << 32); }
static int32_t key_unit(uint64_t key) { return (int32_t)(key & 0x7FFFFFFFull); }

static int heap_push(heap64 *h, uint64_t key) {
    if (h->size == h->cap) {
        int64_t nc = h->cap ? h->cap * 2 : 8;
        uint64_t *na = (uint64_t *)realloc(h->a, sizeof(uint64_t) * (size_t)nc);
        if (!na) return OR_ERR_OOM;
        h->a = na;
        h->cap = nc;
    }
    int64_t i = h->size++;
    h->a[i] = key;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p] <= h->a[i]) break;
        uint64_t t = h->a[p]; h->a[p] = h->a[i]; h->a[i] = t;
        i = p;
    }
    return OR_OK;
}

static void heap_pop(heap64 *h) {
    h->a[0] = h->a[--h->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->size && h->a[l] < h->a[m]) m = l;
        if (r < h->size && h->a[r] < h->a[m]) m = r;
        if (m == i) break;
        uint64_t t = h->a[m]; h->a[m] = h->a[i]; h->a[i] = t;
        i = m;
    }
}

/* ------------------------------------------------------------------------
 * Solver state shared by the two ways of obtaining the best-transfer table.
 */
typedef struct {
    int64_t n, k;
    const int32_t *cm, *cap, *qtab;
    int64_t Q;
    int mode;
    int32_t *assign;
    int64_t *load;
    int64_t delta;
    int64_t *tc;      /* k x k snapshot of the best-transfer table */
    int32_t *td;
    heap64 *heaps;    /* MODE_HEAP: k x k (diagonal unused) */
    int64_t *W;       /* (k+1) x (k+1) graph for Bellman-Ford */
    int64_t *dist;
    int32_t *par;
    int32_t *path;    /* node list, source first */
    int32_t *units;   /* unit moved along each path edge */
    int32_t *dests;
    oracle_stats st;
} asral;

/* Push the k-1 transfer edges of unit d, now allotted to center a (the
 * "Update Gamma DS" steps of Alg. 2, Alg. 1 and Alg. 4). */
static int heap_add_unit(asral *S, int32_t d, int32_t a) {
    for (int64_t v = 0; v < S->k; ++v) {
        if (v == a) continue;
        int64_t t = (int64_t)S->cm[(int64_t)d * S->k + v] - (int64_t)S->cm[(int64_t)d * S->k + a];
        int rc = heap_push(&S->heaps[(int64_t)a * S->k + v], pack_key(t, d));
        if (rc) return rc;
    }
    return OR_OK;
}

/* Snapshot of the best-transfer table: the tops of the heaps (MODE_HEAP) or
 * the definition recomputed from the allotment (MODE_DEFINITION). */
static int refresh_table(asral *S) {
    if (S->mode == MODE_DEFINITION)
        return oracle_best_transfer(S->n, S->k, S->cm, S->assign, S->tc, S->td);
    int64_t k = S->k;
    for (int64_t u = 0; u < k; ++u) {
        for (int64_t v = 0; v < k; ++v) {
            int64_t idx = u * k + v;
            S->tc[idx] = OR_INF;
            S->td[idx] = -1;
            if (u == v) continue;
            heap64 *h = &S->heaps[idx];
            while (h->size > 0 && S->assign[key_unit(h->a[0])] != (int32_t)u) heap_pop(h);
            if (h->size > 0) {
                S->tc[idx] = key_cost(h->a[0]);
                S->td[idx] = key_unit(h->a[0]);
            }
        }
    }
    return OR_OK;
}

/* NegCycle graph NCyc(Gamma(A), j), Def. 9.  Node u < k is center u; the
 * anchor j plays s*out (the source) and node k is s*in (the sink).
 *  (a) u, v not the anchor: best transfer u -> v;
 *  (b) s*out -> v: best transfer j -> v;
 *  (c) u -> s*in: best transfer u -> j;
 * no edge enters s*out or leaves s*in, and there are no self loops. */
static void build_ncyc(asral *S, int32_t j) {
    int64_t k = S->k, N = k + 1;
    for (int64_t i = 0; i < N * N; ++i) S->W[i] = OR_INF;
    for (int64_t u = 0; u < k; ++u) {
        for (int64_t v = 0; v < k; ++v) {
            if (u == v || v == j) continue;
            S->W[u * N + v] = S->tc[u * k + v];
        }
        if (u != j) S->W[u * N + k] = S->tc[u * k + j];
    }
}

/* NegPath graph NPath(Gamma(B3), j), Def. 10.  Transfer edges as in (a)/(b);
 * (c) u -> s*in costs q_u() - q_{s*}(): the penalty of one more unit at u
 * (q_u(load_u - c_u + 1) if u is at or above capacity, else 0) minus the
 * penalty saved at the overloaded anchor, q_j(load_j - c_j), the penalty of
 * its last unit beyond capacity; (d) self loops cost 0 and are omitted
 * because a 0-cost loop never shortens a path. */
static void build_npath(asral *S, int32_t j) {
    int64_t k = S->k, N = k + 1;
    for (int64_t i = 0; i < N * N; ++i) S->W[i] = OR_INF;
    for (int64_t u = 0; u < k; ++u) {
        for (int64_t v = 0; v < k; ++v) {
            if (u == v || v == j) continue;
            S->W[u * N + v] = S->tc[u * k + v];
        }
        if (u != j) {
            int64_t qu = S->load[u] >= S->cap[u]
                             ? q_of(S->qtab, S->Q, u, S->load[u] - S->cap[u] + 1) : 0;
            S->W[u * N + k] = qu - q_of(S->qtab, S->Q, j, S->load[j] - S->cap[j]);
        }
    }
}

/* Follow parents from the sink back to the source; returns the number of
 * edges, or -1 if the walk exceeds N edges (broken parent structure). */
static int64_t extract_path(asral *S, int32_t src) {
    int64_t N = S->k + 1;
    int64_t len = 0;
    int32_t v = (int32_t)S->k;
    /* collect sink .. source into path[], then reverse */
    while (v != src) {
        if (len > N || v < 0) return -1;
        S->path[len++] = v;
        v = S->par[v];
    }
    S->path[len] = src;
    for (int64_t a = 0, b = len; a < b; ++a, --b) {
        int32_t t = S->path[a]; S->path[a] = S->path[b]; S->path[b] = t;
    }
    return len; /* path[0] = src, path[len] = sink */
}

/* Apply the transfers of a path (the "cost < 0" branch of Alg. 1 and Alg. 4).  All
 * moved units are read from the table snapshot before any move.  For NCyc
 * the edge into the sink moves a unit into the anchor j; for NPath that edge
 * is the penalty edge and moves nothing.  Returns the terminal center of a
 * negative path (the tail of the penalty edge). */
static int apply_path(asral *S, int64_t len, int32_t j, int is_npath, int32_t *terminal) {
    int64_t k = S->k;
    int64_t m = 0;
    for (int64_t i = 0; i < len; ++i) {
        int32_t u = S->path[i], v = S->path[i + 1];
        if (v == (int32_t)k) {
            if (is_npath) { *terminal = u; break; }
            v = j;
        }
        S->units[m] = S->td[(int64_t)u * k + v];
        S->dests[m] = v;
        if (S->units[m] < 0) return OR_ERR_INVARIANT;
        ++m;
    }
    for (int64_t i = 0; i < m; ++i) {
        int32_t d = S->units[i];
        S->assign[d] = S->dests[i];
        if (S->mode == MODE_HEAP) {
            int rc = heap_add_unit(S, d, S->dests[i]);
            if (rc) return rc;
        }
    }
    S->st.moves += m;
    return OR_OK;
}

/* Alg. 1 (Negative Cycle Refinement) with anchor j. */
static int negcycle_refine(asral *S, int32_t j) {
    int rc = refresh_table(S);
    if (rc) return rc;
    build_ncyc(S, j);
    int64_t sw = 0;
    rc = oracle_bf(S->k + 1, j, S->W, S->dist, S->par, &sw);
    S->st.bf_calls++;
    S->st.bf_sweeps += sw;
    if (sw > S->st.bf_max_sweeps) S->st.bf_max_sweeps = sw;
    if (rc) return rc;
    int64_t cost = S->dist[S->k];
    if (cost < 0 && cost < OR_INF) {
        int64_t len = extract_path(S, j);
        if (len < 0) return OR_ERR_INVARIANT;
        int32_t term = -1;
        rc = apply_path(S, len, j, 0, &term);
        if (rc) return rc;
        S->delta += cost;
        S->st.cycles_applied++;
    }
    return OR_OK;
}

/* Alg. 4 (Negative Path Refinement) with the overloaded anchor j. */
static int negpath_refine(asral *S, int32_t j) {
    int rc = refresh_table(S);
    if (rc) return rc;
    build_npath(S, j);
    int64_t sw = 0;
    rc = oracle_bf(S->k + 1, j, S->W, S->dist, S->par, &sw);
    S->st.bf_calls++;
    S->st.bf_sweeps += sw;
    if (sw > S->st.bf_max_sweeps) S->st.bf_max_sweeps = sw;
    if (rc) return rc;
    int64_t cost = S->dist[S->k];
    if (cost < 0) {
        int64_t len = extract_path(S, j);
        if (len < 0) return OR_ERR_INVARIANT;
        int32_t term = -1;
        rc = apply_path(S, len, j, 1, &term);
        if (rc) return rc;
        if (term < 0) return OR_ERR_INVARIANT;
        S->load[j] -= 1;    /* the overload leaves the anchor ... */
        S->load[term] += 1; /* ... and lands on the path's last center */
        S->delta += cost;
        S->st.paths_applied++;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Negative-cycle test on the min-edge graph of Gamma (Lemmas 1 and 2 state
 * that none exists after each refinement).  Synchronous Bellman-Ford from a
 * virtual source joined to every node at cost 0; a label that still changes
 * at sweep k proves a negative cycle.  Returns 1 if one exists, 0 if not.
 */
int oracle_has_negative_cycle(int64_t k, const int64_t *tc) {
    int64_t *d = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int64_t *p = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    if (!d || !p) { free(d); free(p); return -1; }
    int neg = 0;
    for (int64_t t = 1; t <= k; ++t) {
        memcpy(p, d, sizeof(int64_t) * (size_t)k);
        int changed = 0;
        for (int64_t v = 0; v < k; ++v) {
            for (int64_t u = 0; u < k; ++u) {
                if (u == v || tc[u * k + v] >= OR_INF) continue;
                int64_t c = p[u] + tc[u * k + v];
                if (c < d[v]) { d[v] = c; changed = 1; }
            }
        }
        if (!changed) break;
        if (t == k) neg = 1;
    }
    free(d); free(p);
    return neg;
}

static int asral_init(asral *S, int64_t n, int64_t k, const int32_t *cm, const int32_t *cap,
                      const int32_t *qtab, int64_t Q, int mode, int32_t *assign) {
    memset(S, 0, sizeof(*S));
    S->n = n; S->k = k; S->cm = cm; S->cap = cap; S->qtab = qtab; S->Q = Q; S->mode = mode;
    S->assign = assign;
    int64_t N = k + 1;
    S->load = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    S->tc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k * k));
    S->td = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k * k));
    S->W = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N * N));
    S->dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    S->par = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    S->path = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 2));
    S->units = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 2));
    S->dests = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 2));
    if (mode == MODE_HEAP) S->heaps = (heap64 *)calloc((size_t)(k * k), sizeof(heap64));
    if (!S->load || !S->tc || !S->td || !S->W || !S->dist || !S->par || !S->path ||
        !S->units || !S->dests || (mode == MODE_HEAP && !S->heaps))
        return OR_ERR_OOM;
    for (int64_t d = 0; d < n; ++d) assign[d] = -1;
    return OR_OK;
}

static void asral_free(asral *S) {
    if (S->heaps) {
        for (int64_t i = 0; i < S->k * S->k; ++i) free(S->heaps[i].a);
        free(S->heaps);
    }
    free(S->load); free(S->tc); free(S->td); free(S->W); free(S->dist); free(S->par);
    free(S->path); free(S->units); free(S->dests);
}

/* ------------------------------------------------------------------------
 * Alg. 2 (ASRAL).  Runs `max_rounds` rounds (or all n if max_rounds < 0) of:
 * extract the next unit from the MinDistance order, allot it to its most
 * suitable center j (paying q_j(load - c + 1) if j had no vacancy), Negative Cycle
 * Refinement at j, and, if the allotment overloaded j, Negative Path
 * Refinement at j.
 *   mode: 0 = best-transfer table recomputed by definition every time,
 *         1 = maintained with the paper's BestTransHeaps.
 *   check: if nonzero, after every round verify Lemmas 1/2 (no negative
 *          cycle in Gamma) and the incremental objective against Eq. (1).
 *   order_in: the extraction order of the units (a permutation of 0..n-1),
 *          or NULL for the MinDistance order.  Inserting demand units into
 *          a solved instance (the dynamic update of the paper's proof
 *          sketch: "identical to one iteration of the loop" of Alg. 2) is
 *          this loop with the inserted units extracted after all others,
 *          in insertion order.
 * Outputs assign[n] (-1 = not yet allotted), load[k], *delta, *stats.
 */
int oracle_asral_order(int64_t n, int64_t k, const int32_t *cm, const int32_t *cap,
                       const int32_t *qtab, int64_t Q, int mode, int64_t max_rounds, int check,
                       const int32_t *order_in, int32_t *assign, int64_t *load_out,
                       int64_t *delta_out, oracle_stats *stats) {
    if (n < 1 || k < 1 || Q < 1 || !cm || !cap || !qtab || !assign) return OR_ERR_ARG;
    for (int64_t s = 0; s < k; ++s) {
        if (cap[s] < 1) return OR_ERR_ARG;
        for (int64_t j = 0; j < Q; ++j)   /* positive and non-decreasing (Def. 4) */
            if (qtab[s * Q + j] < 1 || (j > 0 && qtab[s * Q + j] < qtab[s * Q + j - 1]))
                return OR_ERR_ARG;
    }
    for (int64_t i = 0; i < n * k; ++i)
        if (cm[i] < 1) return OR_ERR_ARG;
    asral S;
    int rc = asral_init(&S, n, k, cm, cap, qtab, Q, mode, assign);
    int32_t *smin = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (rc == OR_OK && (!smin || !order)) rc = OR_ERR_OOM;
    if (rc == OR_OK) rc = oracle_smin_order(n, k, cm, smin, order);
    if (rc == OR_OK && order_in) {   /* a permutation of the units */
        char *seen = (char *)calloc((size_t)n, 1);
        if (!seen) rc = OR_ERR_OOM;
        for (int64_t r = 0; r < n && rc == OR_OK; ++r) {
            if (order_in[r] < 0 || order_in[r] >= n || seen[order_in[r]]) rc = OR_ERR_ARG;
            else { seen[order_in[r]] = 1; order[r] = order_in[r]; }
        }
        free(seen);
    }
    int64_t R = (max_rounds < 0 || max_rounds > n) ? n : max_rounds;
    for (int64_t r = 0; r < R && rc == OR_OK; ++r) {
        int32_t d = order[r];
        int32_t j = smin[d];
        int over = S.load[j] >= cap[j]; /* no vacancy at j */
        int64_t q = over ? q_of(qtab, Q, j, S.load[j] - cap[j] + 1) : 0;
        assign[d] = j;
        S.load[j] += 1;
        S.delta += (int64_t)cm[(int64_t)d * k + j] + q;
        if (mode == MODE_HEAP) rc = heap_add_unit(&S, d, j);
        if (rc == OR_OK) rc = negcycle_refine(&S, j);
        if (rc == OR_OK && over) rc = negpath_refine(&S, j);
        S.st.rounds = r + 1;
        if (rc == OR_OK && check) {
            rc = oracle_best_transfer(n, k, cm, assign, S.tc, S.td);
            if (rc == OR_OK && oracle_has_negative_cycle(k, S.tc) != 0) rc = OR_ERR_INVARIANT;
            if (rc == OR_OK && oracle_objective_q(n, k, cm, cap, qtab, Q, assign) != S.delta)
                rc = OR_ERR_INVARIANT;
        }
    }
    if (load_out)
        for (int64_t s = 0; s < k; ++s) load_out[s] = S.load[s];
    if (delta_out) *delta_out = S.delta;
    if (stats) *stats = S.st;
    free(smin);
    free(order);
    asral_free(&S);
    return rc;
}

/* Alg. 2 in the MinDistance order. */
int oracle_asral_q(int64_t n, int64_t k, const int32_t *cm, const int32_t *cap,
                   const int32_t *qtab, int64_t Q, int mode, int64_t max_rounds, int check,
                   int32_t *assign, int64_t *load_out, int64_t *delta_out, oracle_stats *stats) {
    return oracle_asral_order(n, k, cm, cap, qtab, Q, mode, max_rounds, check, NULL, assign,
                              load_out, delta_out, stats);
}

/* Alg. 2 with the constant per-unit penalty pen[s] of the experiments. */
int oracle_asral(int64_t n, int64_t k, const int32_t *cm, const int32_t *cap,
                 const int32_t *pen, int mode, int64_t max_rounds, int check, int32_t *assign,
                 int64_t *load_out, int64_t *delta_out, oracle_stats *stats) {
    if (!pen) return OR_ERR_ARG;
    return oracle_asral_q(n, k, cm, cap, pen, 1, mode, max_rounds, check, assign, load_out,
                          delta_out, stats);
}

/* ------------------------------------------------------------------------
 * Appendix B, Alg. 5 (strict-LBDD): no overload allowed.  If total capacity
 * is below n, a dummy center k with capacity n - sum(cap) and cost max+1 for
 * every unit absorbs the excess.  Every center starts full of dummy units of
 * zero cost, so a center holding p dummies has a 0-cost transfer edge to
 * every other center.  Units are visited in index order (the "unvisited"
 * reading of the loop condition); each replaces a dummy at the cheapest
 * center that still holds one (lowest index on ties), then Alg. 1 runs at
 * that center.  Dummy units sort after real units on equal transfer cost.
 * Outputs assign[n] over the extended center set (k means the dummy center)
 * and the extended objective (dummy center cost included).
 */
int oracle_strict(int64_t n, int64_t k, const int32_t *cm, const int32_t *cap, int32_t *assign,
                  int64_t *cost_out, oracle_stats *stats) {
    if (n < 1 || k < 1 || !cm || !cap || !assign) return OR_ERR_ARG;
    int64_t capsum = 0, mx = 0;
    for (int64_t s = 0; s < k; ++s) capsum += cap[s];
    for (int64_t i = 0; i < n * k; ++i) if (cm[i] > mx) mx = cm[i];
    int64_t K = capsum < n ? k + 1 : k;
    int64_t N = K + 1;
    int32_t *cmx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * K));
    int64_t *dummies = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *tc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K * K));
    int32_t *td = (int32_t *)malloc(sizeof(int32_t) * (size_t)(K * K));
    int64_t *W = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N * N));
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 2));
    int32_t *mv_u = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 2));
    int32_t *mv_from = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 2));
    int32_t *mv_to = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 2));
    int rc = OR_OK;
    if (!cmx || !dummies || !tc || !td || !W || !dist || !par || !path || !mv_u || !mv_from ||
        !mv_to)
        rc = OR_ERR_OOM;
    oracle_stats st;
    memset(&st, 0, sizeof(st));
    if (rc == OR_OK) {
        for (int64_t d = 0; d < n; ++d) {
            for (int64_t s = 0; s < k; ++s) cmx[d * K + s] = cm[d * k + s];
            if (K > k) cmx[d * K + k] = (int32_t)(mx + 1);
            assign[d] = -1;
        }
        for (int64_t s = 0; s < k; ++s) dummies[s] = cap[s];
        if (K > k) dummies[k] = n - capsum;
    }
    for (int64_t d = 0; d < n && rc == OR_OK; ++d) {
        int32_t j = -1;
        for (int64_t s = 0; s < K; ++s)
            if (dummies[s] > 0 && (j < 0 || cmx[d * K + s] < cmx[d * K + j])) j = (int32_t)s;
        if (j < 0) { rc = OR_ERR_INVARIANT; break; }
        dummies[j] -= 1;
        assign[d] = j;
        /* best-transfer table over real units plus dummy edges */
        oracle_best_transfer(n, K, cmx, assign, tc, td);
        for (int64_t u = 0; u < K; ++u) {
            if (dummies[u] <= 0) continue;
            for (int64_t v = 0; v < K; ++v) {
                if (u == v) continue;
                int64_t idx = u * K + v;
                if (0 < tc[idx]) { tc[idx] = 0; td[idx] = OR_DUMMY_UNIT; }
            }
        }
        /* Def. 9 graph and Alg. 1 at anchor j */
        for (int64_t i = 0; i < N * N; ++i) W[i] = OR_INF;
        for (int64_t u = 0; u < K; ++u) {
            for (int64_t v = 0; v < K; ++v) {
                if (u == v || v == j) continue;
                W[u * N + v] = tc[u * K + v];
            }
            if (u != j) W[u * N + K] = tc[u * K + j];
        }
        int64_t sw = 0;
        rc = oracle_bf(N, j, W, dist, par, &sw);
        st.bf_calls++;
        st.bf_sweeps += sw;
        if (rc) break;
        if (dist[K] < 0) {
            int64_t len = 0;
            int32_t v = (int32_t)K;
            while (v != j) {
                if (len > N || v < 0) { rc = OR_ERR_INVARIANT; break; }
                path[len++] = v;
                v = par[v];
            }
            if (rc) break;
            path[len] = j;
            for (int64_t a = 0, b = len; a < b; ++a, --b) {
                int32_t t = path[a]; path[a] = path[b]; path[b] = t;
            }
            int64_t m = 0;
            for (int64_t i = 0; i < len; ++i) {
                int32_t u = path[i], w = path[i + 1];
                if (w == (int32_t)K) w = j;
                mv_u[m] = td[(int64_t)u * K + w];
                mv_from[m] = u;
                mv_to[m] = w;
                ++m;
            }
            for (int64_t i = 0; i < m; ++i) {
                if (mv_u[i] == OR_DUMMY_UNIT) {
                    dummies[mv_from[i]] -= 1;
                    dummies[mv_to[i]] += 1;
                } else {
                    assign[mv_u[i]] = mv_to[i];
                }
            }
            st.moves += m;
            st.cycles_applied++;
        }
        st.rounds = d + 1;
    }
    if (rc == OR_OK && cost_out) {
        int64_t c = 0;
        for (int64_t d = 0; d < n; ++d) c += cmx[d * K + assign[d]];
        *cost_out = c;
    }
    if (stats) *stats = st;
    free(cmx); free(dummies); free(tc); free(td); free(W); free(dist); free(par); free(path);
    free(mv_u); free(mv_from); free(mv_to);
    return rc;
}

/* ------------------------------------------------------------------------
 * Cost matrix from a road network (Section 3.4 "Demand-service cost matrix
 * construction", Section 5 "Datasets"): CM(d, s) is the shortest-path length
 * from center node centers[s] to demand node demand[d] over the directed
 * graph (row_ptr, col, w) with positive integer lengths.  Plain Dijkstra
 * with a binary heap, one source at a time.  Returns OR_ERR_ARG for a bad
 * graph or an unreachable demand node.
 */
typedef struct { int64_t key; int32_t v; } dj_item;

static void dj_push(dj_item *h, int64_t *len, int64_t key, int32_t v) {
    int64_t i = (*len)++;
    h[i].key = key; h[i].v = v;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].key <= h[i].key) break;
        dj_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static dj_item dj_pop(dj_item *h, int64_t *len) {
    dj_item top = h[0];
    h[0] = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *len && h[l].key < h[m].key) m = l;
        if (r < *len && h[r].key < h[m].key) m = r;
        if (m == i) break;
        dj_item t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

int oracle_road_cm(int64_t V, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                   int64_t k, const int32_t *centers, int64_t n, const int32_t *demand,
                   int32_t *cm_out) {
    if (V < 1 || k < 1 || n < 1 || !row_ptr || !col || !w || !centers || !demand || !cm_out)
        return OR_ERR_ARG;
    int64_t E = row_ptr[V];
    for (int64_t e = 0; e < E; ++e)
        if (w[e] < 1 || col[e] < 0 || col[e] >= V) return OR_ERR_ARG;
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    dj_item *heap = (dj_item *)malloc(sizeof(dj_item) * (size_t)(E + 1));
    if (!dist || !heap) { free(dist); free(heap); return OR_ERR_OOM; }
    int rc = OR_OK;
    for (int64_t s = 0; s < k && rc == OR_OK; ++s) {
        if (centers[s] < 0 || centers[s] >= V) { rc = OR_ERR_ARG; break; }
        for (int64_t v = 0; v < V; ++v) dist[v] = OR_INF;
        int64_t len = 0;
        dist[centers[s]] = 0;
        dj_push(heap, &len, 0, centers[s]);
        while (len > 0) {
            dj_item it = dj_pop(heap, &len);
            if (it.key > dist[it.v]) continue;   /* stale entry */
            for (int32_t e = row_ptr[it.v]; e < row_ptr[it.v + 1]; ++e) {
                int64_t nd = it.key + w[e];
                if (nd < dist[col[e]]) {
                    dist[col[e]] = nd;
                    dj_push(heap, &len, nd, col[e]);
                }
            }
        }
        for (int64_t d = 0; d < n; ++d) {
            int32_t v = demand[d];
            if (v < 0 || v >= V || dist[v] >= OR_INF || dist[v] < 1 || dist[v] > INT32_MAX) {
                rc = OR_ERR_ARG;
                break;
            }
            cm_out[d * k + s] = (int32_t)dist[v];
        }
    }
    free(dist);
    free(heap);
    return rc;
}
