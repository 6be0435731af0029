/*
 * lbdd.h -- C ABI of the GB300 (sm_103a) ASRAL solver for Load Balanced
 * Demand Distribution (LBDD).
 *
 * Problem (paper Section 2.1, "Problem Statement"): given service centers
 * S = {s_0..s_{k-1}}, demand units D = {d_0..d_{n-1}}, a cost matrix CM
 * (n x k, positive integers, Table 1 and the cost-matrix definition of
 * Section 2), a positive integer capacity c_s per center and a penalty q_s
 * per center (Def. 4; here the constant per-unit form of the paper's
 * experiments, Section 5: every unit beyond c_s costs pen[s]), find a
 * complete allotment minimising Eq. (1):
 *     sum_d CM(d, a(d)) + sum_s pen[s] * max(0, load_s - c_s).
 * The solver runs ASRAL (Alg. 2 with Alg. 1 and Alg. 4) with canonical
 * tie-breaking, so its output is one deterministic allotment that equals the
 * project's CPU oracle bit for bit.
 *
 * Conventions shared by every call:
 *  - Every call returns an lbdd_status code (0 = success); none aborts.
 *  - CM is demand-major: entry (d, s) at index d*k + s.  Pointers flagged
 *    "_is_device" are CUDA device pointers, otherwise host pointers.
 *  - The library copies all inputs into device memory it owns; the caller's
 *    buffers may be freed as soon as lbdd_create returns.
 *  - All work is ordered on the CUDA stream given to lbdd_create (NULL = the
 *    legacy default stream) and every call that produces a result
 *    synchronises that stream before returning.
 *  - An lbdd_solver is not thread-safe; distinct solvers are independent.
 *  - A CUDA failure returns LBDD_ERR_CUDA; lbdd_last_cuda_error() gives the
 *    CUDA error string of the most recent such failure in this process.
 */
#ifndef LBDD_H
#define LBDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbdd_status {
  LBDD_OK = 0,
  LBDD_ERR_ARG = -1,        /* invalid argument (sizes, CM < 1, cap < 1, pen < 1) */
  LBDD_ERR_OOM = -2,        /* device or host allocation failed */
  LBDD_ERR_CUDA = -3,       /* a CUDA runtime call failed */
  LBDD_ERR_TIMEOUT = -4,    /* a bounded wait gave up (server polling, or a solver
                               kernel whose cluster exchange stopped answering) */
  LBDD_ERR_INVARIANT = -5,  /* Lemma 1/2 violated: Bellman-Ford did not converge */
  LBDD_ERR_STATE = -6,      /* call not valid in the object's current state */
  LBDD_ERR_NODEV = -7,      /* no CUDA device of compute capability 10.3 */
  LBDD_ERR_BUDGET = -8      /* server: request larger than the memory budget */
} lbdd_status;

typedef enum lbdd_cm_dtype {
  LBDD_CM_I32 = 0,          /* int32 entries */
  LBDD_CM_I16 = 1           /* int16 entries (exact when every cost < 32768) */
} lbdd_cm_dtype;

typedef struct lbdd_solver lbdd_solver;   /* opaque, owned by the library */

typedef struct lbdd_stats {
  int64_t rounds;           /* rounds of Alg. 2 completed */
  int64_t cycles_applied;   /* negative cycles removed (Alg. 1) */
  int64_t paths_applied;    /* negative paths removed (Alg. 4) */
  int64_t bf_calls;         /* Bellman-Ford runs to convergence */
  int64_t bf_sweeps;        /* synchronous sweeps over all those runs */
  int64_t bf_max_sweeps;    /* longest run, in sweeps */
  int64_t moves;            /* demand units transferred between centers */
  int64_t ncyc_skipped;     /* Alg. 1 calls answered without Bellman-Ford because
                               the new unit lowered no best-transfer cost */
  int64_t rows_scanned;     /* CM rows read by best-transfer segment rescans */
  int64_t cm_elem_bytes;    /* 2 or 4: element size of the stored CM */
  int64_t cluster_size;     /* CTAs per thread-block cluster used by solves */
  /* Device-side phase timers of the cluster's first CTA, nanoseconds summed
     over all launches (tracing aid; phases overlap barriers of other CTAs). */
  int64_t prologue_ns;      /* s_min + MinDistance order + state init */
  int64_t rounds_ns;        /* whole round loop */
  int64_t merge_ns;         /* allotment + merge of the new unit's row */
  int64_t relax_ns;         /* Bellman-Ford relaxation of owned columns */
  int64_t sync_ns;          /* Bellman-Ford cluster barriers */
  int64_t gather_ns;        /* Bellman-Ford exchange of label changes */
  int64_t apply_ns;         /* path application (member lists, loads) */
  int64_t rescan_ns;        /* segment rescans of the best-transfer rows */
  int64_t relax_loop_ns;    /* part of relax_ns: the relaxation loop itself */
  int64_t relax_reduce_ns;  /* part of relax_ns: loop + cross-warp reduction and record */
  int64_t cost_slice_in_smem; /* 1 if the last solve kept each CTA's best-transfer cost
                                 columns in shared memory */
  int64_t npath_reused;     /* Alg. 4 calls answered from the labels of an Alg. 1
                               Bellman-Ford that applied nothing (exact: same graph
                               except for the sink edges) */
  int64_t col_rows;         /* member rows read by column-subset rescans */
  int64_t front_sum;        /* sum over sweeps of the Bellman-Ford frontier size */
  int64_t front_hist[6];    /* sweeps with frontier 1, 2-4, 5-16, 17-64, 65-256, >256 */
} lbdd_stats;

/* Options for lbdd_set_option. */
typedef enum lbdd_option {
  LBDD_OPT_CLUSTER = 1,     /* CTAs per cluster for lbdd_solve: 1, 2, 4, 8 or 16
                               (0 = auto) */
  LBDD_OPT_NCYC_SKIP = 2,   /* 1 (default): skip Alg. 1's Bellman-Ford when the new
                               unit lowers no best-transfer cost (exact by Lemma 1);
                               0: always run it */
  LBDD_OPT_TC_SMEM = 4,     /* 1 (default): keep each CTA's best-transfer cost columns in
                               shared memory when they fit; 0: read them from global memory */
  LBDD_OPT_NPATH_REUSE = 3, /* 1 (default): answer Alg. 4 from the converged labels of
                               an Alg. 1 run that applied nothing; 0: always run a
                               separate Bellman-Ford */
  LBDD_OPT_PHASE_TIMERS = 5,/* 0 (default): only the total time of the rounds is kept;
                               1: also time every phase (the *_ns fields of lbdd_stats
                               and the frontier counters), which slows the rounds */
} lbdd_option;

/* Create a solver for one LBDD instance (Section 2.1 inputs).
 *   n, k        : demand units and service centers, n >= 1,
 *                 1 <= k <= lbdd_max_centers() (5,376; larger k returns
 *                 LBDD_ERR_ARG).
 *   cm          : n*k entries, demand-major, every entry >= 1; dtype per
 *                 cm_dtype; host memory unless cm_is_device != 0.
 *                 int32 input whose maximum is below 32768 is stored as
 *                 int16 (exact, half the bytes per scan).
 *   cap, pen    : k entries each, host memory, cap[s] >= 1, pen[s] >= 1.
 *   cuda_stream : cudaStream_t for all work of this solver, or NULL.
 * On success *out owns device memory of about n*k*elem + 32*n + 8*k*k bytes.
 * Errors: LBDD_ERR_ARG, LBDD_ERR_OOM, LBDD_ERR_CUDA, LBDD_ERR_NODEV; *out
 * is set to NULL on failure. */
int lbdd_create(lbdd_solver** out, int32_t n, int32_t k, const void* cm, int cm_dtype,
                int cm_is_device, const int32_t* cap, const int32_t* pen, void* cuda_stream);

/* The most service centers a solver accepts: every CTA of a 16-CTA cluster
 * keeps per-center label, hop, load, capacity and penalty replicas and a
 * frontier of k + 1 keys in its shared memory (at most 227 KB, of which the
 * kernel's static variables take a little).  A strict-LBDD instance whose
 * capacities sum below n counts its dummy center too.  Host arithmetic; no
 * device needed. */
int32_t lbdd_max_centers(void);

/* Set an lbdd_option; LBDD_ERR_ARG for an unknown option or bad value. */
int lbdd_set_option(lbdd_solver* s, int option, int64_t value);

/* General penalty functions (Def. 4): q_s(j), the extra cost of the j-th
 * allotment beyond center s's capacity, positive and non-decreasing in j.
 * qtab is a host k x Q table, q_s(j) = qtab[s*Q + min(j, Q) - 1] (the last
 * value repeats); it replaces the constant pen[] given to lbdd_create (which
 * is the Q = 1 table).  The allotment of Alg. 2 pays q_j(load - c + 1), the
 * penalty edge of Def. 10 (c) costs q_u(load_u - c_u + 1) (0 with a vacancy)
 * minus q_j(load_j - c_j), and the objective sums q_s(1..load - c).  Call
 * before the first lbdd_solve (or after lbdd_reset).  Errors: LBDD_ERR_ARG
 * (non-positive or decreasing rows, strict solver), LBDD_ERR_STATE (rounds
 * already run). */
int lbdd_set_penalty_table(lbdd_solver* s, const int32_t* qtab, int32_t Q);

/* Create a solver for a strict-LBDD instance (Appendix B, Alg. 5, Theorem 2):
 * no center may exceed its capacity.  If the capacities sum to less than n,
 * a dummy center k is added with capacity n - sum(cap) and cost max(CM) + 1
 * for every unit, so the solver has k + 1 centers and the assignment may use
 * index k.  lbdd_solve then runs Alg. 5: units in index order, each to the
 * cheapest center with a vacancy (lowest index on ties), then Negative Cycle
 * Refinement at that center, where a center with a vacancy can pass a dummy
 * unit on at cost 0 (its transfer costs are min(T, 0)).  The final allotment
 * minimises the cost over capacity-respecting allotments of the extended
 * instance; lbdd_objective returns that cost.  Arguments as lbdd_create,
 * without penalties.  Errors as lbdd_create. */
int lbdd_create_strict(lbdd_solver** out, int32_t n, int32_t k, const void* cm, int cm_dtype,
                       int cm_is_device, const int32_t* cap, void* cuda_stream);

/* Run rounds of Alg. 2 (each: allot the next unit of the MinDistance order
 * to its most suitable center, Negative Cycle Refinement at that center,
 * and Negative Path Refinement if the center was full).  max_rounds < 0
 * runs to completion (n rounds in total); otherwise at most max_rounds more
 * rounds run and a later call resumes exactly where this one stopped.
 * Synchronous on return.  Errors: LBDD_ERR_INVARIANT (Lemma 1/2 broken,
 * the solver is then unusable), LBDD_ERR_CUDA. */
int lbdd_solve(lbdd_solver* s, int64_t max_rounds);

/* Forget all progress: the next lbdd_solve starts again from round 0 on the
 * CM already resident on the device (the prologue of Alg. 2 is redone).
 * Stream-ordered; no host synchronisation. */
int lbdd_reset(lbdd_solver* s);

/* ---------------------------------------------------------------------
 * Batched solves.  Every instance is an independent run of Alg. 2 (the
 * paper solves one instance at a time; batching many is this library's
 * addition), so a batch is a scheduling problem only: which cluster size
 * each instance gets and how the SMs are shared.
 *
 * lbdd_batch_create plans a batch of m solvers (all created on the current
 * device; they stay owned by the caller and must outlive the batch):
 *   - each instance gets a thread-block cluster of C CTAs (1, 2, 4, 8, 16),
 *     from the per-device table that lbdd_autotune measures (the SM-time per
 *     round, least first; instances that would outlast the rest of the
 *     batch move to faster clusters); without measurements about k/128
 *     CTAs; cluster_size > 0 forces one size for all;
 *   - instances with the same cost width, C and solver options (strict,
 *     lbdd_option flags) form a group, at most 16 groups per batch (more:
 *     LBDD_ERR_ARG): one persistent launch whose clusters take instances
 *     from a device-side queue, the longest estimated solve first; the SMs
 *     are shared between the groups
 *     in proportion to their estimated SM-time (max_clusters > 0 caps each
 *     group's clusters) and the groups run concurrently;
 *   - one pass (set the round targets, the concurrent group launches, read
 *     the statuses) is captured once as a CUDA graph.
 * lbdd_batch_run replays the graph on `stream` (given at create) and waits:
 * every instance advances by up to max_rounds rounds (< 0: to completion),
 * exactly as lbdd_solve(s, max_rounds) would advance it alone.  Returns the
 * first failing instance's status.
 * lbdd_batch_plan reports the plan: cluster_of[m] (nullable), the number of
 * groups, and per group (up to max_groups) its cluster size, cluster count
 * and instance count (each nullable).
 * lbdd_solve_batch is create + run + destroy without the graph. */
typedef struct lbdd_batch lbdd_batch;
int lbdd_batch_create(lbdd_batch** out, lbdd_solver* const* solvers, int m, int cluster_size,
                      int max_clusters, void* stream);
int lbdd_batch_run(lbdd_batch* b, int64_t max_rounds);
int lbdd_batch_plan(const lbdd_batch* b, int32_t* cluster_of, int32_t* ngroups,
                    int32_t* group_cluster, int32_t* group_clusters, int32_t* group_size,
                    int max_groups);
void lbdd_batch_destroy(lbdd_batch* b);
int lbdd_solve_batch(lbdd_solver* const* solvers, int m, int64_t max_rounds,
                     int cluster_size, int max_clusters, void* stream);

/* Autotuner of the batch plan: for every (cost width, k bucket
 * 2^(b-1) < k <= 2^b) present among the m solvers, takes the instance with
 * the most units, builds a scaled-down copy (its first probe_rounds units,
 * capacities scaled by the same ratio) and times a complete solve of it on
 * one cluster of each size that fits; the ns per round are kept per device for
 * the process's lifetime and used by every later batch plan and server pass.
 * The solvers themselves are not modified.  lbdd_tune_get reads one entry
 * (0 = not measured); lbdd_tune_clear forgets all. */
int lbdd_autotune(lbdd_solver* const* solvers, int m, int probe_rounds, void* stream);
int lbdd_tune_get(int cm_dtype, int32_t k, int cluster_size, double* ns_per_round);
int lbdd_tune_clear(void);

/* ---------------------------------------------------------------------
 * Request server (continuous batching; no counterpart in the paper).
 * Solve requests of mixed sizes are admitted in arrival order while the
 * device-memory budget and the active-slot limit allow; admitted requests
 * keep CM, allotment and loads resident on the device and advance together
 * in time-sliced passes (the batch plan above: SM shares in proportion to
 * remaining work, shortest remaining work first within a cluster size;
 * each pass ends after quantum_us); a request that made no progress for 8
 * passes in a row goes first within its cluster size until it runs again.
 * Requests admitted during a pass join the next one, finished ones are
 * retired (allotment copied to the caller's buffer, device memory freed)
 * while others keep solving.  Each result is bit-identical to the same
 * instance solved alone. */
typedef struct lbdd_server lbdd_server;
typedef struct lbdd_server_config {
  size_t budget_bytes;   /* device bytes all admitted requests may hold */
  int max_active;        /* requests admitted at once (0 = one per SM) */
  int64_t quantum_us;    /* pass length in microseconds (0 = 20000) */
  int cluster_size;      /* 0 = from the batch plan, else forced (1..16) */
} lbdd_server_config;
typedef enum lbdd_request_state {
  LBDD_REQ_QUEUED = 0, LBDD_REQ_ACTIVE = 1, LBDD_REQ_DONE = 2, LBDD_REQ_FAILED = 3
} lbdd_request_state;
typedef struct lbdd_request_info {
  int32_t state;         /* lbdd_request_state */
  int32_t status;        /* LBDD_OK, or why the request failed */
  int64_t objective;     /* Eq. (1) of the final allotment (state DONE) */
  int64_t rounds;        /* rounds done at the end of the last pass */
  int64_t submit_ns, admit_ns, done_ns;  /* server clock (ns since create); -1 = not yet */
} lbdd_request_info;
typedef struct lbdd_server_stats {
  int64_t passes, admitted, completed, failed, queued;
  int64_t bytes_in_use, peak_bytes;      /* budget held now / at most */
  int64_t busy_ns, uptime_ns;            /* time with a pass in flight / since create */
  int64_t peak_active;                   /* most requests in one pass */
  int64_t launches;                      /* kernels launched by all passes */
} lbdd_server_stats;
/* The server runs on the current device with its own streams and threads. */
int lbdd_server_create(lbdd_server** out, const lbdd_server_config* cfg);
/* Queue one request.  cm (host, n*k demand-major, cm_dtype) and assign_out
 * (host int32[n]) must stay valid until the request is DONE or FAILED;
 * cap and pen are copied.  *ticket identifies the request.  A request whose
 * footprint exceeds the whole budget fails with LBDD_ERR_BUDGET. */
int lbdd_server_submit(lbdd_server* srv, int32_t n, int32_t k, const void* cm, int cm_dtype,
                       const int32_t* cap, const int32_t* pen, int32_t* assign_out,
                       int64_t* ticket);
/* As lbdd_server_submit, with cm in device memory of the server's device
 * when cm_is_device = 1 (0: host, the same as lbdd_server_submit).  A
 * device cm must already hold its values when the call is made (work that
 * writes it must have completed) and stay valid until the request is DONE
 * or FAILED; admission copies it on the server's own stream.  Other
 * values of cm_is_device return LBDD_ERR_ARG. */
int lbdd_server_submit_ex(lbdd_server* srv, int32_t n, int32_t k, const void* cm, int cm_dtype,
                          int cm_is_device, const int32_t* cap, const int32_t* pen,
                          int32_t* assign_out, int64_t* ticket);
/* Wait up to timeout_ms (< 0: forever, 0: do not wait) for a request to end;
 * fills *out either way.  LBDD_OK when it ended, LBDD_ERR_TIMEOUT if not. */
int lbdd_server_poll(lbdd_server* srv, int64_t ticket, int64_t timeout_ms,
                     lbdd_request_info* out);
/* Forget an ended request's record (its ticket becomes invalid). */
int lbdd_server_release(lbdd_server* srv, int64_t ticket);
int lbdd_server_get_stats(lbdd_server* srv, lbdd_server_stats* out);
/* Stop: queued requests fail with LBDD_ERR_STATE, the pass in flight ends
 * at its quantum, everything is freed (request records included).  No other
 * call on the same server may be in progress or follow it: a thread still
 * waiting in lbdd_server_poll would wait on freed state. */
void lbdd_server_destroy(lbdd_server* srv);

/* Insert one demand unit into a solver.  The paper's proof sketch of its
 * dynamic-update theorem (commented out of the text, end of Section 4 and of
 * the appendix): adding a demand unit is one more iteration of the loop of
 * Alg. 2 -- allot it to its most suitable center, then Negative Cycle
 * Refinement and, if that center was full, Negative Path Refinement.
 *   row      : the unit's k costs (host memory, cm_dtype), every one >= 1; a
 *              solver that stores its CM as int16 refuses a cost above 32767.
 *   unit_out : the unit's index, the solver's unit count before the call.
 * The unit is extracted after every unit already in the solver, in insertion
 * order: the next lbdd_solve allots it (a solve that has finished runs just
 * the new rounds).  Before the first round of a solver, inserted units simply
 * join the instance (the first solve orders all units).  lbdd_reset restarts
 * a solve of all units in the MinDistance order.  Device arrays grow by half
 * when full (a short synchronous reallocation).  Errors: LBDD_ERR_ARG (bad
 * arguments or costs), LBDD_ERR_STATE (a strict-LBDD solver, or one held by a
 * batch), LBDD_ERR_OOM / LBDD_ERR_CUDA (growth failed; the solver is
 * unchanged).  Deletion is not provided: the proof sketch leaves the edges of
 * the reverse path undefined. */
int lbdd_insert(lbdd_solver* s, const void* row, int cm_dtype, int32_t* unit_out);

/* Tracked objective Delta of Alg. 2 (equals Eq. (1) of the current
 * allotment).  out: host pointer. */
int lbdd_objective(const lbdd_solver* s, int64_t* out);

/* Copy the allotment: n int32 center indices, -1 for units not allotted yet.
 * out is a host pointer unless out_is_device != 0. */
int lbdd_assignment(const lbdd_solver* s, int32_t* out, int out_is_device);

/* Copy the k center loads (int32, host). */
int lbdd_loads(const lbdd_solver* s, int32_t* out);

int lbdd_rounds_done(const lbdd_solver* s, int64_t* out);

/* Counters of the solve so far (host struct). */
int lbdd_get_stats(const lbdd_solver* s, lbdd_stats* out);

/* Copy the solver's best-transfer table (Defs. 8-10: for every ordered pair
 * (u, v), the cheapest transfer of a unit allotted to u over to v):
 * tc[u*k+v] = CM(d,v) - CM(d,u) of the lexicographically smallest
 * (cost, d), INT32_MAX if u holds no unit or u == v; td[u*k+v] = that d or
 * -1.  k*k int32 each, host memory unless out_is_device != 0. */
int lbdd_best_transfer_table(const lbdd_solver* s, int32_t* tc, int32_t* td, int out_is_device);

/* Release everything the solver owns.  NULL is accepted. */
void lbdd_destroy(lbdd_solver* s);

/* Human-readable text of a status code (static storage). */
const char* lbdd_strerror(int code);

/* Most recent CUDA error string seen by the library (static storage). */
const char* lbdd_last_cuda_error(void);

/* ---------------------------------------------------------------------
 * Best-transfer table from scratch (the data-parallel scan replacing the
 * paper's Gamma-DS update, Section 3.4 "Allotment subspace multi-graph
 * implementation" and Section 3.5.2): for an allotment assign[n] (entries
 * < 0 are skipped), compute for every ordered pair (u, v), u != v,
 *     T[u][v] = lexmin over d with assign[d] == u of (CM(d,v) - CM(d,u), d)
 * with the tc/td encoding of lbdd_best_transfer_table.
 *   cm_dev     : device CM, rows of ld >= k elements, ld*elem a multiple of
 *                16 bytes, the allocation readable for 128 elements past the
 *                last row; cm_dtype an lbdd_cm_dtype.  Entries are positive
 *                (Section 2: CM holds positive integers); the int16 scan
 *                relies on it (every difference then fits 16 bits).
 *   assign_dev : device int32[n], values in [-1, k).
 *   tc_dev, td_dev : device int32[k*k] outputs.
 *   workspace  : device scratch of lbdd_best_transfer_workspace(n, k) bytes,
 *                owned by the caller; contents on entry are ignored.
 *   stream     : cudaStream_t or NULL.  Asynchronous: results are ready
 *                when the stream reaches this point.
 * Errors: LBDD_ERR_ARG (sizes, alignment, workspace too small),
 * LBDD_ERR_CUDA (launch failure).  Every wait inside the scan is bounded
 * (1 s); one that runs out marks the whole table (tc = INT32_MAX, td = -2)
 * instead of returning a partial result. */
size_t lbdd_best_transfer_workspace(int32_t n, int32_t k);
int lbdd_best_transfer(int32_t n, int32_t k, const void* cm_dev, int cm_dtype, int64_t ld,
                       const int32_t* assign_dev, int32_t* tc_dev, int32_t* td_dev,
                       void* workspace, size_t workspace_bytes, void* stream);

/* The same table as lbdd_best_transfer, computed without allocating any
 * device memory.  The paper has no counterpart: this call exists for callers
 * that must not call cudaMalloc when they need the table, because cudaMalloc
 * can synchronise the whole device or because their device memory is fixed
 * in advance by a host application.  Instead of a caller workspace, the
 * scratch is one file-scope device array of 64 MiB, reserved on every GPU that
 * loads this library until the process exits.
 *   Arguments as for lbdd_best_transfer (inputs and outputs are still the
 *   caller's device buffers), without the workspace.
 *   Limit: lbdd_best_transfer_workspace(n, k) must not exceed 64 MiB, else
 *   LBDD_ERR_BUDGET is returned and nothing is launched (the city-scale
 *   200,000 x 500 case needs 34,988,800 bytes, about 33.4 MiB).
 *   The first call on each device looks up the device address of the array
 *   (with that device current); make that first call before any stream
 *   capture.
 *   All calls on a device share the one array and every call rewrites what
 *   it reads, so consecutive calls are independent; calls whose work overlaps
 *   on the GPU (different streams, or different host threads) race on it and
 *   must be serialised by the caller.
 * Errors: LBDD_ERR_ARG, LBDD_ERR_BUDGET, LBDD_ERR_NODEV, LBDD_ERR_CUDA. */
int lbdd_best_transfer_noalloc(int32_t n, int32_t k, const void* cm_dev, int cm_dtype, int64_t ld,
                               const int32_t* assign_dev, int32_t* tc_dev, int32_t* td_dev,
                               void* stream);

/* ---------------------------------------------------------------------
 * Cost matrix from a road network (Section 3.4 "Demand-service cost matrix
 * construction": shortest paths when centers and demand lie on a road
 * network; Section 5 uses the New Delhi network this way).
 *   V            : nodes; row_ptr (V + 1), col, w (row_ptr[V] each): a
 *                  directed CSR graph, lengths w >= 1 (give both directions
 *                  of a two-way road); (V - 1) * max(w) must be < 2^31.
 *   centers (k)  : center nodes; demand (n): one node per demand unit.
 *   cm (n x ld)  : output, int32, CM[d * ld + s] = shortest path length from
 *                  centers[s] to demand[d] (ld >= k).
 * All arrays are device memory; work is ordered on `stream` and the call
 * waits for it.  Scratch (k x V labels and per-CTA frontier queues) is
 * allocated from the stream-ordered pool and freed before returning.
 * Errors: LBDD_ERR_ARG (bad graph or ids, lengths that could overflow, a
 * demand node no center reaches, a demand node that is a center's node:
 * CM entries must be >= 1), LBDD_ERR_CUDA, LBDD_ERR_OOM. */
int lbdd_road_cm(int32_t V, const int32_t* row_ptr, const int32_t* col, const int32_t* w,
                 int32_t k, const int32_t* centers, int32_t n, const int32_t* demand,
                 int32_t* cm, int64_t ld, void* stream);

/* Row pitch (elements) that lbdd_create uses for a CM of k columns, and the
 * device pointer / pitch of a solver's stored CM (for lbdd_best_transfer). */
int64_t lbdd_cm_pitch(int32_t k, int cm_dtype);
int lbdd_solver_cm(const lbdd_solver* s, const void** cm_dev, int* cm_dtype, int64_t* ld);

#ifdef __cplusplus
}
#endif

#endif /* LBDD_H */
