// Persistent ASRAL solver: one thread-block cluster runs whole solves.
//
// Paper: Ramnath et al., "Load Balanced Demand Distribution under Overload
// Penalties" (arXiv 2304.06543).  Alg. 2 (ASRAL main loop), Alg. 1 (Negative
// Cycle Refinement), Alg. 4 (Negative Path Refinement, Appendix A), Defs. 8-10
// (allotment subspace multigraph, NCyc and NPath graphs), Alg. 3 (parallel
// Bellman-Ford).
//
// GB300 design (not the paper's JCuda design, which copied the graph to the
// GPU and synchronised the host after every Bellman-Ford sweep):
//  * the whole solve - prologue, all n rounds - runs inside one launch on one
//    cluster of C CTAs; nothing returns to the host between rounds;
//  * the best-transfer table T (the heap tops of the paper's BestTransHeaps)
//    is a dense k x k table, column-partitioned: CTA r of the cluster owns
//    columns [r*w, r*w + w) of every row and is the only CTA that reads or
//    writes them.  The cost half of the owned slice also lives in the CTA's
//    shared memory when it fits (int16 when CM is int16), so Bellman-Ford
//    relaxations read shared memory; the unit half stays in global memory;
//  * Bellman-Ford is the synchronous form with a frontier (only labels that
//    changed in the previous sweep can improve a label); after each sweep
//    every CTA pushes a fixed-size message with its owned label changes into
//    every other CTA's shared memory (st.async) and waits on a transaction
//    barrier of its own for the messages of all others, so a sweep costs one
//    one-way transfer instead of a cluster barrier plus a remote read;
//  * when a unit changes center, the rows of T of the centers on the path are
//    recomputed from their member lists (segment rescan), reading CM rows with
//    16-byte vector loads.
// Tie-breaking is canonical and identical to the CPU oracle: (cost, unit)
// lexicographic in T, lowest predecessor index on equal Bellman-Ford labels.
#include <limits>
#include <type_traits>
#include <mutex>

#include "lbdd_device.cuh"

namespace lbdd {

struct Layout {
  uint32_t dist, hop, slack, pen, par, inbox, npart, path, pathu, misc, tail, rsink, elist, red, tsm,
      msg, base_total, total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline int32_t own_width(int32_t k, int32_t C, int32_t vpl) {
  int32_t w = (k + C - 1) / C;
  return (w + vpl - 1) / vpl * vpl;
}

// Row stride of the shared cost slice: w plus padding that makes the stride
// an odd number of 4-byte words, so lanes reading one column of different
// rows hit different banks.
__host__ __device__ inline int32_t slice_stride(int32_t w, int32_t elem) {
  return w + (elem == 2 ? 2 : 1);
}

constexpr uint32_t kRedBytes = kThreads * 8 * 8;  // rescan partials, int16 CM

// Bytes of one CTA's Bellman-Ford message for one sweep: a label per owned
// column (4 bytes with int16 costs, 8 with int32 costs), then a 16-byte tail
// (merge flag, padding, sink key).  A multiple of 16 because w is a
// multiple of 16 / elem.
__host__ __device__ inline uint32_t msg_bytes(int32_t w, int32_t elem) {
  return (uint32_t)w * (elem == 2 ? 4u : 8u) + 16u;
}

// Shared-memory carve-up; `base_total` excludes the cost slice, `total`
// includes it (k x w entries of elem bytes).
__host__ __device__ inline Layout make_layout(int32_t k, int32_t C, int32_t elem) {
  Layout L;
  uint32_t o = 0;
  const int32_t vpl = 16 / elem;
  const uint32_t w = (uint32_t)own_width(k, C, vpl);
  const uint32_t ku = (uint32_t)k, Cu = (uint32_t)C;
  L.msg = msg_bytes((int32_t)w, elem);
  L.dist = o;   o = align16(o + 8u * w);                // labels of the owned columns
  L.hop = o;    o = align16(o + 4u * w);
  L.slack = o;  o = align16(o + 4u * ku);               // load - capacity per center
  L.pen = o;    o = align16(o + 4u * ku);
  L.par = o;    o = align16(o + 4u * w);
  L.inbox = o;  o = align16(o + 2u * Cu * L.msg);       // [2][C] messages, by sweep parity
  L.npart = o;  o = align16(o + Cu * 16u);               // per-CTA partial minima
  L.path = o;   o = align16(o + 4u * (ku + 2));
  L.pathu = o;  o = align16(o + 4u * (ku + 2));
  L.misc = o;   o = align16(o + 8u * 16u);
  L.tail = o;   o = align16(o + 8u * kMaxCluster);      // count and merge flag per sender
  L.rsink = o;  o = align16(o + 8u * kWarps);           // per-warp NPath sink candidates
  L.elist = o;  o = align16(o + (elem == 2 ? 8u : 16u) * 32u * kWarps);   // per-warp frontier lists
  // rescan partials, and the per-warp column minima of a sweep ([kWarps][w + 1] keys)
  const uint32_t redb = 8u * kWarps * (w + 1);
  L.red = o;    o = align16(o + (redb > kRedBytes ? redb : kRedBytes));
  L.base_total = o;
  L.tsm = o;    o = align16(o + (uint32_t)elem * ku * (uint32_t)slice_stride((int32_t)w, elem));
  L.total = o;
  return L;
}

constexpr uint64_t kNoKey = ~0ull;   // no candidate (no real key has all bits set)
// Slots of the per-CTA scalar block.
enum { MS_SINK_DIST = 0, MS_SINK_PAR, MS_PATHLEN, MS_NAFF, MS_MERGE_ANY, MS_STOP0, MS_STOP1,
       MS_ABORT, MS_SINK_IN };

// Longest wait for the other CTAs' messages of one sweep (globaltimer ns).
// A sweep's messages arrive within microseconds; reaching this limit means
// a broken exchange, which is reported as LBDD_ERR_TIMEOUT.
constexpr uint64_t kWaitLimitNs = 1000000000ull;
// Longest sleep inside one barrier test (the waiting warp wakes when the
// phase completes, so a long limit only keeps the warp from spinning).
constexpr uint32_t kSleepNs = 10000000;

// Rounds between two checks of the launch's time quantum.
constexpr int kQuantumCheck = 8;

// Counters and timers kept by thread 0 of CTA 0 (shared memory, so that
// they cost no registers in the other threads).
struct Book {
  int64_t delta, free_top, cycles, paths, bf_calls, bf_sweeps, bf_max, moves, skipped, rows;
  int64_t t_merge, t_relax, t_sync, t_gather, t_apply, t_rescan, t_rloop, t_rred;
  int64_t npath_reused, col_rows, front_sum, front_hist[6];
  int64_t err0;   // a guard tripped (corrupt state; never expected)
  uint64_t deadline;   // globaltimer ns at which the launch yields (0: never)
};

template <typename T>
struct Solver {
  __device__ explicit Solver(const DevInst& inst) : I(inst) {}

  static constexpr int VPL = 16 / (int)sizeof(T);
  using TS = T;                                           // cost type of the shared slice
  static constexpr int32_t kTsInf = std::numeric_limits<TS>::max();
  // Bellman-Ford label of a frontier node and in a message.  With int16
  // costs every transfer edge is below 2^15 in magnitude and a frontier
  // label sums at most k + 1 <= 4801 of them, so 32 bits hold it exactly
  // (the sink, whose penalty edges are larger, is never a frontier node and
  // travels as a 64-bit key).  int32 costs need 64 bits.
  using LT = typename std::conditional<sizeof(T) == 2, int32_t, int64_t>::type;
  static constexpr LT kNoLab = std::numeric_limits<LT>::max();

  const DevInst& I;   // shared-memory copy of the current instance
  const T* cm;
  int32_t n, k, C, rank, w, ws, c0, c1, wr;
  int tid;
  int flags;
  bool quantum_on;    // the launch is time-sliced (Book::deadline set)
  bool tsm_on;        // owned cost slice resident in shared memory
  int64_t* s_dist;    // [w] labels of the owned columns
  int32_t* s_hop;     // [w] sweep of each owned column's last label change
  int32_t* s_slack;   // [k] load - capacity of every center (>= 0: no vacancy)
  int32_t* s_pen;     // [k] penalty one more unit would pay at each center, q_c(load_c - cap_c + 1)
  int32_t* s_par;     // parents of the owned columns
  unsigned char* s_inbox;  // [2][C] messages of every CTA, by sweep parity (msg_bytes each)
  uint32_t mbytes;    // bytes of one message
  uint64_t* s_mbar;   // [2][kMaxCluster] transaction barriers, by parity and sender
  uint32_t mph;       // phase parity of the barriers of each message parity
  int32_t* s_tail;    // [kMaxCluster][2] count and merge flag of each sender's last message
  uint64_t* s_rsink;  // [kWarps] per-warp NPath sink candidates
  unsigned char* s_elist;  // [kWarps][32] per-warp frontier entries (label, node)
  int64_t* s_npart;   // [C][2]: per-CTA partial minima (label; hop << 16 | node)
  int32_t* s_path;
  int32_t* s_pathu;
  int64_t* s_misc;
  unsigned char* s_red;
  TS* s_tc;           // [k][ws] owned costs (if tsm_on)
  int buf;            // exchange buffer parity, advances every sweep

  Book* B;            // CTA 0 thread 0 bookkeeping (shared memory)
  int32_t pending_d = -1, pending_j = -1, pending_own = 0;

  // Phase timers run on CTA 0's thread 0, on the path every other CTA waits
  // for at the cluster barriers, so they are off unless asked for.
  __device__ __forceinline__ bool timer() const {
    return (flags & OPT_PHASE_TIMERS) && rank == 0 && tid == 0;
  }
  __device__ __forceinline__ const T* row(int32_t d) const { return cm + (int64_t)d * I.ld; }

  // Member idx of c's list; the member's own cost CM(d, c) sits kPage
  // words further in the same page, so rescans need no CM read for it.
  __device__ __forceinline__ int32_t* mslot(int32_t c, int32_t idx) const {
    int32_t page = __ldcg(I.page_tab + (int64_t)c * I.max_pages + (idx >> kPageShift));
    return I.pool + (int64_t)page * kPageWords + (idx & (kPage - 1));
  }

  // Owned cost of row u, owned column cl (kTInf for "no edge").
  __device__ __forceinline__ int32_t own_cost(int32_t u, int cl) const {
    if (tsm_on) {
      const int32_t t = (int32_t)s_tc[u * ws + cl];
      return t == kTsInf ? kTInf : t;
    }
    return I.tc[(int64_t)u * k + c0 + cl];
  }
  __device__ __forceinline__ void set_entry(int32_t u, int cl, int32_t t, int32_t d) {
    I.tc[(int64_t)u * k + c0 + cl] = t;
    I.td[(int64_t)u * k + c0 + cl] = d;
    if (tsm_on) s_tc[u * ws + cl] = (TS)(t == kTInf ? kTsInf : t);
  }

  // Member-list primitives, called by one thread of CTA 0 only.  `own` is
  // CM(d, c).
  __device__ void list_append(int32_t c, int32_t d, int32_t own) {
    int32_t idx = I.seg_size[c];
    if (c < 0 || c >= k || d < 0 || d >= n || idx < 0 || idx >= n) { B->err0 = ST_ERR_INVARIANT; return; }
    if ((idx & (kPage - 1)) == 0) {
      if (B->free_top <= 0) { B->err0 = ST_ERR_INVARIANT; return; }
      int32_t page = I.free_stack[--B->free_top];
      I.page_tab[(int64_t)c * I.max_pages + (idx >> kPageShift)] = page;
    }
    int32_t* slot = mslot(c, idx);
    slot[0] = d;
    slot[kPage] = own;
    I.pos[d] = idx;
    I.seg_size[c] = idx + 1;
  }
  // Remove the unit stored at index idx of c's list (its position before
  // any move of this path was applied).
  __device__ void list_remove_at(int32_t c, int32_t idx) {
    int32_t last = I.seg_size[c] - 1;
    if (c < 0 || c >= k || idx < 0 || idx > last || B->free_top >= I.npages) {
      B->err0 = ST_ERR_INVARIANT;
      return;
    }
    if (idx != last) {
      const int32_t* from = mslot(c, last);
      int32_t* to = mslot(c, idx);
      const int32_t moved = from[0];
      to[0] = moved;
      to[kPage] = from[kPage];
      I.pos[moved] = idx;
    }
    if ((last & (kPage - 1)) == 0)
      I.free_stack[B->free_top++] = I.page_tab[(int64_t)c * I.max_pages + (last >> kPageShift)];
    I.seg_size[c] = last;
  }

  // ------------------------------------------------------------ prologue --
  // Alg. 2, first step: s_min(d) = lowest-index minimum of CM row d; the
  // MinDistance heap's extraction order = stable sort of d by CM(d, s_min).
  __device__ void prologue() {
    const int lane = tid & 31, warp = tid >> 5;
    int32_t* keys0 = I.sort_tmp;
    int32_t* vals0 = I.sort_tmp + n;
    uint32_t kmax = 0;
    const bool strict = flags & OPT_STRICT;
    if (strict) {   // Alg. 5 visits the units in index order; centers are chosen per round
      for (int64_t d = (int64_t)rank * kThreads + tid; d < n; d += (int64_t)C * kThreads) {
        I.order[d] = (int32_t)d;
        I.assign[d] = -1;
      }
    }
    for (int64_t d = (int64_t)rank * kWarps + warp; d < n && !strict; d += (int64_t)C * kWarps) {
      const T* r = row((int32_t)d);
      int32_t bv = INT32_MAX, bj = INT32_MAX;
      for (int col = lane * VPL; col < k; col += 32 * VPL) {
        Vec16<T> x = load16(r + col);
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
          int32_t v = (int32_t)x.v[q];
          if (col + q < k && v < bv) { bv = v; bj = col + q; }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        int32_t ov = __shfl_xor_sync(0xffffffffu, bv, off);
        int32_t oj = __shfl_xor_sync(0xffffffffu, bj, off);
        if (ov < bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
      }
      if (lane == 0) {
        I.smin[d] = bj;
        keys0[d] = bv;
        vals0[d] = (int32_t)d;
        I.assign[d] = -1;
      }
      kmax = max(kmax, (uint32_t)bv);
    }
    // fresh state: empty lists, zero loads, empty best-transfer table
    const int64_t gt = (int64_t)rank * kThreads + tid, gs = (int64_t)C * kThreads;
    for (int64_t i = gt; i < k; i += gs) { I.seg_size[i] = 0; I.load[i] = 0; }
    for (int64_t u = 0; u < k; ++u)   // each CTA clears the columns it owns
      for (int cl = tid; cl < wr; cl += kThreads) {
        I.tc[u * k + c0 + cl] = kTInf;
        I.td[u * k + c0 + cl] = -1;
      }
    for (int64_t i = gt; i < I.npages; i += gs) I.free_stack[i] = I.npages - 1 - (int32_t)i;
    if (kmax) atomicMax(reinterpret_cast<unsigned long long*>(&I.ctl[CTL_MAXKEY]),
                        (unsigned long long)kmax);
    __syncthreads();
    cluster_sync_all();
    if (rank == 0 && !strict) sort_order();
    __syncthreads();
    cluster_sync_all();
  }

  // Alg. 5: the cheapest center that still has a vacancy (a dummy unit),
  // lowest index on equal cost; every CTA computes the same answer from the
  // row and its load/capacity replicas.  -1 if no center has a vacancy.
  __device__ int32_t strict_target(int32_t d) {
    const T* r = row(d);
    int32_t bv = INT32_MAX, bj = -1;
    for (int s = tid; s < k; s += kThreads) {
      if (s_slack[s] < 0) {
        const int32_t v = (int32_t)r[s];
        if (v < bv) { bv = v; bj = s; }
      }
    }
    auto better = [](int32_t v, int32_t j, int32_t bv_, int32_t bj_) {
      return bj_ < 0 || (j >= 0 && (v < bv_ || (v == bv_ && j < bj_)));
    };
    for (int off = 16; off > 0; off >>= 1) {
      const int32_t ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, off);
      if (better(ov, oj, bv, bj)) { bv = ov; bj = oj; }
    }
    int2* part = reinterpret_cast<int2*>(s_red);
    if ((tid & 31) == 0) part[tid >> 5] = make_int2(bv, bj);
    __syncthreads();
    bv = INT32_MAX;
    bj = -1;
    for (int w2 = 0; w2 < kWarps; ++w2)
      if (better(part[w2].x, part[w2].y, bv, bj)) { bv = part[w2].x; bj = part[w2].y; }
    __syncthreads();   // part is scratch for the next user
    return bj;
  }

  // Stable LSD radix sort of (key, d) by key, by CTA 0 alone.  The values
  // start in d order, so the result is ordered by (key, d).
  __device__ void sort_order() {
    const int lane = tid & 31, warp = tid >> 5;
    int32_t* s_off = reinterpret_cast<int32_t*>(s_red);   // 256
    int32_t* s_wc = s_off + 256;                          // kWarps x 256
    const uint32_t kmax = (uint32_t)__ldcg(I.ctl + CTL_MAXKEY);
    const int bits = 32 - __clz((int)max(kmax, 1u));
    const int passes = (bits + 7) / 8;
    int32_t *k0 = I.sort_tmp, *v0 = I.sort_tmp + n, *k1 = I.sort_tmp + 2 * (int64_t)n,
            *v1 = I.order;
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (int p = 0; p < passes; ++p) {
      const int shift = 8 * p;
      int32_t *sk = (p & 1) ? k1 : k0, *sv = (p & 1) ? v1 : v0;
      int32_t *dk = (p & 1) ? k0 : k1, *dv = (p & 1) ? v0 : v1;
      for (int i = tid; i < 256; i += kThreads) s_off[i] = 0;
      __syncthreads();
      for (int64_t i = tid; i < n; i += kThreads) atomicAdd(&s_off[(__ldcg(sk + i) >> shift) & 255], 1);
      __syncthreads();
      if (tid == 0) {
        int32_t run = 0;
        for (int b = 0; b < 256; ++b) { int32_t c = s_off[b]; s_off[b] = run; run += c; }
      }
      __syncthreads();
      for (int64_t base = 0; base < n; base += kThreads) {
        const int64_t i = base + tid;
        const bool valid = i < n;
        const int32_t key = valid ? __ldcg(sk + i) : 0, val = valid ? __ldcg(sv + i) : 0;
        const int dig = valid ? ((key >> shift) & 255) : 256;
        const uint32_t peers = __match_any_sync(0xffffffffu, dig);
        const int rk = __popc(peers & lt);
        const bool leader = (__ffs(peers) - 1) == lane;
        for (int x = tid; x < kWarps * 256; x += kThreads) s_wc[x] = 0;
        __syncthreads();
        if (valid && leader) s_wc[warp * 256 + dig] = __popc(peers);
        __syncthreads();
        if (tid < 256) {
          int32_t run = s_off[tid];
          for (int ww = 0; ww < kWarps; ++ww) {
            int32_t c = s_wc[ww * 256 + tid];
            s_wc[ww * 256 + tid] = run;
            run += c;
          }
          s_off[tid] = run;
        }
        __syncthreads();
        if (valid) {
          const int32_t at = s_wc[warp * 256 + dig] + rk;
          dk[at] = key;
          dv[at] = val;
        }
        __syncthreads();
      }
    }
    if ((passes & 1) == 0)
      for (int64_t i = tid; i < n; i += kThreads) I.order[i] = v0[i];
    __syncthreads();
  }

  // Owned cost slice from the global table (after a prologue or on resume).
  __device__ void load_slice() {
    if (!tsm_on) return;
    for (int64_t u = 0; u < k; ++u)
      for (int cl = tid; cl < w; cl += kThreads) {
        const int32_t t = cl < wr ? __ldcg(I.tc + u * k + c0 + cl) : kTInf;
        s_tc[u * ws + cl] = (TS)(t == kTInf ? kTsInf : t);
      }
    __syncthreads();
  }

  // ---------------------------------------------------- best-transfer T --
  // Alg. 2, allotment step: unit d joins center j; its k-1 transfer edges
  // CM(d, v) - CM(d, j) (Def. 8) enter the per-pair minima of row j.
  // Returns whether a cost of row j decreased in this CTA's columns.
  __device__ bool merge_row(int32_t d, int32_t j) {
    bool changed = false;
    const int S = w / VPL;
    if (tid < S) {
      const T* r = row(d);
      const int32_t own = (int32_t)r[j];
      const int cl0 = tid * VPL;
      Vec16<T> x = load16(r + c0 + cl0);
#pragma unroll
      for (int q = 0; q < VPL; ++q) {
        const int cl = cl0 + q, v = c0 + cl;
        if (v < k && v != j) {
          const int32_t t = (int32_t)x.v[q] - own;
          const int32_t bt = own_cost(j, cl);
          if (t <= bt) {
            const int32_t bd = I.td[(int64_t)j * k + v];
            if (lex_less(t, d, bt, bd)) {
              set_entry(j, cl, t, d);
              changed |= (t < bt);
            }
          }
        }
      }
    }
    return __syncthreads_or(changed) != 0;
  }

  // Row c of T over the owned columns, recomputed from c's member list:
  // T[c][v] = lexmin over d in seg(c) of (CM(d, v) - CM(d, c), d).
  __device__ void rescan(int32_t c) {
    constexpr int U = 4;   // member rows in flight per thread
    const int S = w / VPL;
    const int R = kThreads / S;
    const int slot = tid % S, g = tid / S;
    // member lists are written by CTA 0: read them past L1
    const int32_t s = __ldcg(I.seg_size + c);
    int32_t bt[VPL], bd[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) { bt[q] = kTInf; bd[q] = -1; }
    if (g < R) {
      for (int32_t base = g; base < s; base += U * R) {
        int32_t dd[U], own[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t idx = base + u * R;
          const int32_t* sl = idx < s ? mslot(c, idx) : nullptr;
          dd[u] = sl ? __ldcg(sl) : -1;
          own[u] = sl ? __ldcg(sl + kPage) : 0;
          if ((uint32_t)dd[u] >= (uint32_t)n) dd[u] = -1;   // guard: corrupt entry
        }
        Vec16<T> x[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (dd[u] >= 0) x[u] = load16(row(dd[u]) + c0 + slot * VPL);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (dd[u] < 0) continue;
#pragma unroll
          for (int q = 0; q < VPL; ++q) {
            const int32_t t = (int32_t)x[u].v[q] - own[u];
            if (lex_less(t, dd[u], bt[q], bd[q])) { bt[q] = t; bd[q] = dd[u]; }
          }
        }
      }
    }
    int2* red = reinterpret_cast<int2*>(s_red);   // [R][w]
    if (g < R) {
#pragma unroll
      for (int q = 0; q < VPL; ++q) red[g * w + slot * VPL + q] = make_int2(bt[q], bd[q]);
    }
    __syncthreads();
    for (int cl = tid; cl < wr; cl += kThreads) {
      const int v = c0 + cl;
      int32_t t = kTInf, d = -1;
      for (int gg = 0; gg < R; ++gg) {
        int2 e = red[gg * w + cl];
        if (lex_less(e.x, e.y, t, d)) { t = e.x; d = e.y; }
      }
      if (v == c) { t = kTInf; d = -1; }
      set_entry(c, cl, t, d);
    }
    if (rank == 0 && tid == 0) B->rows += s;
    __syncthreads();
  }

  // -------------------------------------------------------- Bellman-Ford --
  // Keys pack (label, node) so that one unsigned 64-bit minimum is the
  // lexicographic minimum of (label, node): node in the low 16 bits
  // (k <= 65535), label + 2^47 above it (labels are sums of at most k + 1
  // edge weights below 2^31 in magnitude, so |label| < 2^47).
  static __device__ __forceinline__ uint64_t pack_key(int64_t label, int32_t node) {
    return ((uint64_t)(label + ((int64_t)1 << 47)) << 16) | (uint32_t)node;
  }
  static __device__ __forceinline__ int64_t key_label(uint64_t key) {
    return (int64_t)(key >> 16) - ((int64_t)1 << 47);
  }

  // Message of CTA r for the sweep of parity p, in this CTA's inbox.
  __device__ __forceinline__ unsigned char* msg(int parity, int r) const {
    return s_inbox + ((uint32_t)(parity * C + r)) * mbytes;
  }
  __device__ __forceinline__ LT* msg_lab(unsigned char* m) const { return reinterpret_cast<LT*>(m); }
  // message tail: merge flag, padding, sink key
  __device__ __forceinline__ int32_t* msg_merge(unsigned char* m) const {
    return reinterpret_cast<int32_t*>(m + mbytes - 16);
  }
  __device__ __forceinline__ uint64_t* msg_sink(unsigned char* m) const {
    return reinterpret_cast<uint64_t*>(m + mbytes - 8);
  }
  // Transaction barrier of this CTA for CTA r's messages of parity p.
  __device__ __forceinline__ uint64_t* mbar(int parity, int r) const {
    return s_mbar + parity * kMaxCluster + r;
  }

  // q_c(x), x >= 1: penalty of the x-th allotment beyond capacity (Def. 4).
  __device__ __forceinline__ int32_t qval(int32_t c, int32_t x) const {
    return __ldg(I.pen + (int64_t)c * I.Q + min(max(x, 1), I.Q) - 1);
  }
  // Penalty replica entry of center c for its current load.  With a
  // constant penalty (Q = 1) the replica never changes, so callers skip the
  // update (a global load on the round's critical path).
  __device__ __forceinline__ int32_t qnext(int32_t c) const {
    return qval(c, s_slack[c] + 1);
  }
  // q_j of the anchor's last unit beyond capacity (load > cap).
  __device__ __forceinline__ int32_t qlast(int32_t j) const {
    return I.Q == 1 ? s_pen[j] : qval(j, s_slack[j]);
  }

  // Alg. 5 edge cost: a center with a vacancy can pass a dummy unit on for
  // free, so its transfer costs are min(T, 0) (an absent edge becomes 0).
  __device__ __forceinline__ int32_t strict_cost(int32_t t, int32_t u, int32_t inf) const {
    return (t == inf || t > 0) && s_slack[u] < 0 ? 0 : t;
  }

  // Cost of the transfer edge u -> owned column cl; kTsInf (TSM: slice in
  // shared memory) or kTInf (slice in global memory) for no edge.
  template <bool TSM>
  __device__ __forceinline__ int32_t edge(int32_t u, int cl) const {
    if (TSM) return (int32_t)s_tc[u * ws + cl];
    return I.tc[(int64_t)u * k + c0 + cl];
  }

  // One frontier entry of a warp's list: a label and its node.
  struct Ent {
    LT l;
    int32_t u;
  };

  // Relaxes the edges out of the n entries el[0..n) (node order) into owned
  // column cl (lane = column; `colok` false: no such column), folding the
  // candidates into (bl, bu); the strict "<" keeps the lowest node among
  // equal labels.  Warp-uniform n.
  template <bool STRICT, bool TSM>
  __device__ __forceinline__ void relax_list(const Ent* el, int n, int cl, bool colok, LT& bl,
                                             int32_t& bu) const {
    constexpr int32_t inf = TSM ? kTsInf : kTInf;
    constexpr int U = 4;
    int f = 0;
    for (; f + U - 1 < n; f += U) {
      Ent e[U];
      int32_t t[U];
#pragma unroll
      for (int q = 0; q < U; ++q) e[q] = el[f + q];
#pragma unroll
      for (int q = 0; q < U; ++q) t[q] = colok ? edge<TSM>(e[q].u, cl) : inf;
#pragma unroll
      for (int q = 0; q < U; ++q) {
        if (STRICT) t[q] = strict_cost(t[q], e[q].u, inf);
        const LT c = e[q].l + (LT)t[q];
        if (t[q] != inf && c < bl) { bl = c; bu = e[q].u; }
      }
    }
    for (; f < n; ++f) {
      const Ent e = el[f];
      int32_t t = colok ? edge<TSM>(e.u, cl) : inf;
      if (STRICT) t = strict_cost(t, e.u, inf);
      const LT c = e.l + (LT)t;
      if (t != inf && c < bl) { bl = c; bu = e.u; }
    }
  }

  // Strict improvement of owned column cl < wr.  Returns the label to
  // publish for it (kNoLab if it did not improve); the sink column (v == j)
  // writes its candidate key into the message tail instead and is never a
  // frontier node.  Only the owner reads and writes an owned column's label.
  __device__ __forceinline__ LT record(int cl, uint64_t best, int32_t j, int64_t sink_dist,
                                       int sweep, unsigned char* my) {
    const int v = c0 + cl;
    if (v == j) {
      *msg_sink(my) = best != ~0ull && key_label(best) < sink_dist ? best : kNoKey;
      return kNoLab;
    }
    if (best == ~0ull) return kNoLab;
    const int64_t bc = key_label(best);
    if (bc >= s_dist[cl]) return kNoLab;
    s_dist[cl] = bc;
    s_hop[cl] = sweep;
    s_par[cl] = (int32_t)(best & 0xffffu);
    return (LT)bc;
  }

  // Frontier-size statistics (phase timers only): a sweep relaxing `n` labels.
  __device__ __forceinline__ void front_stat(int n) {
    B->front_sum += n;
    B->front_hist[n <= 1 ? 0 : n <= 4 ? 1 : n <= 16 ? 2 : n <= 64 ? 3 : n <= 256 ? 4 : 5]++;
  }

  // Waits until the message of CTA r for the sweep of parity p is in: the
  // calling warp sleeps on the barrier (lane 0 of the first such warp
  // announces the message's bytes).  Bounded: past kWaitLimitNs the CTA
  // records LBDD_ERR_TIMEOUT and goes on.
  __device__ __forceinline__ void wait_message(int p, int r, bool announce) {
    uint64_t* b = mbar(p, r);
    if (announce && (tid & 31) == 0) mbar_arrive_expect(b, mbytes);
    __syncwarp();
    const uint32_t parity = (mph >> p) & 1u;
    if (!mbar_try_wait(b, parity, kSleepNs)) {
      const uint64_t t0 = gtimer_ns();
      while (!mbar_try_wait(b, parity, kSleepNs)) {
        if (gtimer_ns() - t0 > kWaitLimitNs) {
          s_misc[MS_ABORT] = 1;   // read after the next CTA barrier
          atomicExch(reinterpret_cast<unsigned long long*>(I.ctl + CTL_STATUS),
                     (unsigned long long)(int64_t)ST_ERR_TIMEOUT);
          break;
        }
      }
    }
  }

  // Canonical synchronous Bellman-Ford from the anchor j (Alg. 3 / Sections
  // 3.3-3.4).  Node u < k is center u, node j is s*out (the source) and the
  // sink s*in is represented by column j: an edge u -> s*in is
  //   NCyc (Def. 9 (c)): the best transfer u -> j,
  //   NPath (Def. 10 (c)): q_u() - q_j(), q_u() = pen[u] if load[u] >= cap[u].
  // No edge enters the source.  Labels change only on strict improvement and
  // take the lowest-index predecessor among equal candidates.
  //
  // Sweep s: every CTA writes a message (the new label of each owned column
  // that improved, kNoLab for the others, its merge flag and, at the owner
  // of column j, the sink candidate) into its own inbox slot and
  // bulk-copies it into the same slot of every other CTA's inbox (warp p to
  // the p-th other CTA; the copy engine moves the data, so the load/store
  // pipe stays free for relaxations), completing bytes on the receiver's
  // barrier for that sender and parity.  Sweep s + 1 relaxes the edges out
  // of the labels of sweep s (the frontier): the 16 warps are split among
  // the C senders; each warp waits only for its sender's message, compacts
  // its share of the sender's improved labels into a list of its own and
  // relaxes them into every owned column (lane = column), so relaxation
  // overlaps the arrival of the other messages.  A shared-memory transpose
  // then combines the warps' per-column minima.  Every CTA sees the same
  // messages, so all of them take the same decisions.  A CTA's slot r of a
  // parity is rewritten by CTA r two sweeps later, after r received this
  // CTA's next message, which this CTA sends after it has read the slot; and
  // a CTA rewrites its own slot (the copies' source) only after every other
  // CTA's next message arrived, each sent after the copy into it completed.
  // Returns 1 for a negative sink label (path to apply), 0 for none, and
  // < 0 on a broken invariant (-1) or exchange (-2).  `merged` says whether
  // this CTA's merge of the round's unit lowered a cost of row j (NegCycle
  // only).
  __device__ int bellman_ford(int32_t j, bool npath, bool merged, bool allow_skip) {
    for (int cl = tid; cl < w; cl += kThreads) {
      s_dist[cl] = kDInf;
      s_hop[cl] = -1;
      s_par[cl] = -1;
    }
    if (tid == 0) s_misc[MS_ABORT] = 0;
    __syncthreads();
    const int owner_j = j / w;
    // NPath (Def. 10 (c)): the penalty the anchor's last unit beyond capacity paid
    const int32_t pen_j = npath ? qlast(j) : 0;
    const bool strict = flags & OPT_STRICT;
    const bool sink_here = npath && rank == owner_j;   // this CTA relaxes Def. 10 (c) edges
    const int lane = tid & 31, warp = tid >> 5;
    const int WPS = kWarps / C;                         // warps per sender
    const int src = warp / WPS, sub = warp - src * WPS;
    const int ncb = (w + 31) / 32;                      // column blocks
    const int RS = w + 1;                               // row stride of the partial minima
    uint64_t* red = reinterpret_cast<uint64_t*>(s_red);  // [kWarps][RS] per-warp column minima
    Ent* el = reinterpret_cast<Ent*>(s_elist) + warp * 32;
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    int64_t sink_dist = kDInf;
    int32_t sink_par = -1;
    int result = 0;
    bool skipped_bf = false;
    for (int sweep = 1;; ++sweep) {
      const bool tmr = timer();
      const uint64_t t0 = tmr ? clock_cycles() : 0;
      if (tmr && sweep == 1) front_stat(1);
      const int pb = buf;        // parity of the message this sweep writes
      const int q = pb ^ 1;      // parity of the messages it reads (sweep - 1)
      // ---- relax the frontier (labels of sweep - 1; the source at sweep 1)
      unsigned char* in = msg(q, src);
      const LT* labs = msg_lab(in);
      if (sweep > 1 && src != rank) wait_message(q, src, sub == 0);
      uint64_t skey = ~0ull;     // this warp's best NPath sink candidate
      int cnt = 0;               // improved labels of the sender (sub 0)
      if (WPS == 1) {
        // one warp per sender: per column block and 32-slot block, the
        // sender's labels are compacted into the warp's list and relaxed
        const int nsb = sweep > 1 ? (w + 31) / 32 : 1;
        for (int cb = 0; cb < ncb; ++cb) {
          const int cl = cb * 32 + lane;
          const bool colok = cl < wr && !(sink_here && c0 + cl == j);
          LT bl = kNoLab;
          int32_t bu = -1;
          for (int sb = 0; sb < nsb; ++sb) {
            LT l = 0;
            bool valid = lane == 0 && src == 0;   // sweep 1: the source alone
            if (sweep > 1) {
              const int s = sb * 32 + lane;
              l = s < w ? labs[s] : kNoLab;
              valid = l != kNoLab;
            }
            unsigned bits = __ballot_sync(0xffffffffu, valid);
            if (cb == 0) cnt += __popc(bits);
            if (WPS > 1) {   // the sender's entries are shared among its warps
              valid = valid && (int)(__popc(bits & lt) % WPS) == sub;
              bits = __ballot_sync(0xffffffffu, valid);
            }
            const int32_t u = (sweep > 1 ? src * w + sb * 32 : j) + lane;
            if (cb == 0 && sink_here) {   // Def. 10 (c): q_u() - q_{s*}()
              uint64_t key = ~0ull;
              if (valid && u != j) key = pack_key((int64_t)l + (s_slack[u] >= 0 ? s_pen[u] : 0) - pen_j, u);
  #pragma unroll
              for (int off = 16; off > 0; off >>= 1)
                key = min(key, (uint64_t)__shfl_xor_sync(0xffffffffu, key, off));
              skey = min(skey, key);
            }
            const int n = __popc(bits);
            if (n == 0) continue;
            __syncwarp();   // earlier reads of the list are done
            if (valid) el[__popc(bits & lt)] = Ent{l, u};
            __syncwarp();
            if (tsm_on) {
              if (strict) relax_list<true, true>(el, n, cl, colok, bl, bu);
              else relax_list<false, true>(el, n, cl, colok, bl, bu);
            } else {
              if (strict) relax_list<true, false>(el, n, cl, colok, bl, bu);
              else relax_list<false, false>(el, n, cl, colok, bl, bu);
            }
          }
          if (cl < w) red[warp * RS + cl] = bu < 0 ? ~0ull : pack_key(bl, bu);
        }
      } else {
        // The sender's slots in groups of 32 * WPS: each group's entries are
        // dealt round-robin to the sender's WPS warps (at most 32 each), put
        // into the warp's list once, and relaxed into every owned column block;
        // the warp's row of `red` keeps its minimum per column (stored once
        // when there is one group, the usual case of 32 columns per CTA).
        const int gslots = 32 * WPS;
        const int ngroups = sweep > 1 ? (w + gslots - 1) / gslots : 1;
        if (ngroups > 1)
          for (int cl = lane; cl < w; cl += 32) red[warp * RS + cl] = ~0ull;
        for (int g = 0; g < ngroups; ++g) {
          int n = 0, seen = 0;
          __syncwarp();   // earlier reads of the list are done
          for (int sb = g * gslots; sb < min(w, (g + 1) * gslots) || (sweep == 1 && sb == 0);
               sb += 32) {
            LT l = 0;
            bool valid = lane == 0 && src == 0;   // sweep 1: the source alone
            if (sweep > 1) {
              const int s = sb + lane;
              l = s < w ? labs[s] : kNoLab;
              valid = l != kNoLab;
            }
            const unsigned bits = __ballot_sync(0xffffffffu, valid);
            cnt += __popc(bits);
            const bool mine = valid && (int)((seen + __popc(bits & lt)) & (WPS - 1)) == sub;
            seen += __popc(bits);
            const unsigned mb = __ballot_sync(0xffffffffu, mine);
            const int32_t u = (sweep > 1 ? src * w + sb : j) + lane;
            if (mine) el[n + __popc(mb & lt)] = Ent{l, u};
            n += __popc(mb);
            if (sink_here) {   // Def. 10 (c): q_u() - q_{s*}()
              uint64_t key = ~0ull;
              if (mine && u != j) key = pack_key((int64_t)l + (s_slack[u] >= 0 ? s_pen[u] : 0) - pen_j, u);
  #pragma unroll
              for (int off = 16; off > 0; off >>= 1)
                key = min(key, (uint64_t)__shfl_xor_sync(0xffffffffu, key, off));
              skey = min(skey, key);
            }
            if (sweep == 1) break;
          }
          __syncwarp();
          if (n == 0) {
            if (ngroups == 1)
              for (int cl = lane; cl < w; cl += 32) red[warp * RS + cl] = ~0ull;
            continue;
          }
          for (int cb = 0; cb < ncb; ++cb) {
            const int cl = cb * 32 + lane;
            const bool colok = cl < wr && !(sink_here && c0 + cl == j);
            LT bl = kNoLab;
            int32_t bu = -1;
            if (tsm_on) {
              if (strict) relax_list<true, true>(el, n, cl, colok, bl, bu);
              else relax_list<false, true>(el, n, cl, colok, bl, bu);
            } else {
              if (strict) relax_list<true, false>(el, n, cl, colok, bl, bu);
              else relax_list<false, false>(el, n, cl, colok, bl, bu);
            }
            if (cl < w) {
              const uint64_t key = bu < 0 ? ~0ull : pack_key(bl, bu);
              red[warp * RS + cl] = ngroups == 1 ? key : min(red[warp * RS + cl], key);
            }
          }
        }
      }
      if (lane == 0) s_rsink[warp] = skey;
      if (sweep > 1 && sub == 0 && lane == 0) {   // the sender's tail, for the decisions
        s_tail[2 * src] = cnt;
        s_tail[2 * src + 1] = *msg_merge(in);
        if (src == owner_j) s_misc[MS_SINK_IN] = (int64_t)*msg_sink(in);
      }
      if (tmr) B->t_rloop += clock_cycles() - t0;
      __syncthreads();
      const uint64_t t1 = tmr ? clock_cycles() : 0;
      // ---- decisions on the messages of sweep - 1 (the same in every CTA)
      if (sweep > 1) {
        mph ^= 1u << q;
        const int total = __reduce_add_sync(0xffffffffu, lane < C ? s_tail[2 * lane] : 0);
        const bool any_merge =
            __ballot_sync(0xffffffffu, lane < C && s_tail[2 * lane + 1] != 0) != 0u;
        if (tmr) front_stat(total);
        const uint64_t sink_key = (uint64_t)s_misc[MS_SINK_IN];
        const bool sink_chg = sink_key != kNoKey;
        if (sink_chg) {
          sink_dist = key_label(sink_key);
          sink_par = (int32_t)(sink_key & 0xffffu);
        }
        if (s_misc[MS_ABORT] != 0) { result = -2; break; }   // exchange timed out
        if (sweep == 2 && allow_skip && !any_merge) {
          // T is unchanged since the last round, whose Gamma had no negative
          // cycle (Lemmas 1/2): the NegCycle sink label cannot be negative.
          if (rank == 0 && tid == 0) B->skipped++;
          result = 0;
          skipped_bf = true;
          break;
        }
        if (total == 0 && !sink_chg) {   // sweep - 1 changed nothing: converged
          if (rank == 0 && tid == 0) {
            B->bf_calls++;
            B->bf_sweeps += sweep - 1;
            B->bf_max = max(B->bf_max, (int64_t)(sweep - 1));
          }
          result = sink_dist < 0 ? 1 : 0;
          break;
        }
        if (sweep - 1 >= k + 1) { result = -1; break; }
      }
      // ---- combine the warps' minima per owned column, record, write the message
      unsigned char* my = msg(pb, rank);
      LT* lab = msg_lab(my);
      for (int base = 0; base < w; base += 2 * kWarps) {
        const int cl = base + 2 * warp + (lane >> 4);
        const int sw = lane & 15;
        uint64_t best = ~0ull;
        if (cl < w) best = sink_here && c0 + cl == j ? s_rsink[sw] : red[sw * RS + cl];
#pragma unroll
        for (int off = 8; off > 0; off >>= 1)
          best = min(best, (uint64_t)__shfl_xor_sync(0xffffffffu, best, off));
        if (sw == 0 && cl < w) lab[cl] = cl < wr ? record(cl, best, j, sink_dist, sweep, my) : kNoLab;
      }
      if (tid == 0) {
        *msg_merge(my) = merged ? 1 : 0;
        if (rank != owner_j) *msg_sink(my) = kNoKey;
        s_misc[MS_SINK_IN] = (int64_t)kNoKey;
      }
      __syncthreads();   // the message is complete
      const uint64_t t2 = tmr ? clock_cycles() : 0;
      if (C > 1 && warp < C - 1 && lane == 0) {   // warp p copies the message to the p-th other CTA
        const uint32_t peer = (uint32_t)(warp < rank ? warp : warp + 1);
        fence_proxy_async_smem();
        bulk_copy_to_cta(dsmem_addr(my, peer), my, mbytes, dsmem_addr(mbar(pb, rank), peer));
      }
      // the allotment of the round's unit enters the member lists off the
      // sweep's critical path (every CTA finished reading them once the
      // messages of sweep 1 were in)
      if (sweep == 2) commit_pending();
      if (tmr) {
        const uint64_t t3 = clock_cycles();
        B->t_relax += t1 - t0;
        B->t_sync += t2 - t1;
        B->t_gather += t3 - t2;
      }
      buf ^= 1;
    }
    commit_pending();   // if the call ended at its first decision
    if (tid == 0) {
      s_misc[MS_SINK_DIST] = sink_dist;
      s_misc[MS_SINK_PAR] = sink_par;
      s_misc[MS_MERGE_ANY] = skipped_bf ? 0 : 1;   // 1: the labels converged
    }
    __syncthreads();
    // the path walk reads the owners' parent arrays: order their writes
    if (result > 0 && C > 1) cluster_sync_all();
    return result;
  }

  // Relaxes the frontier entries slice, slice + step, ... (node order) into
  // owned column cl, folding into (bl, bu) (one-CTA clusters).
  template <bool STRICT, bool TSM>
  __device__ __forceinline__ void relax_front(const Ent* fr, int nfront, int slice, int step,
                                              int cl, bool colok, LT& bl, int32_t& bu) const {
    constexpr int32_t inf = TSM ? kTsInf : kTInf;
    constexpr int U = 4;
    int f = slice;
    for (; f + (U - 1) * step < nfront; f += U * step) {
      Ent e[U];
      int32_t t[U];
#pragma unroll
      for (int q = 0; q < U; ++q) e[q] = fr[f + q * step];
#pragma unroll
      for (int q = 0; q < U; ++q) t[q] = colok ? edge<TSM>(e[q].u, cl) : inf;
#pragma unroll
      for (int q = 0; q < U; ++q) {
        if (STRICT) t[q] = strict_cost(t[q], e[q].u, inf);
        const LT c = e[q].l + (LT)t[q];
        if (t[q] != inf && c < bl) { bl = c; bu = e[q].u; }
      }
    }
    for (; f < nfront; f += step) {
      const Ent e = fr[f];
      int32_t t = colok ? edge<TSM>(e.u, cl) : inf;
      if (STRICT) t = strict_cost(t, e.u, inf);
      const LT c = e.l + (LT)t;
      if (t != inf && c < bl) { bl = c; bu = e.u; }
    }
  }

  // The same Bellman-Ford for a one-CTA cluster: no messages.  The frontier
  // (the labels that improved in the last sweep, in node order) is one list
  // in shared memory; the warps split into column blocks of 32 owned columns
  // and, per block, into slices of the frontier; the slices' minima are
  // combined per column, the improved labels recorded and compacted into
  // the next frontier in node order.
  __device__ int bellman_ford_1cta(int32_t j, bool npath, bool merged, bool allow_skip) {
    Ent* fr = reinterpret_cast<Ent*>(s_inbox);   // the inbox is unused without peers
    for (int cl = tid; cl < w; cl += kThreads) {
      s_dist[cl] = kDInf;
      s_hop[cl] = -1;
      s_par[cl] = -1;
    }
    if (tid == 0) fr[0] = Ent{0, j};
    __syncthreads();
    const int32_t pen_j = npath ? qlast(j) : 0;
    const bool strict = flags & OPT_STRICT;
    const int lane = tid & 31, warp = tid >> 5;
    const int CB = max(1, (wr + 31) / 32);
    const int WPB = max(1, kWarps / CB);
    const int RS = w + 1;
    uint64_t* red = reinterpret_cast<uint64_t*>(s_red);   // [WPB][RS] per-slice column minima
    int* wcnt = s_tail;                                    // [kWarps] frontier counts
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    int64_t sink_dist = kDInf;
    int32_t sink_par = -1;
    int nfront = 1;
    int result = 0;
    for (int sweep = 1;; ++sweep) {
      const bool tmr = timer();
      const uint64_t t0 = tmr ? clock_cycles() : 0;
      if (tmr) front_stat(nfront);
      // relax: warp (block, slice) over its slice of the frontier
      for (int bw = warp; bw < CB * WPB; bw += kWarps) {
        const int blk = bw / WPB, slice = bw - blk * WPB;
        const int cl = blk * 32 + lane;
        LT bl = kNoLab;
        int32_t bu = -1;
        uint64_t key = ~0ull;
        if (npath && c0 + cl == j) {   // Def. 10 (c): q_u() - q_{s*}()
          for (int f = slice; f < nfront; f += WPB) {
            const Ent e = fr[f];
            if (e.u == j) continue;
            const int64_t t = (int64_t)(s_slack[e.u] >= 0 ? s_pen[e.u] : 0) - pen_j;
            key = min(key, pack_key((int64_t)e.l + t, e.u));
          }
        } else {
          const bool colok = cl < wr;
          if (tsm_on) {
            if (strict) relax_front<true, true>(fr, nfront, slice, WPB, cl, colok, bl, bu);
            else relax_front<false, true>(fr, nfront, slice, WPB, cl, colok, bl, bu);
          } else {
            if (strict) relax_front<true, false>(fr, nfront, slice, WPB, cl, colok, bl, bu);
            else relax_front<false, false>(fr, nfront, slice, WPB, cl, colok, bl, bu);
          }
          if (bu >= 0) key = pack_key(bl, bu);
        }
        if (cl < w) red[slice * RS + cl] = key;
      }
      if (tmr) B->t_rloop += clock_cycles() - t0;
      __syncthreads();
      const uint64_t t1 = tmr ? clock_cycles() : 0;
      // combine the slices per column, record, and compact the improved
      // labels into the next frontier (node order: column order)
      int total = 0;
      bool sink_chg = false;
      for (int base = 0; base < w; base += kThreads) {
        const int cl = base + tid;
        LT l = kNoLab;
        if (cl < wr) {
          uint64_t best = ~0ull;
          for (int sl = 0; sl < WPB; ++sl) best = min(best, red[sl * RS + cl]);
          if (c0 + cl == j) {   // the sink
            if (best != ~0ull && key_label(best) < sink_dist) {
              s_misc[MS_SINK_IN] = (int64_t)best;
              sink_chg = true;
            }
          } else if (best != ~0ull) {
            const int64_t bc = key_label(best);
            if (bc < s_dist[cl]) {
              s_dist[cl] = bc;
              s_hop[cl] = sweep;
              s_par[cl] = (int32_t)(best & 0xffffu);
              l = (LT)bc;
            }
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, l != kNoLab);
        if (lane == 0) wcnt[warp] = __popc(m);
        sink_chg = __syncthreads_or(sink_chg) != 0 || sink_chg;
        const int wc = lane < kWarps ? wcnt[lane] : 0;
        int incl = wc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int o = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += o;
        }
        const int at = total + __shfl_sync(0xffffffffu, incl - wc, warp);
        if (l != kNoLab) fr[at + __popc(m & lt)] = Ent{l, c0 + cl};
        total += __shfl_sync(0xffffffffu, incl, kWarps - 1);
        __syncthreads();   // counts read before the next chunk rewrites them
      }
      if (sink_chg) {
        const uint64_t sk = (uint64_t)s_misc[MS_SINK_IN];
        sink_dist = key_label(sk);
        sink_par = (int32_t)(sk & 0xffffu);
      }
      if (tmr) {
        const uint64_t t2 = clock_cycles();
        B->t_relax += t1 - t0;
        B->t_sync += t2 - t1;
      }
      if (sweep == 1) commit_pending();
      if (sweep == 1 && allow_skip && !merged) {
        // T is unchanged since the last round, whose Gamma had no negative
        // cycle (Lemmas 1/2): the NegCycle sink label cannot be negative.
        if (tid == 0) B->skipped++;
        result = 0;
        if (tid == 0) s_misc[MS_MERGE_ANY] = 0;
        break;
      }
      if (total == 0 && !sink_chg) {
        if (tid == 0) {
          B->bf_calls++;
          B->bf_sweeps += sweep;
          B->bf_max = max(B->bf_max, (int64_t)sweep);
          s_misc[MS_MERGE_ANY] = 1;
        }
        result = sink_dist < 0 ? 1 : 0;
        break;
      }
      if (sweep >= k + 1) { result = -1; break; }
      nfront = total;
    }
    if (tid == 0) {
      s_misc[MS_SINK_DIST] = sink_dist;
      s_misc[MS_SINK_PAR] = sink_par;
    }
    __syncthreads();
    return result;
  }

  // Alg. 4 right after an Alg. 1 that applied nothing: T and the loads are
  // unchanged, and the NPath graph differs from the NCyc graph only in the
  // edges into the sink, which have no successors.  The converged node
  // labels are therefore already the NPath labels, and the sink's label and
  // parent follow from one reduction: the synchronous sweep reaches the
  // minimum first through the predecessors u of smallest hop count (the
  // sweep of u's last change), and among those takes the lowest index.
  // Each CTA reduces over the columns it owns, the partial minima are
  // exchanged, and every CTA combines the same partials.  Returns 1 if the
  // sink label is negative.
  __device__ int npath_from_ncyc(int32_t j) {
    const int32_t pen_j = qlast(j);
    int64_t bc = kDInf;
    uint32_t bhu = 0xffffffffu;   // hop << 16 | node
    auto better = [](int64_t c, uint32_t hu, int64_t bc_, uint32_t bhu_) {
      return c < bc_ || (c == bc_ && hu < bhu_);
    };
    for (int cl = tid; cl < wr; cl += kThreads) {
      const int u = c0 + cl;
      if (u == j || s_dist[cl] >= kDInf) continue;
      const int64_t c = s_dist[cl] + (int64_t)(s_slack[u] >= 0 ? s_pen[u] : 0) - pen_j;
      const uint32_t hu = ((uint32_t)s_hop[cl] << 16) | (uint32_t)u;
      if (better(c, hu, bc, bhu)) { bc = c; bhu = hu; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const int64_t oc = __shfl_xor_sync(0xffffffffu, bc, off);
      const uint32_t ohu = __shfl_xor_sync(0xffffffffu, bhu, off);
      if (better(oc, ohu, bc, bhu)) { bc = oc; bhu = ohu; }
    }
    int64_t* rc = reinterpret_cast<int64_t*>(s_red);
    uint32_t* rhu = reinterpret_cast<uint32_t*>(s_red + 8 * kWarps);
    if ((tid & 31) == 0) { rc[tid >> 5] = bc; rhu[tid >> 5] = bhu; }
    __syncthreads();
    if (tid < C) {   // thread r sends this CTA's partial to CTA r
      for (int i = 0; i < kWarps; ++i)
        if (better(rc[i], rhu[i], bc, bhu)) { bc = rc[i]; bhu = rhu[i]; }
      dsmem_st64(dsmem_addr(s_npart + 2 * rank, tid), bc);
      dsmem_st64(dsmem_addr(s_npart + 2 * rank + 1, tid), (int64_t)bhu);
    }
    cluster_sync_all();
    bc = kDInf;
    bhu = 0xffffffffu;
    for (int r = 0; r < C; ++r) {
      const int64_t c = s_npart[2 * r];
      const uint32_t hu = (uint32_t)s_npart[2 * r + 1];
      if (better(c, hu, bc, bhu)) { bc = c; bhu = hu; }
    }
    if (tid == 0) {
      s_misc[MS_SINK_DIST] = bc;
      s_misc[MS_SINK_PAR] = bc < kDInf ? (int64_t)(bhu & 0xffffu) : -1;
      if (rank == 0) B->npath_reused++;
    }
    __syncthreads();
    return bc < 0 ? 1 : 0;
  }

  // Follow parents from the sink back to the anchor (every CTA does this,
  // reading the parent arrays of the owning CTAs).  Fills s_path with the
  // centers j = p0, p1, ..., p_{m-1}; returns m or -1 if the walk is bad.
  __device__ int walk_path(int32_t j) {
    if (tid == 0) {
      int m = 0;
      bool bad = false;
      int32_t v = (int32_t)s_misc[MS_SINK_PAR];
      for (;;) {
        if (v < 0 || v >= k || m > k) { bad = true; break; }
        s_pathu[m++] = v;    // reversed, temporarily
        if (v == j) break;
        const int owner = v / w;
        v = dsmem_ld32(dsmem_addr(s_par + (v - owner * w), owner));
      }
      if (!bad) for (int i = 0; i < m; ++i) s_path[i] = s_pathu[m - 1 - i];
      s_misc[MS_PATHLEN] = bad ? -1 : m;
    }
    __syncthreads();
    return (int)s_misc[MS_PATHLEN];
  }

  // Apply the transfers of the path (Alg. 1 and Alg. 4, "if cost < 0" branch);
  // then recompute the rows of T of every center on it.  For NCyc every
  // center on the cycle loses one unit and gains one; for NPath the anchor
  // only loses one and the terminal center only gains one.
  __device__ void apply(int32_t j, bool npath, int m) {
    uint64_t t0 = timer() ? clock_cycles() : 0;
    if (tid < 32) {
      // every CTA reads the moved units (T is not written before the
      // barrier below, so all CTAs see the same entries)
      const bool strict = flags & OPT_STRICT;
      for (int i = tid; i < m; i += 32) {
        const int32_t from = s_path[i];
        const int32_t to = (i + 1 < m) ? s_path[i + 1] : (npath ? -1 : j);
        int32_t x = to >= 0 ? __ldcg(I.td + (int64_t)from * k + to) : -1;
        // Alg. 5: a dummy unit moves where the edge cost came from a vacancy
        const bool dummy = strict && to >= 0 && s_slack[from] < 0 &&
                           __ldcg(I.tc + (int64_t)from * k + to) > 0;
        if (dummy) x = -1;
        else if (to >= 0 && (uint32_t)x >= (uint32_t)n) { x = -1; if (rank == 0) B->err0 = ST_ERR_INVARIANT; }
        s_pathu[i] = x;
      }
      __syncwarp();
    }
    if (rank == 0 && tid < 32) {
      const int lane = tid;
      int32_t* ppos = reinterpret_cast<int32_t*>(s_red);   // positions of the outgoing units
      for (int i = lane; i < m; i += 32) ppos[i] = s_pathu[i] >= 0 ? I.pos[s_pathu[i]] : -1;
      __syncwarp();
      // in-place replacements: center p_i swaps its leaving unit for the
      // arriving unit x_{i-1} (cyclically for NCyc)
      for (int i = lane; i < m; i += 32) {
        const int32_t c = s_path[i];
        const int32_t x_out = s_pathu[i];
        const int32_t x_in = (i > 0) ? s_pathu[i - 1] : (npath ? -1 : s_pathu[m - 1]);
        if (x_out >= 0 && x_in >= 0 && ppos[i] >= 0 && ppos[i] < n) {
          int32_t* slot = mslot(c, ppos[i]);
          slot[0] = x_in;
          slot[kPage] = (int32_t)row(x_in)[c];
          I.pos[x_in] = ppos[i];
        }
        if (x_out >= 0) I.assign[x_out] = (i + 1 < m) ? s_path[i + 1] : j;
      }
      __syncwarp();
      if (lane == 0 && (flags & OPT_STRICT)) {
        // centers that only lose or only gain a real unit (the other side of
        // their edge pair is a dummy); pages are shared, so one thread
        for (int i = 0; i < m; ++i) {
          const int32_t c = s_path[i];
          const int32_t x_out = s_pathu[i], x_in = s_pathu[i > 0 ? i - 1 : m - 1];
          if (x_out >= 0 && x_in < 0) {
            list_remove_at(c, ppos[i]);
            I.load[c] -= 1;
          } else if (x_out < 0 && x_in >= 0) {
            list_append(c, x_in, (int32_t)row(x_in)[c]);
            I.load[c] += 1;
          }
        }
      }
      if (lane == 0) {
        if (npath) {
          // the anchor loses x_0, the terminal center gains x_{m-2}
          list_remove_at(j, ppos[0]);
          if (s_pathu[m - 2] >= 0)
            list_append(s_path[m - 1], s_pathu[m - 2], (int32_t)row(s_pathu[m - 2])[s_path[m - 1]]);
          else B->err0 = ST_ERR_INVARIANT;
          I.load[j] -= 1;
          I.load[s_path[m - 1]] += 1;
          B->paths++;
          B->moves += m - 1;
        } else {
          B->cycles++;
          B->moves += m;
        }
        B->delta += s_misc[MS_SINK_DIST];
      }
    }
    if (npath && tid == 0) {   // load and penalty replicas in every CTA
      s_slack[j] -= 1;
      s_slack[s_path[m - 1]] += 1;
      if (I.Q > 1) {
        s_pen[j] = qnext(j);
        s_pen[s_path[m - 1]] = qnext(s_path[m - 1]);
      }
    }
    if ((flags & OPT_STRICT) && tid == 0) {
      for (int i = 0; i < m; ++i) {
        const int32_t x_out = s_pathu[i], x_in = s_pathu[i > 0 ? i - 1 : m - 1];
        if (x_out >= 0 && x_in < 0) s_slack[s_path[i]] -= 1;
        else if (x_out < 0 && x_in >= 0) s_slack[s_path[i]] += 1;
      }
    }
    __syncthreads();
    cluster_sync_all();   // member lists updated before anyone rescans
    uint64_t t1 = timer() ? clock_cycles() : 0;
    for (int i = 0; i < m; ++i) {
      const int32_t x_out = s_pathu[i];
      const int32_t x_in = (i > 0) ? s_pathu[i - 1] : (npath ? -1 : s_pathu[m - 1]);
      rescan_incremental(s_path[i], x_out, x_in);
    }
    if (timer()) {
      const uint64_t t2 = clock_cycles();
      B->t_apply += t1 - t0;
      B->t_rescan += t2 - t1;
    }
  }

  // Row c of T after c lost unit x_out and gained unit x_in (either may be
  // -1), equal to a full rescan of c's new member list:
  //  * columns whose best unit was not x_out keep their minimum over the
  //    remaining members, so only x_in is merged in;
  //  * columns whose best unit was x_out are recomputed over all members;
  //    with many such columns the whole owned row is rescanned instead.
  __device__ void rescan_incremental(int32_t c, int32_t x_out, int32_t x_in) {
    int32_t* s_aff = reinterpret_cast<int32_t*>(s_red);                       // [w]
    unsigned long long* s_best =
        reinterpret_cast<unsigned long long*>(s_red + 4 * ((w + 1) & ~1));   // [naff]
    if (tid == 0) s_misc[MS_NAFF] = 0;
    __syncthreads();
    int32_t in_own = 0;
    const T* rin = nullptr;
    if (x_in >= 0) { rin = row(x_in); in_own = (int32_t)rin[c]; }
    for (int cl = tid; cl < wr; cl += kThreads) {
      const int v = c0 + cl;
      if (v == c) continue;
      const int32_t bd = I.td[(int64_t)c * k + v];
      if (x_out >= 0 && bd == x_out) {
        s_aff[atomicAdd(reinterpret_cast<int*>(&s_misc[MS_NAFF]), 1)] = cl;
      } else if (x_in >= 0) {
        const int32_t t = (int32_t)rin[v] - in_own;
        const int32_t bt = own_cost(c, cl);
        if (lex_less(t, x_in, bt, bd)) set_entry(c, cl, t, x_in);
      }
    }
    __syncthreads();
    const int naff = (int)s_misc[MS_NAFF];
    if (naff == 0) return;
    if (naff * 4 > wr) { rescan(c); return; }
    for (int a = tid; a < naff; a += kThreads) s_best[a] = ~0ull;
    __syncthreads();
    const int32_t s = __ldcg(I.seg_size + c);
    const int stride = kThreads / naff;
    const int a = tid % naff, i0 = tid / naff;
    if (i0 < stride) {
      const int v = c0 + s_aff[a];
      unsigned long long best = ~0ull;
      constexpr int U = 4;
      for (int32_t base = i0; base < s; base += U * stride) {
        int32_t dd[U], own[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t idx = base + u * stride;
          const int32_t* sl = idx < s ? mslot(c, idx) : nullptr;
          dd[u] = sl ? __ldcg(sl) : -1;
          own[u] = sl ? __ldcg(sl + kPage) : 0;
          if ((uint32_t)dd[u] >= (uint32_t)n) dd[u] = -1;   // guard: corrupt entry
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (dd[u] < 0) continue;
          const int32_t t = (int32_t)row(dd[u])[v] - own[u];
          const unsigned long long key =
              ((unsigned long long)(uint32_t)(t + (int64_t)2147483648LL) << 32) | (uint32_t)dd[u];
          best = min(best, key);
        }
      }
      if (best != ~0ull) atomicMin(&s_best[a], best);
    }
    __syncthreads();
    for (int b = tid; b < naff; b += kThreads) {
      const unsigned long long e = s_best[b];
      if (e == ~0ull) set_entry(c, s_aff[b], kTInf, -1);
      else set_entry(c, s_aff[b], (int32_t)((int64_t)(e >> 32) - 2147483648LL), (int32_t)(e & 0xffffffffu));
    }
    if (rank == 0 && tid == 0) B->col_rows += s;
    __syncthreads();
  }

  // ---------------------------------------------------------- the loop --
  __device__ void run_rounds() {
    const uint64_t tstart = rank == 0 && tid == 0 ? gtimer_ns() : 0;
    const uint64_t cstart = rank == 0 && tid == 0 ? clock_cycles() : 0;
    const int64_t r_begin = I.ctl[CTL_ROUNDS];
    const int64_t r_end = min((int64_t)n, I.ctl[CTL_TARGET]);
    for (int v = tid; v < k; v += kThreads) {
      s_slack[v] = __ldcg(I.load + v) - __ldg(I.cap + v);
      s_pen[v] = qval(v, s_slack[v] + 1);
    }
    if (rank == 0 && tid == 0) {
      B->delta = I.ctl[CTL_DELTA];
      B->free_top = I.ctl[CTL_FREE_TOP];
      B->cycles = B->paths = B->bf_calls = B->bf_sweeps = B->bf_max = B->moves = B->skipped = B->rows = 0;
      B->t_merge = B->t_relax = B->t_sync = B->t_gather = B->t_apply = B->t_rescan = 0;
      B->t_rloop = B->t_rred = 0;
      B->err0 = 0;
      B->npath_reused = 0;
      B->col_rows = 0;
      B->front_sum = 0;
      for (int h = 0; h < 6; ++h) B->front_hist[h] = 0;
    }
    load_slice();
    __syncthreads();
    const bool allow_skip = !(flags & OPT_NO_NCYC_SKIP);
    int64_t status = ST_OK;
    int64_t r = r_begin;
    int nchk = 0;
    for (; r < r_end; ++r) {
      // Time-sliced launches yield between rounds once the quantum is spent.
      // CTA 0 decides; the flag alternates between two slots, so a slot is
      // rewritten only after the barrier that follows every CTA's read of it.
      if (quantum_on && r > r_begin && (r - r_begin) % kQuantumCheck == 0) {
        const int slot = MS_STOP0 + (nchk & 1);
        ++nchk;
        if (rank == 0 && tid == 0) s_misc[slot] = gtimer_ns() >= B->deadline ? 1 : 0;
        cluster_sync_all();
        if (dsmem_ld64(dsmem_addr(&s_misc[slot], 0)) != 0) break;
      }
      // Alg. 2 (extract-min, allot, objective update): next unit of the MinDistance order goes
      // to its most suitable center; pay the penalty if it had no vacancy.
      const uint64_t tm0 = timer() ? clock_cycles() : 0;
      const int32_t d = __ldcg(I.order + r);
      if ((uint32_t)d >= (uint32_t)n) { status = ST_ERR_INVARIANT; break; }   // uniform guard
      const bool strict = flags & OPT_STRICT;
      const int32_t j = strict ? strict_target(d) : __ldcg(I.smin + d);
      if ((uint32_t)j >= (uint32_t)k) { status = ST_ERR_INVARIANT; break; }
      const bool over = !strict && s_slack[j] >= 0;
      const int32_t q_over = over ? s_pen[j] : 0;   // q_j(load - cap + 1), Alg. 2
      const bool merged = merge_row(d, j);
      if (tid == 0) {
        s_slack[j] += 1;
        if (!strict && I.Q > 1) s_pen[j] = qnext(j);
      }
      if (rank == 0 && tid == 0) {
        // Member lists are touched only after the next cluster barrier (the
        // first Bellman-Ford sweep), when every CTA has finished reading
        // them for the previous round's rescans.
        pending_own = (int32_t)row(d)[j];
        B->delta += (int64_t)pending_own + q_over;
        if (timer()) B->t_merge += clock_cycles() - tm0;
      }
      __syncthreads();
      // Alg. 1 at j
      pending_d = d;
      pending_j = j;
      int res = C == 1 ? bellman_ford_1cta(j, false, merged, allow_skip)
                       : bellman_ford(j, false, merged, allow_skip);
      if (res < 0) { status = res == -2 ? ST_ERR_TIMEOUT : ST_ERR_INVARIANT; break; }
      // labels converged (not skipped) and nothing applied: Alg. 4 can reuse them
      const bool reusable = (s_misc[MS_MERGE_ANY] != 0 || !allow_skip) && res == 0;
      if (res > 0) {
        const int m = walk_path(j);
        if (m < 2) { status = ST_ERR_INVARIANT; break; }
        apply(j, false, m);
      }
      // Alg. 4 at j when the allotment overloaded it
      if (over) {
        res = reusable && !(flags & OPT_NO_NPATH_REUSE) ? npath_from_ncyc(j)
              : C == 1 ? bellman_ford_1cta(j, true, true, false)
                       : bellman_ford(j, true, true, false);
        if (res < 0) { status = res == -2 ? ST_ERR_TIMEOUT : ST_ERR_INVARIANT; break; }
        if (res > 0) {
          const int m = walk_path(j);
          if (m < 2) { status = ST_ERR_INVARIANT; break; }
          apply(j, true, m);
        }
      }
    }
    __syncthreads();
    cluster_sync_all();
    if (rank == 0 && tid == 0) {
      I.ctl[CTL_ROUNDS] = r;
      I.ctl[CTL_DELTA] = B->delta;
      I.ctl[CTL_FREE_TOP] = B->free_top;
      I.ctl[CTL_STATUS] = status != ST_OK ? status : B->err0;
      I.ctl[CTL_CYCLES] += B->cycles;
      I.ctl[CTL_PATHS] += B->paths;
      I.ctl[CTL_BF_CALLS] += B->bf_calls;
      I.ctl[CTL_BF_SWEEPS] += B->bf_sweeps;
      I.ctl[CTL_BF_MAX] = max(I.ctl[CTL_BF_MAX], B->bf_max);
      I.ctl[CTL_MOVES] += B->moves;
      I.ctl[CTL_NCYC_SKIPPED] += B->skipped;
      I.ctl[CTL_ROWS_SCANNED] += B->rows;
      I.ctl[CTL_T_TOTAL] += gtimer_ns() - tstart;
      I.ctl[CTL_T_CYCLES] += clock_cycles() - cstart;
      I.ctl[CTL_T_MERGE] += B->t_merge;
      I.ctl[CTL_T_RELAX] += B->t_relax;
      I.ctl[CTL_T_SYNC] += B->t_sync;
      I.ctl[CTL_T_GATHER] += B->t_gather;
      I.ctl[CTL_T_APPLY] += B->t_apply;
      I.ctl[CTL_T_RESCAN] += B->t_rescan;
      I.ctl[CTL_T_RLOOP] += B->t_rloop;
      I.ctl[CTL_TSM_ON] = tsm_on ? 1 : 0;
      I.ctl[CTL_T_RRED] += B->t_rred;
      I.ctl[CTL_NPATH_REUSED] += B->npath_reused;
      I.ctl[CTL_COL_ROWS] += B->col_rows;
      I.ctl[CTL_FRONT_SUM] += B->front_sum;
      for (int h = 0; h < 6; ++h) I.ctl[CTL_FRONT_HIST + h] += B->front_hist[h];
    }
  }

  // CTA 0 records the allotment of the round's unit (assign, member list,
  // global load) right after the first sweep's barrier, when no CTA still
  // reads member lists of the previous round.
  __device__ __forceinline__ void commit_pending() {
    if (pending_d >= 0) {
      if (rank == 0 && tid == 0) {
        I.assign[pending_d] = pending_j;
        list_append(pending_j, pending_d, pending_own);
        I.load[pending_j] += 1;
      }
      pending_d = -1;
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
asral_cluster_kernel(const DevInst* __restrict__ insts, int ninst, int* work_counter, int flags,
                     uint64_t quantum_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevInst s_inst;
  __shared__ Book s_book;
  __shared__ __align__(8) uint64_t s_mbar[2 * kMaxCluster];
  Solver<T> S(s_inst);
  S.B = &s_book;
  S.tid = threadIdx.x;
  S.rank = (int)cluster_rank();
  S.C = (int)cluster_nrank();
  S.flags = flags;
  S.buf = 0;
  S.s_mbar = s_mbar;
  S.mph = 0;
  if (S.tid < 2 * kMaxCluster) mbar_init(&s_mbar[S.tid], 1);
  if (S.tid == 0) mbar_fence_init();   // the cluster barrier before the first instance publishes them
  S.quantum_on = quantum_ns != 0;
  if (S.rank == 0 && S.tid == 0) s_book.deadline = S.quantum_on ? gtimer_ns() + quantum_ns : 0;
  int64_t* s_item = reinterpret_cast<int64_t*>(smem);   // first 16 bytes: work item
  unsigned char* base = smem + 16;
  const uint32_t avail = dyn_smem_bytes();
  for (;;) {
    if (S.rank == 0 && S.tid == 0) {
      // Next instance with rounds left and no error; none once the quantum
      // is spent.  Only this thread decides, so the cluster agrees.
      int it = ninst;
      if (!S.quantum_on || gtimer_ns() < s_book.deadline) {
        for (;;) {
          it = atomicAdd(work_counter, 1);
          if (it >= ninst) break;
          const int64_t* c = insts[it].ctl;
          const int64_t target = min((int64_t)insts[it].n, __ldcg(c + CTL_TARGET));
          if (__ldcg(c + CTL_STATUS) == 0 &&
              (__ldcg(c + CTL_PROLOGUE) == 0 || __ldcg(c + CTL_ROUNDS) < target))
            break;
        }
      }
      s_item[0] = it;
    }
    __syncthreads();
    cluster_sync_all();
    const int item = (int)dsmem_ld64(dsmem_addr(s_item, 0));
    cluster_sync_all();
    if (item >= ninst) break;
    if (S.tid == 0) s_inst = insts[item];
    __syncthreads();
    S.cm = static_cast<const T*>(S.I.cm);
    S.n = S.I.n;
    S.k = S.I.k;
    S.w = own_width(S.k, S.C, Solver<T>::VPL);
    S.ws = slice_stride(S.w, (int)sizeof(T));
    S.c0 = S.rank * S.w;
    S.c1 = min(S.k, S.c0 + S.w);
    S.wr = max(0, S.c1 - S.c0);
    const Layout L = make_layout(S.k, S.C, (int)sizeof(T));
    // same decision in every CTA of the cluster
    S.tsm_on = 16 + L.total <= avail && !(flags & OPT_NO_TC_SMEM);
    S.s_dist = reinterpret_cast<int64_t*>(base + L.dist);
    S.s_hop = reinterpret_cast<int32_t*>(base + L.hop);
    S.s_slack = reinterpret_cast<int32_t*>(base + L.slack);
    S.s_pen = reinterpret_cast<int32_t*>(base + L.pen);
    S.s_par = reinterpret_cast<int32_t*>(base + L.par);
    S.s_inbox = base + L.inbox;
    S.mbytes = L.msg;
    S.s_tail = reinterpret_cast<int32_t*>(base + L.tail);
    S.s_rsink = reinterpret_cast<uint64_t*>(base + L.rsink);
    S.s_elist = base + L.elist;
    S.s_npart = reinterpret_cast<int64_t*>(base + L.npart);
    S.s_path = reinterpret_cast<int32_t*>(base + L.path);
    S.s_pathu = reinterpret_cast<int32_t*>(base + L.pathu);
    S.s_misc = reinterpret_cast<int64_t*>(base + L.misc);
    S.s_red = base + L.red;
    S.s_tc = reinterpret_cast<typename Solver<T>::TS*>(base + L.tsm);
    if (S.I.ctl[CTL_PROLOGUE] == 0) {
      const uint64_t t0 = gtimer_ns();
      S.prologue();
      if (S.rank == 0 && S.tid == 0) {
        S.I.ctl[CTL_FREE_TOP] = S.I.npages;
        S.I.ctl[CTL_ROUNDS] = 0;
        S.I.ctl[CTL_DELTA] = 0;
        S.I.ctl[CTL_PROLOGUE] = 1;
        S.I.ctl[CTL_T_PROLOGUE] += gtimer_ns() - t0;
      }
      __syncthreads();
      cluster_sync_all();
    }
    S.run_rounds();
  }
}

// Shared-memory bytes of one CTA for an instance with k centers on C-CTA
// clusters (includes the 16-byte work-item slot).  with_slice: also the
// owned cost slice.
size_t solver_smem_bytes(int32_t k, int C, int elem_bytes, bool with_slice) {
  const Layout L = make_layout(k, C, elem_bytes);
  return 16 + (with_slice ? L.total : L.base_total);
}

int solver_max_k(int C, int elem_bytes) {
  // the rescan maps every owned 16-byte column group to a thread
  return kThreads * (16 / elem_bytes) * C;
}

template <typename T>
cudaError_t prepare_solver_t(int C, size_t smem);

template <typename T>
cudaError_t launch_solver_t(const DevInst* d_insts, int ninst, int* d_counter, int C,
                            int nclusters, size_t smem, int flags, cudaStream_t st,
                            uint64_t quantum_ns, bool set_attrs) {
  auto kern = asral_cluster_kernel<T>;
  if (set_attrs) {
    const cudaError_t e = prepare_solver_t<T>(C, smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * nclusters), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, d_insts, ninst, d_counter, flags, quantum_ns);
}

// Kernel attributes only ever grow (a launch needs at least its own dynamic
// shared memory; concurrent callers must not lower what another one set).
// Attributes belong to the current device, so the high-water marks are kept
// per device.
template <typename T>
cudaError_t prepare_solver_t(int C, size_t smem) {
  constexpr int kDevs = 64;
  static std::mutex mu;
  static size_t cur_smem[kDevs] = {};
  static bool non_portable[kDevs] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  auto kern = asral_cluster_kernel<T>;
  if (smem > cur_smem[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cur_smem[dev] = smem;
  }
  if (C > 8 && !non_portable[dev]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    non_portable[dev] = true;
  }
  return cudaSuccess;
}

cudaError_t prepare_solver(int C, int elem_bytes, size_t smem) {
  return elem_bytes == 2 ? prepare_solver_t<int16_t>(C, smem) : prepare_solver_t<int32_t>(C, smem);
}

cudaError_t launch_solver(const DevInst* d_insts, int ninst, int* d_counter, int C,
                          int nclusters, int elem_bytes, size_t smem, int flags,
                          cudaStream_t st, uint64_t quantum_ns, bool set_attrs) {
  if (elem_bytes == 2)
    return launch_solver_t<int16_t>(d_insts, ninst, d_counter, C, nclusters, smem, flags, st,
                                    quantum_ns, set_attrs);
  return launch_solver_t<int32_t>(d_insts, ninst, d_counter, C, nclusters, smem, flags, st,
                                  quantum_ns, set_attrs);
}

// Largest number of co-resident clusters of size C for this kernel.
template <typename T>
static int max_clusters_t(int C, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  auto kern = asral_cluster_kernel<T>;
  if (prepare_solver_t<T>(C, smem) != cudaSuccess) return -1;
  int num = 0;
  return cudaOccupancyMaxActiveClusters(&num, kern, &cfg) == cudaSuccess ? num : -1;
}

int solver_max_clusters(int C, int elem_bytes, size_t smem) {
  return elem_bytes == 2 ? max_clusters_t<int16_t>(C, smem) : max_clusters_t<int32_t>(C, smem);
}

}  // namespace lbdd
