// Persistent ASRAL solver: one thread-block cluster runs whole solves.
//
// Paper: Ramnath et al., "Load Balanced Demand Distribution under Overload
// Penalties" (arXiv 2304.06543).  Alg. 1 (ASRAL main loop), Alg. 2 (Negative
// Cycle Refinement), Alg. 3 (Negative Path Refinement, Appendix A), Defs. 4-6
// (allotment subspace multigraph, NCyc and NPath graphs), Alg. 4 (parallel
// Bellman-Ford).
//
// GB300 design (not the paper's JCuda design, which copied the graph to the
// GPU and synchronised the host after every Bellman-Ford sweep):
//  * the whole solve - prologue, all n rounds - runs inside one launch on one
//    cluster of C CTAs; nothing returns to the host between rounds;
//  * the best-transfer table T (the heap tops of the paper's BestTransHeaps)
//    is a dense k x k table in global memory, column-partitioned: CTA r of the
//    cluster owns columns [r*w, r*w + w) of every row and is the only CTA
//    that reads or writes them, so Bellman-Ford relaxations, merges and
//    segment rescans need no cross-CTA traffic for T;
//  * Bellman-Ford is the synchronous form with a frontier (only labels that
//    changed in the previous sweep can improve a label); each sweep publishes
//    the owned label changes in shared memory and the CTAs read each other's
//    changes through distributed shared memory after one cluster barrier;
//  * when a unit changes center, the rows of T of the centers on the path are
//    recomputed from their member lists (segment rescan), reading CM rows with
//    16-byte vector loads.
// Tie-breaking is canonical and identical to the CPU oracle: (cost, unit)
// lexicographic in T, lowest predecessor index on equal Bellman-Ford labels.
#include "lbdd_device.cuh"

namespace lbdd {

struct Layout {
  uint32_t dist, load, front, par, outv, outd, outctl, path, pathu, misc, red, total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline int32_t own_width(int32_t k, int32_t C, int32_t vpl) {
  int32_t w = (k + C - 1) / C;
  return (w + vpl - 1) / vpl * vpl;
}

constexpr uint32_t kRedBytes = kThreads * 8 * 8;  // rescan partials, int16 CM

__host__ __device__ inline Layout make_layout(int32_t k, int32_t C, int32_t vpl) {
  Layout L;
  uint32_t o = 0;
  const uint32_t w = (uint32_t)own_width(k, C, vpl);
  const uint32_t ku = (uint32_t)k;
  L.dist = o;   o = align16(o + 8u * ku);
  L.load = o;   o = align16(o + 4u * ku);
  L.front = o;  o = align16(o + 4u * (ku + 1));
  L.par = o;    o = align16(o + 4u * w);
  L.outv = o;   o = align16(o + 2u * 4u * w);
  L.outd = o;   o = align16(o + 2u * 8u * w);
  L.outctl = o; o = align16(o + 2u * 8u * 8u);
  L.path = o;   o = align16(o + 4u * (ku + 2));
  L.pathu = o;  o = align16(o + 4u * (ku + 2));
  L.misc = o;   o = align16(o + 8u * 16u);
  L.red = o;    o = align16(o + kRedBytes);
  L.total = o;
  return L;
}

// Slots of the per-buffer exchange control block.
enum { OC_COUNT = 0, OC_SINK_CHANGED, OC_SINK_DIST, OC_SINK_PAR, OC_MERGE_CHANGED };
// Slots of the per-CTA scalar block.
enum { MS_NFRONT = 0, MS_SINK_DIST, MS_SINK_PAR, MS_CNT, MS_FLAG, MS_TOTAL, MS_PATHLEN,
       MS_ITEM, MS_SINK_CHG, MS_MERGE_ANY, MS_BAD };

template <typename T>
struct Solver {
  static constexpr int VPL = 16 / (int)sizeof(T);

  DevInst I;
  const T* cm;
  int32_t n, k, C, rank, w, c0, c1, wr;
  int tid;
  int flags;
  int64_t* s_dist;
  int32_t* s_load;
  int32_t* s_front;
  int32_t* s_par;
  int32_t* s_outv;    // [2][w]
  int64_t* s_outd;    // [2][w]
  int64_t* s_outctl;  // [2][8]
  int32_t* s_path;
  int32_t* s_pathu;
  int64_t* s_misc;
  unsigned char* s_red;
  int buf;            // exchange buffer parity, advances every sweep

  // rank-0 bookkeeping, valid in thread 0 of CTA 0 only
  int64_t delta, free_top, cycles, paths, bf_calls, bf_sweeps, bf_max, moves, skipped, rows;
  int64_t err0 = 0;   // CTA 0 thread 0: a guard tripped (corrupt state; never expected)

  __device__ __forceinline__ const T* row(int32_t d) const { return cm + (int64_t)d * I.ld; }

  __device__ __forceinline__ int32_t* mslot(int32_t c, int32_t idx) const {
    int32_t page = __ldcg(I.page_tab + (int64_t)c * I.max_pages + (idx >> kPageShift));
    return I.pool + ((int64_t)page << kPageShift) + (idx & (kPage - 1));
  }

  // Member-list primitives, called by one thread of CTA 0 only.
  __device__ void list_append(int32_t c, int32_t d) {
    int32_t idx = I.seg_size[c];
    if (c < 0 || c >= k || d < 0 || d >= n || idx < 0 || idx >= n) { err0 = ST_ERR_INVARIANT; return; }
    if ((idx & (kPage - 1)) == 0) {
      if (free_top <= 0) { err0 = ST_ERR_INVARIANT; return; }
      int32_t page = I.free_stack[--free_top];
      I.page_tab[(int64_t)c * I.max_pages + (idx >> kPageShift)] = page;
    }
    *mslot(c, idx) = d;
    I.pos[d] = idx;
    I.seg_size[c] = idx + 1;
  }
  // Remove the unit stored at index idx of c's list (its position before
  // any move of this path was applied).
  __device__ void list_remove_at(int32_t c, int32_t idx) {
    int32_t last = I.seg_size[c] - 1;
    if (c < 0 || c >= k || idx < 0 || idx > last || free_top >= I.npages) {
      err0 = ST_ERR_INVARIANT;
      return;
    }
    if (idx != last) {
      int32_t moved = *mslot(c, last);
      *mslot(c, idx) = moved;
      I.pos[moved] = idx;
    }
    if ((last & (kPage - 1)) == 0)
      I.free_stack[free_top++] = I.page_tab[(int64_t)c * I.max_pages + (last >> kPageShift)];
    I.seg_size[c] = last;
  }

  // ------------------------------------------------------------ prologue --
  // Alg. 1 line 1: s_min(d) = lowest-index minimum of CM row d; the
  // MinDistance heap's extraction order = stable sort of d by CM(d, s_min).
  __device__ void prologue() {
    const int lane = tid & 31, warp = tid >> 5;
    int32_t* keys0 = I.sort_tmp;
    int32_t* vals0 = I.sort_tmp + n;
    uint32_t kmax = 0;
    for (int64_t d = (int64_t)rank * kWarps + warp; d < n; d += (int64_t)C * kWarps) {
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
    if (rank == 0) sort_order();
    __syncthreads();
    cluster_sync_all();
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
      for (int64_t i = tid; i < n; i += kThreads) atomicAdd(&s_off[(sk[i] >> shift) & 255], 1);
      __syncthreads();
      if (tid == 0) {
        int32_t run = 0;
        for (int b = 0; b < 256; ++b) { int32_t c = s_off[b]; s_off[b] = run; run += c; }
      }
      __syncthreads();
      for (int64_t base = 0; base < n; base += kThreads) {
        const int64_t i = base + tid;
        const bool valid = i < n;
        const int32_t key = valid ? sk[i] : 0, val = valid ? sv[i] : 0;
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

  // ---------------------------------------------------- best-transfer T --
  // Alg. 1 line 6: unit d joins center j; its k-1 transfer edges
  // CM(d, v) - CM(d, j) (Def. 4) enter the per-pair minima of row j.
  // Returns (cluster-uniformly later) whether a cost of row j decreased.
  __device__ bool merge_row(int32_t d, int32_t j) {
    bool changed = false;
    const int S = w / VPL;
    if (tid < S) {
      const T* r = row(d);
      const int32_t own = (int32_t)r[j];
      const int col = c0 + tid * VPL;
      Vec16<T> x = load16(r + col);
#pragma unroll
      for (int q = 0; q < VPL; ++q) {
        const int v = col + q;
        if (v < k && v != j) {
          const int32_t t = (int32_t)x.v[q] - own;
          const int64_t idx = (int64_t)j * k + v;
          const int32_t bt = I.tc[idx], bd = I.td[idx];
          if (lex_less(t, d, bt, bd)) {
            I.tc[idx] = t;
            I.td[idx] = d;
            changed |= (t < bt);
          }
        }
      }
    }
    return __syncthreads_or(changed) != 0;
  }

  // Row c of T over the owned columns, recomputed from c's member list:
  // T[c][v] = lexmin over d in seg(c) of (CM(d, v) - CM(d, c), d).
  __device__ void rescan(int32_t c) {
    const int S = w / VPL;
    const int R = kThreads / S;
    const int slot = tid % S, g = tid / S;
    // member lists are written by CTA 0: read them past L1
    const int32_t s = __ldcg(I.seg_size + c);
    int32_t bt[VPL], bd[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) { bt[q] = kTInf; bd[q] = -1; }
    if (g < R) {
      for (int32_t idx = g; idx < s; idx += R) {
        const int32_t d = __ldcg(mslot(c, idx));
        if ((uint32_t)d >= (uint32_t)n) continue;   // guard: corrupt list entry
        const T* r = row(d);
        const int32_t own = (int32_t)r[c];
        Vec16<T> x = load16(r + c0 + slot * VPL);
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
          const int32_t t = (int32_t)x.v[q] - own;
          if (lex_less(t, d, bt[q], bd[q])) { bt[q] = t; bd[q] = d; }
        }
      }
    }
    int2* red = reinterpret_cast<int2*>(s_red);   // [R][w]
    if (g < R) {
#pragma unroll
      for (int q = 0; q < VPL; ++q) red[g * w + slot * VPL + q] = make_int2(bt[q], bd[q]);
    }
    __syncthreads();
    for (int col = tid; col < w; col += kThreads) {
      const int v = c0 + col;
      if (v >= k) continue;
      int32_t t = kTInf, d = -1;
      for (int gg = 0; gg < R; ++gg) {
        int2 e = red[gg * w + col];
        if (lex_less(e.x, e.y, t, d)) { t = e.x; d = e.y; }
      }
      if (v == c) { t = kTInf; d = -1; }
      I.tc[(int64_t)c * k + v] = t;
      I.td[(int64_t)c * k + v] = d;
    }
    if (rank == 0 && tid == 0) rows += s;
    __syncthreads();
  }

  // -------------------------------------------------------- Bellman-Ford --
  // Lexicographic minimum of (label[u] + weight(u, v), u) over this
  // thread's share of the frontier (entries fg, fg+FG, ...).
  __device__ __forceinline__ void relax_column(int v, bool valid, int fg, int FG, int nfront,
                                               int32_t j, bool npath, int32_t pen_j,
                                               int64_t& bc, int32_t& bu) const {
    bc = kDInf;
    bu = INT32_MAX;
    if (!valid) return;
    for (int f = fg; f < nfront; f += FG) {
      const int32_t u = s_front[f];
      int64_t wgt;
      if (v == j) {                    // edge u -> s*in
        if (u == j) continue;
        if (npath) {
          wgt = (int64_t)(s_load[u] >= I.cap[u] ? I.pen[u] : 0) - pen_j;
        } else {
          const int32_t t = I.tc[(int64_t)u * k + j];
          if (t == kTInf) continue;
          wgt = t;
        }
      } else {                         // transfer edge u -> v
        const int32_t t = I.tc[(int64_t)u * k + v];
        if (t == kTInf) continue;
        wgt = t;
      }
      const int64_t c = s_dist[u] + wgt;
      if (c < bc || (c == bc && u < bu)) { bc = c; bu = u; }
    }
  }

  // Strict improvement of owned column cl: publish it for the gather.
  __device__ __forceinline__ void record_change(int cl, int64_t bc, int32_t bu, int32_t j,
                                                int64_t sink_dist, int32_t* outv,
                                                int64_t* outd, int64_t* oc) {
    const int v = c0 + cl;
    const int64_t cur = (v == j) ? sink_dist : s_dist[v];
    if (bc < cur) {
      if (v == j) {
        oc[OC_SINK_CHANGED] = 1;
        oc[OC_SINK_DIST] = bc;
        oc[OC_SINK_PAR] = bu;
      } else {
        const int at = atomicAdd(reinterpret_cast<int*>(&s_misc[MS_CNT]), 1);
        outv[at] = v;
        outd[at] = bc;
        s_par[cl] = bu;
      }
    }
  }


  // Canonical synchronous Bellman-Ford from the anchor j (Alg. 4 / Sections
  // 3.3-3.4).  Node u < k is center u, node j is s*out (the source) and the
  // sink s*in is represented by column j: an edge u -> s*in is
  //   NCyc (Def. 5 (c)): the best transfer u -> j,
  //   NPath (Def. 6 (c)): q_u() - q_j(), q_u() = pen[u] if load[u] >= cap[u].
  // No edge enters the source.  Labels change only on strict improvement and
  // take the lowest-index predecessor among equal candidates.
  // Returns 1 for a negative sink label (path to apply), 0 for none, and
  // < 0 on a broken invariant.  `merged` says whether this CTA's merge of
  // the round's unit lowered a cost of row j (NegCycle only).
  __device__ int bellman_ford(int32_t j, bool npath, bool merged, bool allow_skip) {
    for (int v = tid; v < k; v += kThreads) s_dist[v] = (v == j) ? 0 : kDInf;
    for (int v = tid; v < w; v += kThreads) s_par[v] = -1;
    if (tid == 0) {
      s_front[0] = j;
      s_misc[MS_NFRONT] = 1;
      s_misc[MS_SINK_DIST] = kDInf;
      s_misc[MS_SINK_PAR] = -1;
    }
    __syncthreads();
    const int owner_j = j / w;
    const int32_t pen_j = I.pen[j];
    const int NTc = min(kThreads, max(32, (wr + 31) / 32 * 32));
    const int FG = kThreads / NTc;
    const int cl0 = tid % NTc, fg = tid / NTc;
    int result = 0;
    for (int sweep = 1;; ++sweep) {
      const int nfront = (int)s_misc[MS_NFRONT];
      const int64_t sink_dist = s_misc[MS_SINK_DIST];
      if (tid == 0) s_misc[MS_CNT] = 0;
      int32_t* outv = s_outv + buf * w;
      int64_t* outd = s_outd + buf * w;
      int64_t* oc = s_outctl + buf * 8;
      if (tid == 0) { oc[OC_SINK_CHANGED] = 0; oc[OC_MERGE_CHANGED] = merged ? 1 : 0; }
      __syncthreads();
      // relax all edges out of the frontier into the owned columns
      int64_t* red_c = reinterpret_cast<int64_t*>(s_red);
      int32_t* red_u = reinterpret_cast<int32_t*>(s_red + 8 * kThreads);
      const bool active = fg < FG;
      if (FG > 1) {
        // one owned column per thread, frontier split over FG groups
        if (active) {
          int64_t bc; int32_t bu;
          relax_column(c0 + cl0, cl0 < wr, fg, FG, nfront, j, npath, pen_j, bc, bu);
          red_c[fg * NTc + cl0] = bc;
          red_u[fg * NTc + cl0] = bu;
        }
        __syncthreads();
        if (fg == 0 && cl0 < wr) {
          int64_t bc = kDInf;
          int32_t bu = INT32_MAX;
          for (int g2 = 0; g2 < FG; ++g2) {
            const int64_t c = red_c[g2 * NTc + cl0];
            const int32_t u = red_u[g2 * NTc + cl0];
            if (c < bc || (c == bc && u < bu)) { bc = c; bu = u; }
          }
          record_change(cl0, bc, bu, j, sink_dist, outv, outd, oc);
        }
      } else if (active) {
        for (int cl = cl0; cl < wr; cl += NTc) {
          int64_t bc; int32_t bu;
          relax_column(c0 + cl, true, 0, 1, nfront, j, npath, pen_j, bc, bu);
          record_change(cl, bc, bu, j, sink_dist, outv, outd, oc);
        }
      }
      __syncthreads();
      if (tid == 0) oc[OC_COUNT] = (int32_t)s_misc[MS_CNT];
      __syncthreads();
      cluster_sync_all();
      commit_pending();
      // gather every CTA's changes (same order in every CTA)
      int32_t* s_cnt = reinterpret_cast<int32_t*>(s_red + 12 * kThreads);   // [C+1] prefix
      if (tid < 32) {
        // lane r reads CTA r's counters; a warp scan forms the offsets
        const int lane = tid;
        int32_t cnt = 0;
        int64_t mg = 0;
        if (lane < C) {
          cnt = (int32_t)dsmem_ld64(dsmem_addr(s_outctl + buf * 8 + OC_COUNT, lane));
          mg = dsmem_ld64(dsmem_addr(s_outctl + buf * 8 + OC_MERGE_CHANGED, lane));
        }
        int32_t inc = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int32_t o = __shfl_up_sync(0xffffffffu, inc, off);
          if (lane >= off) inc += o;
        }
        const unsigned any = __ballot_sync(0xffffffffu, mg != 0);
        if (lane < C) s_cnt[lane] = inc - cnt;
        if (lane == C - 1) { s_cnt[C] = inc; s_misc[MS_TOTAL] = inc; }
        if (lane == 0) {
          s_misc[MS_MERGE_ANY] = any ? 1 : 0;
          const int64_t chg =
              dsmem_ld64(dsmem_addr(s_outctl + buf * 8 + OC_SINK_CHANGED, owner_j));
          s_misc[MS_SINK_CHG] = chg;
          if (chg) {
            s_misc[MS_SINK_DIST] =
                dsmem_ld64(dsmem_addr(s_outctl + buf * 8 + OC_SINK_DIST, owner_j));
            s_misc[MS_SINK_PAR] =
                dsmem_ld64(dsmem_addr(s_outctl + buf * 8 + OC_SINK_PAR, owner_j));
          }
        }
      }
      __syncthreads();
      const int total = (int)s_misc[MS_TOTAL];
      for (int i = tid; i < total; i += kThreads) {
        int r = 0;
        while (s_cnt[r + 1] <= i) ++r;
        const int li = i - s_cnt[r];
        const int32_t v = dsmem_ld32(dsmem_addr(s_outv + buf * w + li, r));
        const int64_t dd = dsmem_ld64(dsmem_addr(s_outd + buf * w + li, r));
        s_front[i] = v;
        s_dist[v] = dd;
      }
      if (tid == 0) s_misc[MS_NFRONT] = total;
      __syncthreads();
      buf ^= 1;
      const bool sink_chg = s_misc[MS_SINK_CHG] != 0;
      if (sweep == 1 && allow_skip && s_misc[MS_MERGE_ANY] == 0) {
        // T is unchanged since the last round, whose Gamma had no negative
        // cycle (Lemmas 1/2): the NegCycle sink label cannot be negative.
        if (rank == 0 && tid == 0) skipped++;
        return 0;
      }
      if (total == 0 && !sink_chg) {
        if (rank == 0 && tid == 0) {
          bf_calls++;
          bf_sweeps += sweep;
          bf_max = max(bf_max, (int64_t)sweep);
        }
        result = s_misc[MS_SINK_DIST] < 0 ? 1 : 0;
        break;
      }
      if (sweep >= k + 1) { result = -1; break; }
    }
    return result;
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

  // Apply the transfers of the path (Alg. 2 lines 5-9, Alg. 3 lines 5-10);
  // then recompute the rows of T of every center on it.  For NCyc every
  // center on the cycle loses one unit and gains one; for NPath the anchor
  // only loses one and the terminal center only gains one.
  __device__ void apply(int32_t j, bool npath, int m) {
    if (rank == 0 && tid < 32) {
      const int lane = tid;
      int32_t* ppos = reinterpret_cast<int32_t*>(s_red);   // positions of the outgoing units
      for (int i = lane; i < m; i += 32) {
        const int32_t from = s_path[i];
        const int32_t to = (i + 1 < m) ? s_path[i + 1] : (npath ? -1 : j);
        int32_t x = to >= 0 ? __ldcg(I.td + (int64_t)from * k + to) : -1;
        if (to >= 0 && (uint32_t)x >= (uint32_t)n) { x = -1; err0 = ST_ERR_INVARIANT; }
        s_pathu[i] = x;
        ppos[i] = x >= 0 ? I.pos[x] : -1;
      }
      __syncwarp();
      // in-place replacements: center p_i swaps its leaving unit for the
      // arriving unit x_{i-1} (cyclically for NCyc)
      for (int i = lane; i < m; i += 32) {
        const int32_t c = s_path[i];
        const int32_t x_out = s_pathu[i];
        const int32_t x_in = (i > 0) ? s_pathu[i - 1] : (npath ? -1 : s_pathu[m - 1]);
        if (x_out >= 0 && x_in >= 0 && ppos[i] >= 0 && ppos[i] < n) {
          *mslot(c, ppos[i]) = x_in;
          I.pos[x_in] = ppos[i];
        }
        if (x_out >= 0) I.assign[x_out] = (i + 1 < m) ? s_path[i + 1] : j;
      }
      __syncwarp();
      if (lane == 0) {
        if (npath) {
          // the anchor loses x_0, the terminal center gains x_{m-2}
          list_remove_at(j, ppos[0]);
          if (s_pathu[m - 2] >= 0) list_append(s_path[m - 1], s_pathu[m - 2]);
          else err0 = ST_ERR_INVARIANT;
          I.load[j] -= 1;
          I.load[s_path[m - 1]] += 1;
          paths++;
          moves += m - 1;
        } else {
          cycles++;
          moves += m;
        }
        delta += s_misc[MS_SINK_DIST];
      }
    }
    if (npath && tid == 0) {   // load replicas in every CTA
      s_load[j] -= 1;
      s_load[s_path[m - 1]] += 1;
    }
    __syncthreads();
    cluster_sync_all();   // member lists updated before anyone rescans
    for (int i = 0; i < m; ++i) rescan(s_path[i]);
  }

  // ---------------------------------------------------------- the loop --
  __device__ void run_rounds() {
    const int64_t r_begin = I.ctl[CTL_ROUNDS];
    const int64_t r_end = min((int64_t)n, I.ctl[CTL_TARGET]);
    for (int v = tid; v < k; v += kThreads) s_load[v] = __ldcg(I.load + v);
    if (rank == 0 && tid == 0) {
      delta = I.ctl[CTL_DELTA];
      free_top = I.ctl[CTL_FREE_TOP];
      cycles = paths = bf_calls = bf_sweeps = bf_max = moves = skipped = rows = 0;
    }
    __syncthreads();
    const bool allow_skip = !(flags & OPT_NO_NCYC_SKIP);
    int64_t status = ST_OK;
    int64_t r = r_begin;
    for (; r < r_end; ++r) {
      // Alg. 1 lines 5-6 and 9-13: next unit of the MinDistance order goes
      // to its most suitable center; pay the penalty if it had no vacancy.
      const int32_t d = __ldcg(I.order + r);
      if ((uint32_t)d >= (uint32_t)n) { status = ST_ERR_INVARIANT; break; }   // uniform guard
      const int32_t j = __ldcg(I.smin + d);
      if ((uint32_t)j >= (uint32_t)k) { status = ST_ERR_INVARIANT; break; }
      const bool over = s_load[j] >= I.cap[j];
      const bool merged = merge_row(d, j);
      if (tid == 0) s_load[j] += 1;
      if (rank == 0 && tid == 0) {
        // Member lists are touched only after the next cluster barrier (the
        // first Bellman-Ford sweep), when every CTA has finished reading
        // them for the previous round's rescans.
        delta += (int64_t)row(d)[j] + (over ? (int64_t)I.pen[j] : 0);
      }
      __syncthreads();
      // Alg. 2 at j
      int res = bellman_ford_with_allot(j, d, false, merged, allow_skip);
      if (res < 0) { status = ST_ERR_INVARIANT; break; }
      if (res > 0) {
        const int m = walk_path(j);
        if (m < 2) { status = ST_ERR_INVARIANT; break; }
        apply(j, false, m);
      }
      // Alg. 3 at j when the allotment overloaded it
      if (over) {
        res = bellman_ford(j, true, true, false);
        if (res < 0) { status = ST_ERR_INVARIANT; break; }
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
      I.ctl[CTL_DELTA] = delta;
      I.ctl[CTL_FREE_TOP] = free_top;
      I.ctl[CTL_STATUS] = status != ST_OK ? status : err0;
      I.ctl[CTL_CYCLES] += cycles;
      I.ctl[CTL_PATHS] += paths;
      I.ctl[CTL_BF_CALLS] += bf_calls;
      I.ctl[CTL_BF_SWEEPS] += bf_sweeps;
      I.ctl[CTL_BF_MAX] = max(I.ctl[CTL_BF_MAX], bf_max);
      I.ctl[CTL_MOVES] += moves;
      I.ctl[CTL_NCYC_SKIPPED] += skipped;
      I.ctl[CTL_ROWS_SCANNED] += rows;
    }
  }

  // The NegCycle Bellman-Ford of a round.  CTA 0 records the allotment of d
  // (assign, member list, global load) right after the first sweep's
  // barrier, when no CTA still reads member lists of the previous round.
  __device__ int bellman_ford_with_allot(int32_t j, int32_t d, bool npath, bool merged,
                                         bool allow_skip) {
    pending_d = d;
    pending_j = j;
    return bellman_ford(j, npath, merged, allow_skip);
  }
  int32_t pending_d = -1, pending_j = -1;

  __device__ __forceinline__ void commit_pending() {
    if (pending_d >= 0) {
      if (rank == 0 && tid == 0) {
        I.assign[pending_d] = pending_j;
        list_append(pending_j, pending_d);
        I.load[pending_j] += 1;
      }
      pending_d = -1;
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
asral_cluster_kernel(const DevInst* __restrict__ insts, int ninst, int* work_counter, int flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  Solver<T> S;
  S.tid = threadIdx.x;
  S.rank = (int)cluster_rank();
  S.C = (int)cluster_nrank();
  S.flags = flags;
  S.buf = 0;
  int64_t* s_item = reinterpret_cast<int64_t*>(smem);   // first 16 bytes: work item
  unsigned char* base = smem + 16;
  for (;;) {
    if (S.rank == 0 && S.tid == 0) s_item[0] = atomicAdd(work_counter, 1);
    __syncthreads();
    cluster_sync_all();
    const int item = (int)dsmem_ld64(dsmem_addr(s_item, 0));
    cluster_sync_all();
    if (item >= ninst) break;
    S.I = insts[item];
    S.cm = static_cast<const T*>(S.I.cm);
    S.n = S.I.n;
    S.k = S.I.k;
    S.w = own_width(S.k, S.C, Solver<T>::VPL);
    S.c0 = S.rank * S.w;
    S.c1 = min(S.k, S.c0 + S.w);
    S.wr = max(0, S.c1 - S.c0);
    const Layout L = make_layout(S.k, S.C, Solver<T>::VPL);
    S.s_dist = reinterpret_cast<int64_t*>(base + L.dist);
    S.s_load = reinterpret_cast<int32_t*>(base + L.load);
    S.s_front = reinterpret_cast<int32_t*>(base + L.front);
    S.s_par = reinterpret_cast<int32_t*>(base + L.par);
    S.s_outv = reinterpret_cast<int32_t*>(base + L.outv);
    S.s_outd = reinterpret_cast<int64_t*>(base + L.outd);
    S.s_outctl = reinterpret_cast<int64_t*>(base + L.outctl);
    S.s_path = reinterpret_cast<int32_t*>(base + L.path);
    S.s_pathu = reinterpret_cast<int32_t*>(base + L.pathu);
    S.s_misc = reinterpret_cast<int64_t*>(base + L.misc);
    S.s_red = base + L.red;
    if (S.I.ctl[CTL_PROLOGUE] == 0) {
      S.prologue();
      if (S.rank == 0 && S.tid == 0) {
        S.I.ctl[CTL_FREE_TOP] = S.I.npages;
        S.I.ctl[CTL_ROUNDS] = 0;
        S.I.ctl[CTL_DELTA] = 0;
        S.I.ctl[CTL_PROLOGUE] = 1;
      }
      __syncthreads();
      cluster_sync_all();
    }
    S.run_rounds();
  }
}

// Shared-memory bytes of one CTA for an instance with k centers on C-CTA
// clusters (includes the 16-byte work-item slot).
size_t solver_smem_bytes(int32_t k, int C, int elem_bytes) {
  const int vpl = 16 / elem_bytes;
  return 16 + make_layout(k, C, vpl).total;
}

int solver_max_k(int C, int elem_bytes) {
  // the rescan maps every owned 16-byte column group to a thread
  return kThreads * (16 / elem_bytes) * C;
}

template <typename T>
cudaError_t launch_solver_t(const DevInst* d_insts, int ninst, int* d_counter, int C,
                            int nclusters, size_t smem, int flags, cudaStream_t st) {
  auto kern = asral_cluster_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
  return cudaLaunchKernelEx(&cfg, kern, d_insts, ninst, d_counter, flags);
}

cudaError_t launch_solver(const DevInst* d_insts, int ninst, int* d_counter, int C,
                          int nclusters, int elem_bytes, size_t smem, int flags,
                          cudaStream_t st) {
  if (elem_bytes == 2)
    return launch_solver_t<int16_t>(d_insts, ninst, d_counter, C, nclusters, smem, flags, st);
  return launch_solver_t<int32_t>(d_insts, ninst, d_counter, C, nclusters, smem, flags, st);
}

// Largest number of co-resident clusters of size C for this kernel.
int solver_max_clusters(int C, int elem_bytes, size_t smem) {
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
  int num = 0;
  cudaError_t e;
  if (elem_bytes == 2) {
    cudaFuncSetAttribute(asral_cluster_kernel<int16_t>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (C > 8)
      cudaFuncSetAttribute(asral_cluster_kernel<int16_t>,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    e = cudaOccupancyMaxActiveClusters(&num, asral_cluster_kernel<int16_t>, &cfg);
  } else {
    cudaFuncSetAttribute(asral_cluster_kernel<int32_t>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (C > 8)
      cudaFuncSetAttribute(asral_cluster_kernel<int32_t>,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    e = cudaOccupancyMaxActiveClusters(&num, asral_cluster_kernel<int32_t>, &cfg);
  }
  return e == cudaSuccess ? num : -1;
}

}  // namespace lbdd
