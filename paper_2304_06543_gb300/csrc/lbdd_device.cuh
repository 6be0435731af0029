// Internal device-side definitions of the LBDD/ASRAL CUDA path (sm_103a).
//
// Everything here is private to the library: the public boundary is the C ABI
// in include/lbdd.h.  All arithmetic is integer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbdd {

constexpr int kThreads = 512;          // threads per CTA of every kernel here
constexpr int kWarps = kThreads / 32;
constexpr int kPageShift = 8;          // member lists are paged, 256 units/page
constexpr int kPage = 1 << kPageShift;
constexpr int kPageWords = 2 * kPage;  // a page: kPage unit ids, then their own costs CM(d, c)
constexpr int kMaxCluster = 16;        // cluster sizes 1..16 (16 is non-portable)
constexpr int32_t kTInf = INT32_MAX;   // best-transfer entry of an empty segment
constexpr int64_t kDInf = (int64_t)1 << 62;  // unreached Bellman-Ford label
constexpr int kColPad = 128;           // CM allocation slack for vector over-reads

// Per-instance control words (int64, device memory).
enum CtlIndex {
  CTL_ROUNDS = 0,      // rounds completed
  CTL_DELTA,           // tracked objective, Eq. (1)
  CTL_FREE_TOP,        // free-page stack height
  CTL_STATUS,          // 0 = ok, else an LBDD_ERR_* code
  CTL_PROLOGUE,        // 1 once s_min/order/state are initialised
  CTL_TARGET,          // rounds to reach in the current launch
  CTL_CYCLES,          // negative cycles applied (Alg. 1)
  CTL_PATHS,           // negative paths applied (Alg. 4)
  CTL_BF_CALLS,        // Bellman-Ford calls actually run
  CTL_BF_SWEEPS,       // total synchronous sweeps
  CTL_BF_MAX,          // longest call, in sweeps
  CTL_MOVES,           // unit transfers
  CTL_NCYC_SKIPPED,    // NegCycle calls skipped because T[j] did not change
  CTL_ROWS_SCANNED,    // CM rows read by segment rescans
  CTL_MAXKEY,          // largest CM(d, s_min(d)) (radix-sort width)
  CTL_T_TOTAL,         // round loop of CTA 0, globaltimer ns
  CTL_T_CYCLES,        // the same interval in SM cycles (converts the phase timers)
  CTL_T_PROLOGUE,      // globaltimer ns
  // phase timers of CTA 0 in SM cycles (reported in ns by lbdd_get_stats)
  CTL_T_MERGE,
  CTL_T_RELAX,
  CTL_T_SYNC,
  CTL_T_GATHER,
  CTL_T_APPLY,
  CTL_T_RESCAN,
  CTL_TSM_ON,          // 1 if the last launch kept the owned cost slice in shared memory
  CTL_T_RLOOP,         // relaxation loop only (cycles, part of CTL_T_RELAX)
  CTL_T_RRED,          // loop + cross-warp reduction (cycles, part of CTL_T_RELAX)
  CTL_NPATH_REUSED,    // Alg. 4 answered from the converged Alg. 1 labels
  CTL_COL_ROWS,        // member rows read by column-subset rescans
  CTL_FRONT_SUM,       // sum of Bellman-Ford frontier sizes over sweeps
  CTL_FRONT_HIST,      // 6 bins of frontier sizes: 1, 2-4, 5-16, 17-64, 65-256, >256
  CTL_COUNT = CTL_FRONT_HIST + 6
};

// Status codes shared with include/lbdd.h.
enum : int64_t {
  ST_OK = 0,
  ST_ERR_TIMEOUT = -4,     // a bounded wait inside a kernel ran out
  ST_ERR_INVARIANT = -5,
};

// Launch-wide option bits.
enum : int {
  OPT_NO_NCYC_SKIP = 1,   // always run the NegCycle Bellman-Ford
  OPT_NO_NPATH_REUSE = 2, // always run the NegPath Bellman-Ford
  OPT_NO_TC_SMEM = 4,     // keep the owned cost slice in global memory only
  OPT_PHASE_TIMERS = 8,   // time the phases of every round (CTA 0, thread 0)
  OPT_STRICT = 32,        // strict-LBDD (Alg. 5): vacancies as zero-cost dummy units
};

// Device view of one instance.  Pointers are device memory owned by the
// library (lbdd_solver).
struct DevInst {
  const void* cm;       // n x ld, int32 or int16, demand-major, padded rows
  int64_t ld;           // row pitch in elements (multiple of 16 bytes)
  int32_t n, k;
  const int32_t* cap;   // k
  const int32_t* pen;   // k x Q penalty table: q_s(j) = pen[s*Q + min(j, Q) - 1] (Def. 4)
  int32_t Q;            // table length (1: constant per-unit penalty)
  int32_t* smin;        // n: most suitable center
  int32_t* order;       // n: MinDistance extraction order
  int32_t* sort_tmp;    // 3n: radix-sort scratch
  int32_t* assign;      // n: center of each unit, -1 before its round
  int32_t* pos;         // n: index of the unit inside its center's list
  int32_t* load;        // k: units allotted per center
  int32_t* seg_size;    // k: length of each member list
  int32_t* page_tab;    // k x max_pages: page ids of each member list
  int32_t* pool;        // pages x kPageWords: member ids, then each member's own cost
  int32_t* free_stack;  // pages
  int32_t* tc;          // k x k best-transfer cost (row u = from u)
  int32_t* td;          // k x k best-transfer unit
  int64_t* ctl;         // CTL_COUNT
  int32_t max_pages;    // per center
  int32_t npages;       // in the pool
};

// ------------------------------------------------------------ cluster ops ---

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_nrank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Full cluster barrier; every thread of every CTA of the cluster must reach
// it.  Release/acquire order shared and global memory across the cluster.
__device__ __forceinline__ void cluster_sync_all() {
  uint32_t nr;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(nr));
  if (nr == 1) {   // a one-CTA cluster: the CTA barrier orders the same accesses
    __syncthreads();
    return;
  }
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;\n\t" ::: "memory");
}
// Address of `p` (a shared variable of this CTA) in CTA `rank`'s window.
__device__ __forceinline__ uint32_t dsmem_addr(const void* p, uint32_t rank) {
  uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p)), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ int32_t dsmem_ld32(uint32_t addr) {
  int32_t v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int64_t dsmem_ld64(uint32_t addr) {
  int64_t v;
  asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void dsmem_st32(uint32_t addr, int32_t v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void dsmem_st64(uint32_t addr, int64_t v) {
  asm volatile("st.shared::cluster.s64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

// ------------------------------------------------- transaction barriers ---
// A CTA's mbarrier in its own shared memory, completed by one local arrival
// plus a byte count of asynchronous stores from the other CTAs of the
// cluster (st.async ... mbarrier::complete_tx::bytes).  The stores may land
// before the local arrival announces their byte count: the pending count
// then goes negative, and the phase still completes only once the arrival
// and all announced bytes are in.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals)
               : "memory");
}
// Makes initialised barriers visible to the other CTAs of the cluster (a
// cluster barrier must follow before any of them signals this barrier).
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// The local arrival of the current phase, announcing `bytes` of incoming
// asynchronous stores.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// True once the phase of parity `parity` has completed; acquires the
// asynchronous stores of the cluster that completed it.  The thread may
// sleep inside the instruction for up to `sleep_ns` while the phase is open
// (it wakes when the phase completes), so a waiting warp issues few
// instructions.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity,
                                              uint32_t sleep_ns = 0) {
  uint32_t done;
  if (sleep_ns == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "r"(sleep_ns) : "memory");
  }
  return done != 0;
}
// Orders this thread's view of earlier generic-proxy writes to shared
// memory (by any thread of the CTA, after a CTA barrier) before later
// bulk copies that read it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from this CTA's shared memory into another CTA's shared memory (cluster
// address `dst`), completing the bytes on that CTA's barrier at cluster
// address `bar`.  The copy engine moves the data; the issuing thread does
// not wait.
__device__ __forceinline__ void bulk_copy_to_cta(uint32_t dst, const void* src, uint32_t bytes,
                                                 uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "r"(smem_u32(src)), "r"(bytes), "r"(bar) : "memory");
}
// One arrival on a barrier of this CTA (release: this thread's earlier
// shared-memory reads and writes are ordered before the phase completes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global memory into this CTA's shared memory (address `dst`),
// completing the bytes on this CTA's barrier at shared address `bar`.
__device__ __forceinline__ void bulk_load_smem(uint32_t dst, const void* src, uint32_t bytes,
                                               uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// 16 bytes into another CTA's shared memory (cluster address `dst`),
// completing that many bytes on its barrier at cluster address `bar`.
__device__ __forceinline__ void st_async16(uint32_t dst, int4 v, uint32_t bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
      ::"r"(dst), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(bar) : "memory");
}

// ------------------------------------------------------------ CM access ---

template <typename T>
struct Vec16 {
  static constexpr int N = 16 / sizeof(T);
  T v[N];
};

template <typename T>
__device__ __forceinline__ Vec16<T> load16(const T* p) {
  Vec16<T> r;
  int4 x = __ldg(reinterpret_cast<const int4*>(p));
  static_assert(sizeof(r) == sizeof(x), "vector size");
  *reinterpret_cast<int4*>(&r) = x;
  return r;
}

__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// SM cycle counter: cheap enough to bracket every Bellman-Ford sweep.
__device__ __forceinline__ uint64_t clock_cycles() { return (uint64_t)clock64(); }

__device__ __forceinline__ uint32_t dyn_smem_bytes() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

// Lexicographic (cost, unit) order used for every best-transfer entry.
__device__ __forceinline__ bool lex_less(int32_t c, int32_t d, int32_t bc, int32_t bd) {
  return c < bc || (c == bc && (uint32_t)d < (uint32_t)bd);
}

}  // namespace lbdd
