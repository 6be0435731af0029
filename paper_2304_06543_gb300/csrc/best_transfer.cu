// Best-transfer table from scratch: the data-parallel replacement of the
// paper's Gamma-DS heap maintenance (Section 3.4 "Allotment subspace
// multi-graph implementation", Section 3.5.2), which took 74% of ASRAL's time
// in the paper's measurements (Section 5).
//
//   T[u][v] = lexmin over d with assign[d] == u of (CM(d,v) - CM(d,u), d)
//
// Pipeline (all device-side, one stream):
//   1. stable LSD radix sort of (assign[d], d) -> units grouped by center,
//      ascending d inside each center (grid-wide, 8-bit digits);
//   2. segment bounds and a list of work items, each at most kChunk rows of
//      one center;
//   3. the scan: each CTA streams its item's CM rows with 16-byte loads,
//      every thread keeps a running minimum for 16 bytes' worth of columns;
//      rows arrive in increasing d, so a strict '<' already keeps the lowest
//      d on equal cost; the partial minima of the CTA are combined in shared
//      memory and merged into a packed (cost, d) 64-bit table with atomicMin;
//   4. unpack to the (tc, td) int32 pair.
// Step 3 reads every CM byte of the allotted rows exactly once and is the
// HBM-bound kernel; everything else moves O(n + k*k) bytes.
#include <atomic>
#include <algorithm>

#include "lbdd_device.cuh"

namespace lbdd {

constexpr int kTile = kThreads * 8;     // radix-sort tile (elements)
constexpr int kChunk = 512;             // rows per scan work item
constexpr int kScanUnroll = 6;          // rows in flight per thread (plus ids of the next 6)

struct BtWorkspace {
  int32_t *k0, *v0, *k1, *v1;   // radix ping-pong
  int32_t* tile_hist;           // 256 x ntiles
  int32_t* seg_start;           // k
  int32_t* seg_end;             // k
  int32_t* item_off;            // k + 1
  unsigned long long* t64;      // k x k packed (cost + 2^31) << 32 | d
  int4* items;                  // explicit work items {center, first row, rows, 0}
  int* err;                     // [0] unused, [1] the work-item queue counter
  int32_t* dsum;                // 256 digit totals of a radix pass
  int32_t* ownv;                // n: CM(d, center of d) in sorted order (int16 scan)
  int64_t ntiles;
  size_t bytes;
};

static inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static BtWorkspace carve(void* base, int32_t n, int32_t k) {
  BtWorkspace W;
  W.ntiles = (n + kTile - 1) / kTile;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = static_cast<char*>(base) + o;
    o = al256(o + bytes);
    return p;
  };
  W.k0 = reinterpret_cast<int32_t*>(take(4ull * n));
  W.v0 = reinterpret_cast<int32_t*>(take(4ull * n));
  W.k1 = reinterpret_cast<int32_t*>(take(4ull * n));
  W.v1 = reinterpret_cast<int32_t*>(take(4ull * n));
  W.tile_hist = reinterpret_cast<int32_t*>(take(4ull * 256 * W.ntiles));
  W.seg_start = reinterpret_cast<int32_t*>(take(4ull * k));
  W.seg_end = reinterpret_cast<int32_t*>(take(4ull * k));
  W.item_off = reinterpret_cast<int32_t*>(take(4ull * (k + 1)));
  W.t64 = reinterpret_cast<unsigned long long*>(take(8ull * k * k));
  W.items = reinterpret_cast<int4*>(take(16ull * ((size_t)n / kChunk + (size_t)k + 1)));
  W.err = reinterpret_cast<int*>(take(16));   // err, then the item queue counter
  W.dsum = reinterpret_cast<int32_t*>(take(4 * 256));
  W.ownv = reinterpret_cast<int32_t*>(take(4ull * n));
  W.bytes = o;
  return W;
}

size_t bt_workspace_bytes(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  return carve(nullptr, n, k).bytes + 256;
}

// ------------------------------------------------------------ radix sort ---

// keys = assign (unallotted units -> bucket k, sorted last); values = d.
__global__ void __launch_bounds__(kThreads) bt_init_keys(const int32_t* __restrict__ assign,
                                                         int32_t n, int32_t k, int32_t* keys,
                                                         int32_t* vals) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    int32_t a = assign[i];
    keys[i] = (a < 0 || a >= k) ? k : a;
    vals[i] = (int32_t)i;
  }
}

__global__ void __launch_bounds__(kThreads) bt_hist(const int32_t* __restrict__ keys, int32_t n,
                                                    int shift, int32_t* tile_hist,
                                                    int64_t ntiles) {
  __shared__ int32_t h[256];
  for (int i = threadIdx.x; i < 256; i += kThreads) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += kThreads) {
    const int64_t g = base + i;
    if (g < n) atomicAdd(&h[(keys[g] >> shift) & 255], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += kThreads) tile_hist[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// Exclusive scan of a device array of length m, one CTA.
__global__ void __launch_bounds__(kThreads) bt_scan(int32_t* a, int64_t m, int32_t* total_out) {
  __shared__ int32_t part[kThreads];
  const int64_t per = (m + kThreads - 1) / kThreads;
  const int64_t lo = threadIdx.x * per, hi = min(m, lo + per);
  int32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int t = 0; t < kThreads; ++t) { int32_t c = part[t]; part[t] = run; run += c; }
    if (total_out) *total_out = run;
  }
  __syncthreads();
  int32_t run = part[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) { int32_t c = a[i]; a[i] = run; run += c; }
}

// Block-wide exclusive scan of one value per thread; returns this thread's
// prefix and writes the block total to *total.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* s_warp,
                                                        int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < kWarps ? s_warp[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < kWarps) s_warp[lane] = w;   // inclusive warp prefixes
  }
  __syncthreads();
  const int32_t before = warp > 0 ? s_warp[warp - 1] : 0;
  *total = s_warp[kWarps - 1];
  return before + x - v;
}

// Digit totals of a radix pass: CTA d sums row d of the digit-major
// histogram (one row per digit, one column per tile).
__global__ void __launch_bounds__(kThreads) bt_digit_sums(const int32_t* __restrict__ tile_hist,
                                                          int64_t ntiles, int32_t* dsum) {
  __shared__ int32_t s_warp[kWarps];
  const int32_t* row = tile_hist + (int64_t)blockIdx.x * ntiles;
  int32_t s = 0;
  for (int64_t i = threadIdx.x; i < ntiles; i += kThreads) s += row[i];
  int32_t total;
  block_exclusive_scan(s, s_warp, &total);
  if (threadIdx.x == 0) dsum[blockIdx.x] = total;
}

// Exclusive scan of the whole digit-major histogram, one CTA per digit row:
// the row's base is the sum of the lower digits' totals, then the row is
// scanned in contiguous per-thread chunks.
__global__ void __launch_bounds__(kThreads) bt_digit_scan(int32_t* tile_hist, int64_t ntiles,
                                                          const int32_t* __restrict__ dsum) {
  __shared__ int32_t s_warp[kWarps];
  __shared__ int32_t s_base;
  const int d = blockIdx.x;
  int32_t b = threadIdx.x < d ? dsum[threadIdx.x] : 0;   // d <= 255 < kThreads
  int32_t btot;
  block_exclusive_scan(b, s_warp, &btot);
  if (threadIdx.x == 0) s_base = btot;
  __syncthreads();
  const int32_t base = s_base;
  int32_t* row = tile_hist + (int64_t)d * ntiles;
  const int64_t per = (ntiles + kThreads - 1) / kThreads;
  const int64_t lo = min(ntiles, (int64_t)threadIdx.x * per), hi = min(ntiles, lo + per);
  int32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += row[i];
  int32_t total;
  __syncthreads();                     // s_warp is reused
  int32_t run = base + block_exclusive_scan(s, s_warp, &total);
  for (int64_t i = lo; i < hi; ++i) {
    const int32_t c = row[i];
    row[i] = run;
    run += c;
  }
}

// Stable scatter of one tile, in order, 512 elements at a time.
__global__ void __launch_bounds__(kThreads) bt_scatter(const int32_t* __restrict__ sk,
                                                       const int32_t* __restrict__ sv,
                                                       int32_t* dk, int32_t* dv, int32_t n,
                                                       int shift,
                                                       const int32_t* __restrict__ tile_hist,
                                                       int64_t ntiles) {
  __shared__ int32_t s_off[256];
  __shared__ int32_t s_wc[kWarps * 256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  for (int i = tid; i < 256; i += kThreads) s_off[i] = tile_hist[(int64_t)i * ntiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int c = 0; c < kTile; c += kThreads) {
    const int64_t i = base + c + tid;
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
        const int32_t cnt = s_wc[ww * 256 + tid];
        s_wc[ww * 256 + tid] = run;
        run += cnt;
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

// Segment bounds of the sorted keys; with cm16, also the own cost
// CM(d, c) of every sorted unit (for the staged int16 scan).
__global__ void __launch_bounds__(kThreads) bt_bounds(const int32_t* __restrict__ keys,
                                                      const int32_t* __restrict__ vals,
                                                      int32_t n, int32_t k, int32_t* seg_start,
                                                      int32_t* seg_end,
                                                      const int16_t* __restrict__ cm16, int64_t ld,
                                                      int32_t* ownv) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const int32_t c = keys[i];
    if (c >= k) continue;
    if (i == 0 || keys[i - 1] != c) seg_start[c] = (int32_t)i;
    if (i == n - 1 || keys[i + 1] != c) seg_end[c] = (int32_t)i + 1;
    if (cm16) ownv[i] = cm16[(int64_t)vals[i] * ld + c];
  }
}

__global__ void __launch_bounds__(kThreads) bt_items(const int32_t* __restrict__ seg_start,
                                                     const int32_t* __restrict__ seg_end,
                                                     int32_t k, int32_t* item_cnt,
                                                     unsigned long long* t64) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * kThreads) {
    const int32_t s = seg_end[i] - seg_start[i];
    item_cnt[i] = (s + kChunk - 1) / kChunk;
  }
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (int64_t)k * k;
       i += (int64_t)gridDim.x * kThreads)
    t64[i] = ~0ull;
}

// Explicit item list: item_off[c] + i -> {c, first row, rows}.
__global__ void __launch_bounds__(kThreads) bt_item_list(const int32_t* __restrict__ seg_start,
                                                         const int32_t* __restrict__ seg_end,
                                                         const int32_t* __restrict__ item_off,
                                                         int32_t k, int4* items) {
  for (int64_t c = blockIdx.x * (int64_t)kThreads + threadIdx.x; c < k;
       c += (int64_t)gridDim.x * kThreads) {
    const int32_t s0 = seg_start[c], s1 = seg_end[c];
    int32_t it = item_off[c];
    for (int32_t r = s0; r < s1; r += kChunk, ++it) items[it] = make_int4((int)c, r, min(kChunk, s1 - r), 0);
  }
}

// ------------------------------------------------------------------ scan ---

template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
bt_scan_rows(const T* __restrict__ cm, int64_t ld, int32_t n, int32_t k,
             const int32_t* __restrict__ perm, const int32_t* __restrict__ item_off,
             const int4* __restrict__ items, unsigned long long* t64, int* work) {
  constexpr int VPL = 16 / (int)sizeof(T);
  constexpr int U = kScanUnroll;
  __shared__ int2 red[kThreads * VPL];
  __shared__ int s_item[2];
  const int S = (k + VPL - 1) / VPL;       // 16-byte column groups per row
  const int R = kThreads / S;              // row groups
  const int tid = threadIdx.x, slot = tid % S, g = tid / S;
  const int32_t total = item_off[k];
  // items come from a global queue: CTAs that finish early take more
  if (tid == 0) s_item[0] = atomicAdd(work, 1);
  __syncthreads();
  for (int32_t item = s_item[0];;) {
    if (item >= total) break;
    const int4 desc = items[item];
    // fetch the next item now; it is read after the reduction's barrier
    if (tid == 0) s_item[1] = atomicAdd(work, 1);
    const int32_t c = desc.x, r0 = desc.y, r1 = desc.y + desc.z;
    int32_t bt[VPL], bd[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) { bt[q] = kTInf; bd[q] = -1; }
    // int16 costs: one 32-bit key per column, ((t + 32768) << 16) | row of
    // the item, so the lexicographic (t, d) minimum is one unsigned min
    // (rows of an item are in increasing d; t fits 16 bits because costs
    // are positive int16)
    uint32_t key[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) key[q] = 0xffffffffu;
    if (g < R) {
      // software pipeline: the unit ids of the next U rows are loaded while
      // the current U rows are loaded and reduced.  Rows of a thread arrive
      // in increasing d, so a strict '<' keeps the lowest d on equal cost.
      int32_t dn[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t pu = r0 + g + u * R;
        dn[u] = pu < r1 ? (int32_t)min((uint32_t)__ldg(perm + pu), (uint32_t)(n - 1)) : -1;
      }
      for (int32_t p = r0 + g; p < r1; p += U * R) {
        int32_t d[U];
#pragma unroll
        for (int u = 0; u < U; ++u) d[u] = dn[u];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t pu = p + (U + u) * R;
          dn[u] = pu < r1 ? (int32_t)min((uint32_t)__ldg(perm + pu), (uint32_t)(n - 1)) : -1;
        }
        int32_t own[U];
        Vec16<T> x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (d[u] >= 0) {
            const T* rp = cm + (int64_t)d[u] * ld;
            own[u] = (int32_t)rp[c];
            x[u] = load16(rp + slot * VPL);
          }
        }
        if constexpr (sizeof(T) == 2) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (d[u] < 0) continue;
            const uint32_t crow = ((uint32_t)(32768 - own[u]) << 16) | (uint32_t)(p + u * R - r0);
            const uint4 wv = *reinterpret_cast<const uint4*>(&x[u]);
            const uint32_t w4[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              key[2 * q] = min(key[2 * q], (w4[q] << 16) + crow);
              key[2 * q + 1] = min(key[2 * q + 1], (w4[q] & 0xffff0000u) + crow);
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (d[u] < 0) continue;
#pragma unroll
            for (int q = 0; q < VPL; ++q) {
              const int32_t t = (int32_t)x[u].v[q] - own[u];
              if (t < bt[q]) { bt[q] = t; bd[q] = d[u]; }
            }
          }
        }
      }
      if constexpr (sizeof(T) == 2) {
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
          if (key[q] != 0xffffffffu) {
            bt[q] = (int32_t)(key[q] >> 16) - 32768;
            bd[q] = (int32_t)min((uint32_t)__ldg(perm + r0 + (int32_t)(key[q] & 0xffffu)),
                                 (uint32_t)(n - 1));
          }
        }
      }
#pragma unroll
      for (int q = 0; q < VPL; ++q) red[g * S * VPL + slot * VPL + q] = make_int2(bt[q], bd[q]);
    }
    __syncthreads();
    for (int col = tid; col < k; col += kThreads) {
      int32_t t = kTInf, dd = -1;
      for (int gg = 0; gg < R; ++gg) {
        const int2 e = red[gg * S * VPL + col];
        if (lex_less(e.x, e.y, t, dd)) { t = e.x; dd = e.y; }
      }
      if (dd >= 0 && col != c) {
        const unsigned long long key =
            ((unsigned long long)(uint32_t)(t + (int64_t)2147483648LL) << 32) | (uint32_t)dd;
        atomicMin(&t64[(int64_t)c * k + col], key);
      }
    }
    item = s_item[1];
    __syncthreads();
    if (tid == 0) s_item[0] = item;   // keep s_item[1] free for the next fetch
  }
}

// ------------------------------------------------ staged int16 row scan ---
//
// The int16 scan of the rows of an item, with each thread's 16-byte chunk of
// a row copied global -> shared by cp.async kStages rows ahead: the bytes in
// flight are bounded by shared memory, not by registers.  A thread waits only
// for its own copies (cp.async.wait_group), so no barrier is involved.  Unit
// ids and own costs (CM(d, c), gathered in sorted order by bt_bounds) travel
// in register rings two and one stages ahead.  Keys as in bt_scan_rows.
constexpr int kStages = 10;

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

size_t bt_staged_smem_bytes() {
  return (size_t)kStages * kThreads * 16 + (size_t)kThreads * 8 * sizeof(int2);
}

__global__ void __launch_bounds__(kThreads, 1)
bt_scan_rows_staged16(const int16_t* __restrict__ cm, int64_t ld, int32_t n, int32_t k,
                      const int32_t* __restrict__ perm, const int32_t* __restrict__ ownv,
                      const int32_t* __restrict__ item_off, const int4* __restrict__ items,
                      unsigned long long* t64, int* work) {
  constexpr int VPL = 8, P = kStages;
  extern __shared__ __align__(16) unsigned char dsm[];
  uint4* stage = reinterpret_cast<uint4*>(dsm);                           // [P][kThreads]
  int2* red = reinterpret_cast<int2*>(dsm + (size_t)P * kThreads * 16);  // [kThreads * VPL]
  __shared__ int s_item[2];
  const int S = (k + VPL - 1) / VPL;
  const int R = kThreads / S;
  const int tid = threadIdx.x, slot = tid % S, g = tid / S;
  const int32_t total = item_off[k];
  if (tid == 0) s_item[0] = atomicAdd(work, 1);
  __syncthreads();
  for (int32_t item = s_item[0];;) {
    if (item >= total) break;
    const int4 desc = items[item];
    if (tid == 0) s_item[1] = atomicAdd(work, 1);
    const int32_t c = desc.x, r0 = desc.y, cnt = desc.z;
    uint32_t key[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) key[q] = 0xffffffffu;
    if (g < R && g < cnt) {
      const int32_t M = (cnt - g + R - 1) / R;        // rows of this thread: g + m * R
      auto row_id = [&](int32_t m) -> int32_t {
        return m < M ? (int32_t)min((uint32_t)__ldg(perm + r0 + g + m * R), (uint32_t)(n - 1)) : 0;
      };
      auto row_own = [&](int32_t m) -> int32_t { return m < M ? __ldg(ownv + r0 + g + m * R) : 0; };
      int32_t idA[P], ownA[P], idB[P], ownB[P], ownS[P];
      // rows 0..P-1 go to the stages now, rows P..2P-1 and 2P..3P-1 are prefetched
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int32_t d0 = row_id(q);
        ownS[q] = row_own(q);
        if (q < M) cp_async16(&stage[q * kThreads + tid], cm + (int64_t)d0 * ld + slot * VPL);
        cp_async_commit();
        idA[q] = row_id(P + q);
        ownA[q] = row_own(P + q);
        idB[q] = row_id(2 * P + q);
        ownB[q] = row_own(2 * P + q);
      }
      for (int32_t m = 0; m < M; m += P) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
          cp_async_wait<P - 1>();                     // row m + q has landed
          if (m + q < M) {
            const uint4 wv = stage[q * kThreads + tid];
            const uint32_t crow = ((uint32_t)(32768 - ownS[q]) << 16) | (uint32_t)(g + (m + q) * R);
            const uint32_t w4[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              key[2 * h] = min(key[2 * h], (w4[h] << 16) + crow);
              key[2 * h + 1] = min(key[2 * h + 1], (w4[h] & 0xffff0000u) + crow);
            }
          }
          // stage q now takes row m + q + P
          if (m + q + P < M) cp_async16(&stage[q * kThreads + tid], cm + (int64_t)idA[q] * ld + slot * VPL);
          cp_async_commit();
          ownS[q] = ownA[q];
          idA[q] = idB[q];
          ownA[q] = ownB[q];
          idB[q] = row_id(m + q + 3 * P);
          ownB[q] = row_own(m + q + 3 * P);
        }
      }
      cp_async_wait<0>();
    }
    if (g < R) {
#pragma unroll
      for (int q = 0; q < VPL; ++q) {
        int32_t bt = kTInf, bd = -1;
        if (key[q] != 0xffffffffu) {
          bt = (int32_t)(key[q] >> 16) - 32768;
          bd = (int32_t)min((uint32_t)__ldg(perm + r0 + (int32_t)(key[q] & 0xffffu)), (uint32_t)(n - 1));
        }
        red[g * S * VPL + slot * VPL + q] = make_int2(bt, bd);
      }
    }
    __syncthreads();
    for (int col = tid; col < k; col += kThreads) {
      int32_t t = kTInf, dd = -1;
      for (int gg = 0; gg < R; ++gg) {
        const int2 e = red[gg * S * VPL + col];
        if (lex_less(e.x, e.y, t, dd)) { t = e.x; dd = e.y; }
      }
      if (dd >= 0 && col != c) {
        const unsigned long long kk =
            ((unsigned long long)(uint32_t)(t + (int64_t)2147483648LL) << 32) | (uint32_t)dd;
        atomicMin(&t64[(int64_t)c * k + col], kk);
      }
    }
    item = s_item[1];
    __syncthreads();
    if (tid == 0) s_item[0] = item;
  }
}

__global__ void __launch_bounds__(kThreads) bt_unpack(const unsigned long long* __restrict__ t64,
                                                      int32_t k, int32_t* tc, int32_t* td,
                                                      const int* err) {
  const bool bad = *err != 0;   // reserved error flag: marks the whole table
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (int64_t)k * k;
       i += (int64_t)gridDim.x * kThreads) {
    const unsigned long long e = t64[i];
    if (bad) {
      tc[i] = kTInf;
      td[i] = -2;
    } else if (e == ~0ull) {
      tc[i] = kTInf;
      td[i] = -1;
    } else {
      tc[i] = (int32_t)((int64_t)(e >> 32) - 2147483648LL);
      td[i] = (int32_t)(e & 0xffffffffu);
    }
  }
}

int bt_max_k(int elem_bytes) { return kThreads * (16 / elem_bytes); }

// Returns a cudaError_t (cudaSuccess on success); argument checks are done
// by the caller.
cudaError_t best_transfer_run(int32_t n, int32_t k, const void* cm, int elem_bytes, int64_t ld,
                              const int32_t* assign, int32_t* tc, int32_t* td, void* ws,
                              cudaStream_t st, int num_sms) {
  void* base = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
  BtWorkspace W = carve(base, n, k);
  const int grid_lin = num_sms * 4;
  bt_init_keys<<<grid_lin, kThreads, 0, st>>>(assign, n, k, W.k0, W.v0);
  const int bits = 32 - __builtin_clz((unsigned)k);   // keys in [0, k]
  const int passes = (bits + 7) / 8;
  int32_t *sk = W.k0, *sv = W.v0, *dk = W.k1, *dv = W.v1;
  for (int p = 0; p < passes; ++p) {
    bt_hist<<<(unsigned)W.ntiles, kThreads, 0, st>>>(sk, n, 8 * p, W.tile_hist, W.ntiles);
    bt_digit_sums<<<256, kThreads, 0, st>>>(W.tile_hist, W.ntiles, W.dsum);
    bt_digit_scan<<<256, kThreads, 0, st>>>(W.tile_hist, W.ntiles, W.dsum);
    bt_scatter<<<(unsigned)W.ntiles, kThreads, 0, st>>>(sk, sv, dk, dv, n, 8 * p, W.tile_hist,
                                                        W.ntiles);
    std::swap(sk, dk);
    std::swap(sv, dv);
  }
  cudaMemsetAsync(W.seg_start, 0, 4ull * k, st);
  cudaMemsetAsync(W.seg_end, 0, 4ull * k, st);
  bt_bounds<<<grid_lin, kThreads, 0, st>>>(sk, sv, n, k, W.seg_start, W.seg_end,
                                            elem_bytes == 2 ? static_cast<const int16_t*>(cm)
                                                            : nullptr,
                                            ld, W.ownv);
  bt_items<<<grid_lin, kThreads, 0, st>>>(W.seg_start, W.seg_end, k, W.item_off, W.t64);
  bt_scan<<<1, kThreads, 0, st>>>(W.item_off, k, W.item_off + k);
  const int grid_scan = num_sms;
  cudaMemsetAsync(W.err, 0, 2 * sizeof(int), st);
  bt_item_list<<<grid_lin, kThreads, 0, st>>>(W.seg_start, W.seg_end, W.item_off, k, W.items);
  if (elem_bytes == 2) {
    // the staged kernel's dynamic shared memory, set once per device
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!(attr_set.load() & (1ull << dev))) {
      e = cudaFuncSetAttribute(bt_scan_rows_staged16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bt_staged_smem_bytes());
      if (e != cudaSuccess) return e;
      attr_set.fetch_or(1ull << dev);
    }
    bt_scan_rows_staged16<<<grid_scan, kThreads, bt_staged_smem_bytes(), st>>>(
        static_cast<const int16_t*>(cm), ld, n, k, sv, W.ownv, W.item_off, W.items, W.t64,
        W.err + 1);
  } else {
    bt_scan_rows<int32_t><<<grid_scan, kThreads, 0, st>>>(
        static_cast<const int32_t*>(cm), ld, n, k, sv, W.item_off, W.items, W.t64, W.err + 1);
  }
  bt_unpack<<<grid_lin, kThreads, 0, st>>>(W.t64, k, tc, td, W.err);
  return cudaGetLastError();
}

}  // namespace lbdd
