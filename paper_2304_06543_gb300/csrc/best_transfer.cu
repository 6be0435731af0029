// Best-transfer table from scratch: the data-parallel replacement of the
// paper's Gamma-DS heap maintenance (Section 3.4 "Allotment subspace
// multi-graph implementation", Section 3.5.2), which took 74% of ASRAL's time
// in the paper's measurements (Section 5).
//
//   T[u][v] = lexmin over d with assign[d] == u of (CM(d,v) - CM(d,u), d)
//
// Pipeline (all device-side, one stream):
//   1. bt_count: units per center.  kTiles CTAs, each a contiguous range of
//      units, count in shared memory; one returned atomic per (tile, center)
//      adds the tile's count to the center's total and gives the tile its
//      block inside the center's segment;
//   2. bt_plan (one CTA): segment offsets from the totals, and work items of
//      at most `chunk` rows of one center, `chunk` chosen so that every SM
//      gets about kItemsPerSm items;
//   3. bt_place: each tile writes its units into its blocks (shared-memory
//      cursors; the order inside a block is arbitrary);
//   4. bt_sort_items: the unit ids of every item in ascending order (bitonic:
//      shuffles below a stride of 32, shared memory above), so that inside
//      an item a lower row index is a lower d; the packed table is set to its
//      identity in the same launch;
//   5. the scan: CM rows are streamed and every 16-byte column group keeps a
//      running lexicographic minimum; at the end of an item (or of a CTA's
//      share of one) the partial minima are folded in shared memory and
//      merged into a packed (cost, d) 64-bit table with atomicMin.  Rows of
//      512 bytes and more: bt_scan_bulk, every CTA an equal contiguous share
//      of the grouped rows, staged whole by bulk copies; shorter rows:
//      bt_scan_rows, items from a queue, 16 bytes per thread and load;
//   6. bt_unpack: the (tc, td) int32 pair.
// Step 5 reads every CM byte of the allotted rows once and is the HBM-bound
// kernel; the other steps move O(n + k*k) bytes.
//
// Tables of 256 to 512 centers take a shorter path with no grouping (rows of
// 512 bytes to 2 KB gather poorly): bt_own, then bt_scan_stream reads the CM
// in row order, one 128-byte column slice and one row range per CTA, keeping
// the minima in shared memory, and bt_merge_ranges combines the ranges into
// (tc, td).
#include <atomic>
#include <algorithm>

#include "lbdd_device.cuh"

namespace lbdd {

constexpr int kChunkMax = 512;          // rows per work item, at most (16-bit row index)
constexpr int kChunkMin = 64;           // rows per work item, at least (bounds the item count)
constexpr int kItemsPerSm = 8;          // work items per SM the plan aims for
constexpr int kScanUnroll = 6;          // bt_scan_rows: rows in flight per thread
constexpr int kTiles = 64;              // unit ranges of bt_count / bt_place
constexpr int kTileThreads = 1024;
constexpr int kTileUnroll = 8;          // assign loads in flight per thread

// ctl words (int32): error flag, scan queue, item count, chunk, allotted rows
enum { BT_ERR = 0, BT_QUEUE, BT_ITEMS, BT_CHUNK, BT_ROWS, BT_CTL_WORDS = 8 };

struct BtWorkspace {
  int* ctl;                     // BT_CTL_WORDS control words
  int32_t* cnt;                 // k + 1: units per center, then segment starts (cnt[k] = rows)
  int32_t* tile_rel;            // kTiles x k: a tile's block offset inside a center's segment
  int32_t* perm;                // n (+ 4 readable): allotted units grouped by center
  int4* items;                  // n / kChunkMin + k + 1 items {center, first row, rows, 0}
  unsigned long long* t64;      // k x k packed ((cost + 2^31) << 32) | d
  uint32_t* part;               // row-order path: one k x k key table per row range
  size_t bytes;
};

// Row-order path (bt_scan_stream): centers in [kStreamMinK, kStreamMaxK];
// int16: at most kStreamMaxRanges row ranges of at most kStreamRowSpan rows,
// int32: at most kStreamMaxRanges / 2 ranges (twice as wide keys, the same
// bytes of partial tables).
constexpr int kStreamMinK = 256, kStreamMaxK = 512;
constexpr int kStreamMaxRanges = 32;
constexpr int64_t kStreamRowSpan = 65536;  // the 16-bit row offset of a key

static size_t stream_part_bytes(int32_t n, int32_t k) {
  if (k < kStreamMinK || k > kStreamMaxK) return 0;
  return 4ull * k * k * (size_t)std::min<int32_t>(kStreamMaxRanges, n);
}

static inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static BtWorkspace carve(void* base, int32_t n, int32_t k) {
  BtWorkspace W;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = static_cast<char*>(base) + o;
    o = al256(o + bytes);
    return p;
  };
  // ctl then cnt: one memset clears both
  W.ctl = reinterpret_cast<int*>(take(4 * BT_CTL_WORDS + 4ull * (k + 1)));
  W.cnt = W.ctl + BT_CTL_WORDS;
  W.tile_rel = reinterpret_cast<int32_t*>(take(4ull * kTiles * k));
  W.perm = reinterpret_cast<int32_t*>(take(4ull * n + 16));   // id windows round up to 16 bytes
  W.items = reinterpret_cast<int4*>(take(16ull * ((size_t)n / kChunkMin + (size_t)k + 1)));
  W.t64 = reinterpret_cast<unsigned long long*>(take(8ull * k * k));
  W.part = reinterpret_cast<uint32_t*>(take(stream_part_bytes(n, k)));
  W.bytes = o;
  return W;
}

size_t bt_workspace_bytes(int32_t n, int32_t k) {
  if (n < 1 || k < 1) return 0;
  return carve(nullptr, n, k).bytes + 256;
}

// ------------------------------------------------------------- grouping ---

// Units of this CTA's tile: [t * per, min(n, (t + 1) * per)).
__device__ __forceinline__ void tile_range(int32_t n, int64_t* lo, int64_t* hi) {
  const int64_t per = ((int64_t)n + kTiles - 1) / kTiles;
  *lo = min((int64_t)n, (int64_t)blockIdx.x * per);
  *hi = min((int64_t)n, *lo + per);
}

// Units per center and per (tile, center).  Entries of assign outside
// [0, k) are not counted.
__global__ void __launch_bounds__(kTileThreads) bt_count(const int32_t* __restrict__ assign,
                                                         int32_t n, int32_t k, int32_t* cnt,
                                                         int32_t* tile_rel) {
  extern __shared__ int32_t h[];   // k counters
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += kTileThreads) h[i] = 0;
  __syncthreads();
  int64_t lo, hi;
  tile_range(n, &lo, &hi);
  for (int64_t b = lo; b < hi; b += (int64_t)kTileThreads * kTileUnroll) {
    int32_t a[kTileUnroll];
#pragma unroll
    for (int u = 0; u < kTileUnroll; ++u) {
      const int64_t i = b + u * kTileThreads + tid;
      a[u] = i < hi ? assign[i] : -1;
    }
#pragma unroll
    for (int u = 0; u < kTileUnroll; ++u)
      if (a[u] >= 0 && a[u] < k) atomicAdd(&h[a[u]], 1);
  }
  __syncthreads();
  for (int i = tid; i < k; i += kTileThreads)
    if (h[i]) tile_rel[(int64_t)blockIdx.x * k + i] = atomicAdd(&cnt[i], h[i]);
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

// One CTA of kThreads: segment starts (exclusive prefix of the counts,
// centers in index order) into cnt[0..k), the allotted total into cnt[k],
// and the work items.  Clears the scan queue; records the item count, the
// chunk and the allotted rows in ctl.
__global__ void __launch_bounds__(kThreads) bt_plan(int32_t* cnt, int32_t k, int num_sms,
                                                    int4* items, int* ctl) {
  __shared__ int32_t s_warp[kWarps];
  const int tid = threadIdx.x;
  const int per = (k + kThreads - 1) / kThreads;
  const int c0 = min(k, tid * per), c1 = min(k, c0 + per);
  int32_t rows = 0;
  for (int c = c0; c < c1; ++c) rows += cnt[c];
  int32_t total;
  int32_t r = block_exclusive_scan(rows, s_warp, &total);
  const int64_t want = (int64_t)num_sms * kItemsPerSm;
  const int64_t even = ((int64_t)total + want - 1) / want;
  const int32_t chunk = (int32_t)(even < kChunkMin ? kChunkMin : even > kChunkMax ? kChunkMax : even);
  int32_t its = 0;
  for (int c = c0; c < c1; ++c) its += (cnt[c] + chunk - 1) / chunk;
  __syncthreads();                       // s_warp is reused
  int32_t nitems;
  int32_t it = block_exclusive_scan(its, s_warp, &nitems);
  for (int c = c0; c < c1; ++c) {
    const int32_t m = cnt[c];
    for (int32_t j = 0; j < m; j += chunk) items[it++] = make_int4(c, r + j, min(chunk, m - j), 0);
    cnt[c] = r;
    r += m;
  }
  if (tid == 0) {
    cnt[k] = total;
    ctl[BT_QUEUE] = 0;
    ctl[BT_ITEMS] = nitems;
    ctl[BT_CHUNK] = chunk;
    ctl[BT_ROWS] = total;
  }
}

// Each tile's units into its blocks: cursor of center c = segment start +
// the tile's offset, advanced by shared-memory atomics.
__global__ void __launch_bounds__(kTileThreads) bt_place(const int32_t* __restrict__ assign,
                                                         int32_t n, int32_t k,
                                                         const int32_t* __restrict__ seg,
                                                         const int32_t* __restrict__ tile_rel,
                                                         int32_t* perm) {
  extern __shared__ int32_t cur[];   // k cursors (entries of centers absent from the tile unused)
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += kTileThreads)
    cur[i] = (int32_t)((uint32_t)seg[i] + (uint32_t)tile_rel[(int64_t)blockIdx.x * k + i]);
  __syncthreads();
  int64_t lo, hi;
  tile_range(n, &lo, &hi);
  for (int64_t b = lo; b < hi; b += (int64_t)kTileThreads * kTileUnroll) {
    int32_t a[kTileUnroll];
#pragma unroll
    for (int u = 0; u < kTileUnroll; ++u) {
      const int64_t i = b + u * kTileThreads + tid;
      a[u] = i < hi ? assign[i] : -1;
    }
#pragma unroll
    for (int u = 0; u < kTileUnroll; ++u)
      if (a[u] >= 0 && a[u] < k)
        perm[atomicAdd(&cur[a[u]], 1)] = (int32_t)(b + u * kTileThreads + tid);
  }
}

// The unit ids of each item in ascending order, one item per CTA at a time:
// thread i holds element i; compare-exchange partners at a stride below 32
// are reached by shuffles, the others through a double-buffered shared
// array (one barrier per step).  Also sets the packed table to ~0.
__global__ void __launch_bounds__(kThreads) bt_sort_items(const int4* __restrict__ items,
                                                          const int* __restrict__ ctl,
                                                          int32_t* perm, int32_t k,
                                                          unsigned long long* t64) {
  __shared__ int32_t xs[2][kChunkMax];
  const int tid = threadIdx.x;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + tid; i < (int64_t)k * k;
       i += (int64_t)gridDim.x * kThreads)
    t64[i] = ~0ull;
  const int total = ctl[BT_ITEMS];
  int buf = 0;     // kept across items: consecutive shared steps alternate buffers
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int4 desc = items[it];
    const int32_t r0 = desc.y, m = desc.z;
    if (m <= 1) continue;
    int P = 2;
    while (P < m) P <<= 1;
    int32_t v = tid < m ? perm[r0 + tid] : INT32_MAX;
    for (int size = 2; size <= P; size <<= 1) {
      const bool up = (tid & size) == 0;
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        int32_t w;
        if (stride >= 32) {
          xs[buf][tid] = v;
          __syncthreads();
          w = xs[buf][tid ^ stride];
          buf ^= 1;
        } else {
          w = __shfl_xor_sync(0xffffffffu, v, stride);
        }
        v = (((tid & stride) == 0) == up) ? min(v, w) : max(v, w);
      }
    }
    if (tid < m) perm[r0 + tid] = v;
  }
}

// ------------------------------------------------------------------ scan ---
//
// Keys of the int16 scan: one 32-bit key per column, ((t + 32768) << 16) |
// row of the item, so the lexicographic (t, d) minimum is one unsigned min
// (rows of an item are in increasing d; t fits 16 bits because costs are
// positive int16).  The int32 scan keeps (t, row) pairs with a strict '<':
// a thread sees the rows of an item in increasing order.

// Rows shorter than 512 bytes: every thread loads its 16-byte column group
// of kScanUnroll rows at once, and the unit ids of the next kScanUnroll rows
// while those are reduced.
template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
bt_scan_rows(const T* __restrict__ cm, int64_t ld, int32_t n, int32_t k,
             const int32_t* __restrict__ perm, const int4* __restrict__ items,
             unsigned long long* t64, int* ctl) {
  constexpr int VPL = 16 / (int)sizeof(T);
  constexpr int U = kScanUnroll;
  __shared__ int2 red[kThreads * VPL];
  __shared__ int s_item[2];
  const int S = (k + VPL - 1) / VPL;       // 16-byte column groups per row
  const int R = kThreads / S;              // row groups
  const int tid = threadIdx.x, slot = tid % S, g = tid / S;
  const int32_t total = ctl[BT_ITEMS];
  int* work = ctl + BT_QUEUE;
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
    uint32_t key[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) key[q] = 0xffffffffu;
    if (g < R) {
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
        const unsigned long long pk =
            ((unsigned long long)(uint32_t)(t + (int64_t)2147483648LL) << 32) | (uint32_t)dd;
        atomicMin(&t64[(int64_t)c * k + col], pk);
      }
    }
    item = s_item[1];
    __syncthreads();
    if (tid == 0) s_item[0] = item;   // keep s_item[1] free for the next fetch
  }
}


// ---------------------------------------------------- bulk-copy row scan ---
//
// Rows of kBulkMinRowBytes and more.  CTA b scans the grouped rows
// [b * rows / G, (b + 1) * rows / G) of perm: equal bytes per CTA, no work
// queue.  Warp kWarps (the producer) walks that range: the segment starts
// (all k + 1 of them, copied into shared memory at start) give the center
// and the item boundaries of every position, the unit ids arrive in windows
// of kIdsWin by bulk copy one window ahead, and every CM row is copied whole
// global -> shared by one bulk copy (cp.async.bulk) into a ring of NS stages
// of at most RS rows of one item; a stage's barrier `full` completes once all
// of its bytes have landed.  The kWarps consumer warps scan the staged rows
// (one 16-byte column group per thread, R row groups; a row's own cost
// CM(d, c) is read from the staged row itself) and release the stage on its
// barrier `empty`.  At the end of an item, or of the part of it in this
// CTA's range, the consumers fold their partial minima (barrier `fold`,
// double-buffered) while the producer goes on filling stages.  Every wait is
// bounded: past kScanWaitLimitNs the waiter sets ctl[BT_ERR] and leaves (the
// producer first waits, bounded, for its copies in flight), and bt_unpack
// then marks the whole table.
constexpr int kBulkMinRowBytes = 512;
constexpr int kStageBytes = 32768;       // target bytes per stage (the producer's cost is per stage)
constexpr int kSmemLimit = 232448;       // dynamic shared memory of one CTA (227 KB)
constexpr int kMaxStages = 16;
constexpr int kIdsWin = 1024;            // unit ids per window (two windows in shared memory)
constexpr int kRedBytes = kThreads * 32; // one fold buffer: R*S*VPL keys (int16) or pairs (int32)
constexpr int kBulkThreads = kThreads + 32;
constexpr int kFoldCols = 8;             // columns per consumer thread in a fold (k <= 4096)
constexpr uint64_t kScanWaitLimitNs = 1000000000ull;
constexpr uint32_t kScanSleepNs = 1000000;

struct StageMeta {
  int32_t c;      // center of the rows
  int32_t r0;     // position in perm of the first row of the fold unit
  int32_t j;      // position of the stage's first row inside the fold unit
  int32_t rows;   // rows in the stage; -1 marks the end of the work
  int32_t last;   // the stage ends its fold unit
  int32_t pad0, pad1, pad2;
};

struct BulkShape {
  int S, R, RS, NS, row_bytes, stage_bytes;
};

__host__ __device__ inline size_t seg_smem_bytes(int32_t k) { return ((4 * (size_t)(k + 1)) + 15) & ~(size_t)15; }

// Shared memory besides the stages (fold buffers, id windows, segment
// starts, stage descriptors and barriers, the latter two at their largest).
static size_t bulk_fixed_bytes(int32_t k) {
  return 2 * (size_t)kRedBytes + 8 * (size_t)kIdsWin + seg_smem_bytes(k) +
         (size_t)kMaxStages * sizeof(StageMeta) + (2 * (size_t)kMaxStages + 3) * 8;
}

static BulkShape bulk_shape(int32_t k, int elem) {
  BulkShape p;
  const int VPL = 16 / elem;
  p.S = (k + VPL - 1) / VPL;
  p.R = kThreads / p.S;
  p.row_bytes = p.S * 16;
  const int per = std::max(1, kStageBytes / p.row_bytes);
  p.RS = std::min(32, std::max(p.R, per / p.R * p.R));
  p.stage_bytes = p.RS * p.row_bytes;
  p.NS = std::max(2, std::min<int>(kMaxStages, (int)((kSmemLimit - bulk_fixed_bytes(k)) / p.stage_bytes)));
  return p;
}

static size_t bulk_smem_bytes(const BulkShape& p, int32_t k) {
  return (size_t)p.NS * p.stage_bytes + 2 * (size_t)kRedBytes + 8 * (size_t)kIdsWin +
         seg_smem_bytes(k) + (size_t)p.NS * sizeof(StageMeta) + (2 * (size_t)p.NS + 3) * 8;
}

// Largest dynamic shared memory any shape needs (the attribute set once).
static size_t bulk_smem_max() { return kSmemLimit; }

__device__ __forceinline__ bool scan_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer_ns();
  while (!mbar_try_wait(bar, parity, kScanSleepNs))
    if (gtimer_ns() - t0 > kScanWaitLimitNs) return false;
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kBulkThreads, 1)
bt_scan_bulk(const T* __restrict__ cm, int64_t ld, int32_t k, const int32_t* __restrict__ perm,
             const int32_t* __restrict__ seg, unsigned long long* t64, int* ctl, BulkShape p) {
  constexpr int VPL = 16 / (int)sizeof(T);
  extern __shared__ __align__(128) unsigned char dsm[];
  const int NS = p.NS, SB = p.stage_bytes, RB = p.row_bytes;
  unsigned char* stages = dsm;
  unsigned char* redb = dsm + (size_t)NS * SB;
  int32_t* s_ids = reinterpret_cast<int32_t*>(redb + 2 * kRedBytes);       // 2 windows
  int32_t* s_seg = s_ids + 2 * kIdsWin;                                    // k + 1
  StageMeta* meta = reinterpret_cast<StageMeta*>(reinterpret_cast<unsigned char*>(s_seg) +
                                                 seg_smem_bytes(k));
  uint64_t* full = reinterpret_cast<uint64_t*>(meta + NS);
  uint64_t* empty = full + NS;
  uint64_t* fold = empty + NS;
  uint64_t* idsbar = fold + 1;                                             // 2
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t rows_total = ctl[BT_ROWS], chunk = ctl[BT_CHUNK];
  const int32_t P0 = (int32_t)((int64_t)blockIdx.x * rows_total / gridDim.x);
  const int32_t P1 = (int32_t)((int64_t)(blockIdx.x + 1) * rows_total / gridDim.x);
  if (tid < NS) {
    mbar_init(&full[tid], 1);
    mbar_init(&empty[tid], kWarps);
  }
  if (tid == 0) {
    mbar_init(fold, kWarps);
    mbar_init(&idsbar[0], 1);
    mbar_init(&idsbar[1], 1);
    mbar_fence_init();
  }
  for (int i = tid; i <= k; i += kBulkThreads) s_seg[i] = seg[i];
  __syncthreads();

  if (warp == kWarps) {
    // ---------------------------------------------------------- producer
    const int32_t A = P0 & ~3;                        // 16-byte aligned start of the id windows
    const int nwin = P1 > P0 ? (P1 - A + kIdsWin - 1) / kIdsWin : 0;
    int issued = -1, ready = -1;                      // id windows copied / waited for
    int s = 0, fills = 0;
    uint32_t eph = 0;                                 // slot s is free once phase eph ^ 1 completed
    bool ok = true;
    // center of P0: the largest c with seg[c] <= P0 (it is not empty)
    int c = 0;
    if (P0 < P1) {
      int lo = 0, hi = k - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_seg[mid] <= P0) lo = mid; else hi = mid - 1;
      }
      c = lo;
    }
    int32_t sb = s_seg[c], se = s_seg[c + 1];
    int32_t win_end = A;                              // ids below this position have landed
    int32_t pos = P0;
    // one fold unit per pass: the part of an item inside [P0, P1)
    while (ok && pos < P1) {
      while (se <= pos) { ++c; sb = s_seg[c]; se = s_seg[c + 1]; }
      const int32_t u0 = pos;
      const int32_t len = min(min(se, sb + ((pos - sb) / chunk + 1) * chunk), P1) - u0;
      for (int32_t j = 0; j < len; j += p.RS) {
        const int rows = min(p.RS, len - j);
        const int32_t q = u0 + j;
        if (q + rows > win_end || (issued < nwin - 1 && q >= A + issued * kIdsWin)) {
          // the window after q's goes out as soon as q enters q's window (its
          // buffer held the window before q's, whose rows are all issued);
          // then wait for the windows this stage reads
          const int wlast = min((q - A) / kIdsWin + 1, nwin - 1);
          while (issued < wlast) {
            ++issued;
            if (lane == 0) {
              const int32_t first = A + issued * kIdsWin;
              const uint32_t bytes = ((uint32_t)min(kIdsWin, P1 - first) * 4u + 15u) & ~15u;
              fence_proxy_async_smem();
              mbar_arrive_expect(&idsbar[issued & 1], bytes);
              bulk_load_smem(smem_u32(s_ids + (issued & 1) * kIdsWin), perm + first, bytes,
                             smem_u32(&idsbar[issued & 1]));
            }
          }
          const int wneed = (q + rows - 1 - A) / kIdsWin;
          while (ok && ready < wneed) {
            ++ready;
            ok = scan_wait(&idsbar[ready & 1], (ready >> 1) & 1);
          }
          win_end = A + (ready + 1) * kIdsWin;
          if (!ok) break;
        }
        if (!scan_wait(&empty[s], eph ^ 1)) { ok = false; break; }
        if (lane == 0) {
          StageMeta m;
          m.c = c; m.r0 = u0; m.j = j; m.rows = rows; m.last = j + p.RS >= len;
          m.pad0 = m.pad1 = m.pad2 = 0;
          meta[s] = m;
          mbar_arrive_expect(&full[s], (uint32_t)(rows * RB));
        }
        __syncwarp();
        const uint32_t dst = smem_u32(stages + (size_t)s * SB);
        for (int i = lane; i < rows; i += 32) {
          const int32_t d = s_ids[(q + i - A) & (2 * kIdsWin - 1)];
          bulk_load_smem(dst + (uint32_t)(i * RB), cm + (int64_t)d * ld, (uint32_t)RB,
                         smem_u32(&full[s]));
        }
        ++fills;
        if (++s == NS) { s = 0; eph ^= 1; }
      }
      pos = u0 + len;
    }
    if (ok) {
      if (scan_wait(&empty[s], eph ^ 1)) {
        if (lane == 0) {
          meta[s].rows = -1;     // end of the work
          mbar_arrive(&full[s]);
        }
      } else {
        ok = false;
      }
    }
    if (!ok) {
      if (lane == 0) atomicExch(&ctl[BT_ERR], 1);
      // copies still in flight: the last NS stage fills and unwaited id windows
      for (int f = max(0, fills - NS); f < fills; ++f) scan_wait(&full[f % NS], (f / NS) & 1);
      for (int w = ready + 1; w <= issued; ++w) scan_wait(&idsbar[w & 1], (w >> 1) & 1);
    }
    return;
  }

  // ------------------------------------------------------------ consumers
  const int S = p.S, R = p.R;
  const int slot = tid % S, g = tid / S;
  const bool act = g < R;
  int s = 0, rb = 0;
  uint32_t fph = 0, cph = 0;
  uint32_t key[VPL];
  int32_t bt[VPL], br[VPL];
#pragma unroll
  for (int q = 0; q < VPL; ++q) { key[q] = 0xffffffffu; bt[q] = kTInf; br[q] = -1; }
  for (;;) {
    if (!scan_wait(&full[s], fph)) {
      if (lane == 0) atomicExch(&ctl[BT_ERR], 1);
      break;
    }
    const StageMeta m = meta[s];
    if (m.rows < 0) break;
    if (act) {
      const unsigned char* sbase = stages + (size_t)s * SB;
      for (int i = g; i < m.rows; i += R) {
        const T* row = reinterpret_cast<const T*>(sbase + (size_t)i * RB);
        const int32_t own = (int32_t)row[m.c];
        const uint4 wv = reinterpret_cast<const uint4*>(row)[slot];
        const int32_t ri = m.j + i;
        if constexpr (sizeof(T) == 2) {
          const uint32_t crow = ((uint32_t)(32768 - own) << 16) | (uint32_t)ri;
          const uint32_t w4[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            key[2 * h] = min(key[2 * h], (w4[h] << 16) + crow);
            key[2 * h + 1] = min(key[2 * h + 1], (w4[h] & 0xffff0000u) + crow);
          }
        } else {
          const int32_t w4[4] = {(int32_t)wv.x, (int32_t)wv.y, (int32_t)wv.z, (int32_t)wv.w};
#pragma unroll
          for (int q = 0; q < VPL; ++q) {
            const int32_t t = w4[q] - own;
            if (t < bt[q]) { bt[q] = t; br[q] = ri; }
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (++s == NS) { s = 0; fph ^= 1; }
    if (!m.last) continue;
    // end of a fold unit: fold the row groups, merge into the table
    unsigned char* red = redb + (size_t)rb * kRedBytes;
    if (act) {
#pragma unroll
      for (int q = 0; q < VPL; ++q) {
        const int at = g * S * VPL + slot * VPL + q;
        if constexpr (sizeof(T) == 2) reinterpret_cast<uint32_t*>(red)[at] = key[q];
        else reinterpret_cast<int2*>(red)[at] = make_int2(bt[q], br[q]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(fold);
    if (!scan_wait(fold, cph)) {
      if (lane == 0) atomicExch(&ctl[BT_ERR], 1);
      break;
    }
    cph ^= 1;
    int32_t ft[kFoldCols], fr[kFoldCols];
#pragma unroll
    for (int q = 0; q < kFoldCols; ++q) {
      const int col = tid + q * kThreads;
      ft[q] = kTInf;
      fr[q] = -1;
      if (col < k) {
        if constexpr (sizeof(T) == 2) {
          uint32_t b = 0xffffffffu;
          for (int gg = 0; gg < R; ++gg)
            b = min(b, reinterpret_cast<const uint32_t*>(red)[gg * S * VPL + col]);
          if (b != 0xffffffffu) { ft[q] = (int32_t)(b >> 16) - 32768; fr[q] = (int32_t)(b & 0xffffu); }
        } else {
          for (int gg = 0; gg < R; ++gg) {
            const int2 e = reinterpret_cast<const int2*>(red)[gg * S * VPL + col];
            if (e.y >= 0 && (fr[q] < 0 || e.x < ft[q] || (e.x == ft[q] && e.y < fr[q]))) {
              ft[q] = e.x;
              fr[q] = e.y;
            }
          }
        }
      }
    }
    int32_t fd[kFoldCols];
#pragma unroll
    for (int q = 0; q < kFoldCols; ++q) fd[q] = fr[q] >= 0 ? perm[m.r0 + fr[q]] : -1;
#pragma unroll
    for (int q = 0; q < kFoldCols; ++q) {
      const int col = tid + q * kThreads;
      if (fr[q] >= 0 && col != m.c) {
        const unsigned long long pk =
            ((unsigned long long)(uint32_t)(ft[q] + (int64_t)2147483648LL) << 32) | (uint32_t)fd[q];
        atomicMin(&t64[(int64_t)m.c * k + col], pk);
      }
    }
    rb ^= 1;
#pragma unroll
    for (int q = 0; q < VPL; ++q) { key[q] = 0xffffffffu; bt[q] = kTInf; br[q] = -1; }
  }
}

__global__ void __launch_bounds__(kThreads) bt_unpack(const unsigned long long* __restrict__ t64,
                                                      int32_t k, int32_t* tc, int32_t* td,
                                                      const int* ctl) {
  const bool bad = ctl[BT_ERR] != 0;   // a scan wait ran out: the whole table is marked
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

// ------------------------------------------------------------ row order ---
//
// Rows of kStreamMinK..kStreamMaxK centers (512 bytes to 2 KB) are short for
// row gathers, so this path reads the CM in row order instead and needs no
// grouping.  CTA (j, r) owns the 128-byte column slice j (64 int16 or 32 int32
// columns) and the row range r, and keeps in shared memory one key per
// (center, column of the slice): ((t + 32768) << 16) | (d - first row of the
// range) in 32 bits for int16, ((t + 2^31) << 32) | (d - first row) in 64
// bits for int32, so the smaller key is the lexicographically smaller (t, d)
// inside the range.  A thread
// owns 16 bytes (8 columns) of every 128th row; each is copied into the
// thread's own shared slot by cp.async kStreamStages rows ahead (the bytes in
// flight are bounded by shared memory, not registers), then the thread
// compares its keys with the table and lowers an entry with a shared atomicMin only where its
// key is smaller (entries only decrease, so a stale read never hides a
// smaller key).  A table row (256 bytes) is laid out as two halves: the
// first half of every thread's keys in the first 128 bytes, the other half in
// the second, so each 128-bit shared load of 8 threads covers 32 banks.  bt_own gathers
// CM(d, assign[d]) first; bt_merge_ranges takes, for every (u, v), the
// smallest t over the ranges in range order (ranges ascend in d, so the first
// range that attains it holds the smallest d) and writes tc/td.
constexpr int kStreamThreads = 1024;    // 8 threads per 128-byte row slice, 128 rows at a time
constexpr int kStreamStages = 5;        // rows in flight per thread (cp.async stages)

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Per cost type: columns per slice (128 bytes of a row), the key, and the
// key's split into cost and row offset.  A key row is 256 bytes either way.
template <typename T> struct StreamKey;
template <> struct StreamKey<int16_t> {
  using K = uint32_t;                    // ((t + 32768) << 16) | row offset
  static constexpr int kCols = 64;
  static __device__ __forceinline__ int32_t cost(K key) { return (int32_t)(key >> 16) - 32768; }
  static __device__ __forceinline__ uint32_t offset(K key) { return key & 0xffffu; }
};
template <> struct StreamKey<int32_t> {
  using K = unsigned long long;          // ((t + 2^31) << 32) | row offset
  static constexpr int kCols = 32;
  static __device__ __forceinline__ int32_t cost(K key) {
    return (int32_t)((int64_t)(key >> 32) - 2147483648LL);
  }
  static __device__ __forceinline__ uint32_t offset(K key) { return (uint32_t)key; }
};

// Programmatic dependent launch: a kernel launched with the attribute may
// start while its predecessor on the stream still runs; it waits here until
// the predecessor's results are visible (a no-op for an ordinary launch).
__device__ __forceinline__ void wait_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel on the stream start launching.
__device__ __forceinline__ void release_successor() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Dynamic shared memory of bt_scan_stream: the key table, then the stages.
static size_t stream_smem_bytes(int32_t k) {
  return 256 * (size_t)k + (size_t)kStreamStages * kStreamThreads * 16;
}

// Row ranges of the row-order path on `num_sms` SMs, 0 if it does not apply.
// int16 keys hold a 16-bit row offset (ranges of at most kStreamRowSpan
// rows); int32 keys are twice as wide, so at most half as many ranges fit the
// partial tables' bytes.
static int stream_ranges(int32_t n, int32_t k, int elem, int num_sms) {
  if (k < kStreamMinK || k > kStreamMaxK) return 0;
  const int cols = elem == 2 ? StreamKey<int16_t>::kCols : StreamKey<int32_t>::kCols;
  const int64_t need = elem == 2 ? ((int64_t)n + kStreamRowSpan - 1) / kStreamRowSpan : 1;
  const int64_t cap = elem == 2 ? std::min<int64_t>(kStreamMaxRanges, n)
                                : std::min<int64_t>(kStreamMaxRanges / 2, n / 2);
  if (cap < 1 || need > cap) return 0;
  const int nslice = (k + cols - 1) / cols;
  return (int)std::min<int64_t>(cap, std::max<int64_t>(need, num_sms / nslice));
}

template <typename T>
__global__ void __launch_bounds__(kThreads) bt_own(const int32_t* __restrict__ assign, int32_t n,
                                                   int32_t k, const T* __restrict__ cm,
                                                   int64_t ld, int32_t* own) {
  release_successor();
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const int32_t a = assign[i];
    own[i] = (a >= 0 && a < k) ? (int32_t)cm[i * ld + a] : 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kStreamThreads, 1)
bt_scan_stream(const T* __restrict__ cm, int64_t ld, int32_t n, int32_t k,
               const int32_t* __restrict__ assign, const int32_t* __restrict__ own, int nslice,
               int nranges, typename StreamKey<T>::K* part) {
  using K = typename StreamKey<T>::K;
  constexpr int COLS = StreamKey<T>::kCols;
  constexpr int VPL = 16 / (int)sizeof(T);   // columns per thread (16 bytes)
  constexpr int HALF = VPL / 2;              // keys per 16-byte half
  constexpr int P = kStreamStages;
  extern __shared__ __align__(16) unsigned char stream_smem[];
  K* acc = reinterpret_cast<K*>(stream_smem);   // k rows of COLS keys, then the stages
  const int tid = threadIdx.x, cg = tid & 7, rl = tid >> 3;
  const int j = blockIdx.x % nslice, r = blockIdx.x / nslice;
  const int64_t R0 = (int64_t)r * n / nranges, R1 = (int64_t)(r + 1) * n / nranges;
  const int c0 = j * COLS;
  const int w = min(COLS, k - c0);
  const bool act = cg * VPL < w;
  const uint4 none = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
  for (int i = tid; i < k * 16; i += kStreamThreads) reinterpret_cast<uint4*>(acc)[i] = none;
  __syncthreads();
  wait_predecessor();   // own[] comes from bt_own
  const T* colp = cm + c0 + cg * VPL;
  // rows of this thread: R0 + rl + 128 i, i < M; row i's 16 bytes go to
  // stage i % P of the thread's own shared slots P rows ahead (cp.async: a
  // thread waits only for its own copies, no barrier), its center and own
  // cost to a register ring P rows ahead
  const int64_t span = R1 - R0;
  const int32_t M = act && rl < span ? (int32_t)((span - rl + 127) / 128) : 0;
  uint4* stage = reinterpret_cast<uint4*>(stream_smem + 256 * (size_t)k);   // [P][kStreamThreads]
  int32_t ra[P], ro[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int64_t d = R0 + rl + 128 * q;
    ra[q] = -1;
    ro[q] = 0;
    if (q < M) {
      cp_async16(&stage[q * kStreamThreads + tid], colp + d * ld);
      ra[q] = __ldg(assign + d);
      ro[q] = __ldg(own + d);
    }
    cp_async_commit();
  }
  for (int32_t m = 0; m < M; m += P) {
#pragma unroll
    for (int q = 0; q < P; ++q) {
      cp_async_wait<P - 1>();                      // row m + q has landed
      const int32_t a = ra[q], o = ro[q];
      const int32_t i = m + q;
      if (i < M && a >= 0 && a < k) {
        const uint4 x = stage[q * kStreamThreads + tid];
        const uint32_t off = (uint32_t)(rl + 128 * i);
        // the thread's first HALF keys sit in the row's first 128 bytes, the
        // others in the second: 8 threads' 16-byte loads cover 32 banks
        K* lo_p = acc + a * COLS + HALF * cg;
        K* hi_p = lo_p + COLS / 2;
        K key[VPL];
        if constexpr (sizeof(T) == 2) {
          const uint32_t crow = ((uint32_t)(32768 - o) << 16) | off;
          const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            key[2 * h] = (w4[h] << 16) + crow;
            key[2 * h + 1] = (w4[h] & 0xffff0000u) + crow;
          }
        } else {
          const int32_t w4[4] = {(int32_t)x.x, (int32_t)x.y, (int32_t)x.z, (int32_t)x.w};
#pragma unroll
          for (int h = 0; h < 4; ++h)
            key[h] = ((K)(uint32_t)((int64_t)w4[h] - o + 2147483648LL) << 32) | off;
        }
        const uint4 lo = *reinterpret_cast<const uint4*>(lo_p);
        const uint4 hi = *reinterpret_cast<const uint4*>(hi_p);
        const K* cl = reinterpret_cast<const K*>(&lo);
        const K* ch = reinterpret_cast<const K*>(&hi);
#pragma unroll
        for (int h = 0; h < HALF; ++h) {
          if (key[h] < cl[h]) atomicMin(lo_p + h, key[h]);
          if (key[HALF + h] < ch[h]) atomicMin(hi_p + h, key[HALF + h]);
        }
      }
      // stage q now takes row i + P
      const int32_t nx = i + P;
      ra[q] = -1;
      if (nx < M) {
        const int64_t d = R0 + rl + 128 * (int64_t)nx;
        cp_async16(&stage[q * kStreamThreads + tid], colp + d * ld);
        ra[q] = __ldg(assign + d);
        ro[q] = __ldg(own + d);
      }
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
  release_successor();
  __syncthreads();
  K* out = part + (int64_t)r * k * k;
  for (int i = tid; i < k * COLS; i += kStreamThreads) {
    const int u = i / COLS, pc = i % COLS;   // pc: key slot in the row; its column:
    const int hh = pc / (COLS / 2), rest = pc % (COLS / 2);
    const int col = (rest / HALF) * VPL + hh * HALF + rest % HALF;
    if (col < w) out[(int64_t)u * k + c0 + col] = acc[i];
  }
}

template <typename K, typename T>
__global__ void __launch_bounds__(kThreads) bt_merge_ranges(const K* __restrict__ part,
                                                            int nranges, int32_t n, int32_t k,
                                                            int32_t* tc, int32_t* td) {
  wait_predecessor();   // the partial tables come from bt_scan_stream
  const int64_t kk = (int64_t)k * k;
  const K none = ~(K)0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < kk;
       i += (int64_t)gridDim.x * kThreads) {
    K best = none;
    int br = -1;
    for (int r = 0; r < nranges; ++r) {
      const K key = part[r * kk + i];
      if (key != none &&
          (br < 0 || StreamKey<T>::cost(key) < StreamKey<T>::cost(best))) { best = key; br = r; }
    }
    const int32_t u = (int32_t)(i / k), v = (int32_t)(i % k);
    if (br < 0 || u == v) {
      tc[i] = kTInf;
      td[i] = -1;
    } else {
      tc[i] = StreamKey<T>::cost(best);
      td[i] = (int32_t)((int64_t)br * n / nranges + StreamKey<T>::offset(best));
    }
  }
}

template <typename T>
static cudaError_t stream_run(const T* cm, int64_t ld, int32_t n, int32_t k, const int32_t* assign,
                              int32_t* tc, int32_t* td, const BtWorkspace& W, int nranges,
                              cudaStream_t st, int num_sms) {
  using K = typename StreamKey<T>::K;
  static std::atomic<uint64_t> attr_set{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!(attr_set.load() & (1ull << dev))) {
    e = cudaFuncSetAttribute(bt_scan_stream<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stream_smem_bytes(kStreamMaxK));
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(1ull << dev);
  }
  const int nslice = (k + StreamKey<T>::kCols - 1) / StreamKey<T>::kCols;
  K* part = reinterpret_cast<K*>(W.part);
  bt_own<T><<<num_sms * 4, kThreads, 0, st>>>(assign, n, k, cm, ld, W.perm);
  // the next two kernels may launch before their predecessor ends; each waits
  // for it (wait_predecessor) before reading its results
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = pdl;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(nslice * nranges);
  cfg.blockDim = dim3(kStreamThreads);
  cfg.dynamicSmemBytes = stream_smem_bytes(k);
  e = cudaLaunchKernelEx(&cfg, bt_scan_stream<T>, cm, ld, n, k, assign, (const int32_t*)W.perm,
                         nslice, nranges, part);
  if (e != cudaSuccess) return e;
  cfg.gridDim = dim3(num_sms * 4);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  e = cudaLaunchKernelEx(&cfg, bt_merge_ranges<K, T>, (const K*)part, nranges, n, k, tc, td);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int bt_max_k(int elem_bytes) { return kThreads * (16 / elem_bytes); }

// Sets the bulk scan's dynamic shared memory limit once per device.
template <typename T>
static cudaError_t bulk_attr() {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!(done.load() & (1ull << dev))) {
    e = cudaFuncSetAttribute(bt_scan_bulk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bulk_smem_max());
    if (e != cudaSuccess) return e;
    done.fetch_or(1ull << dev);
  }
  return cudaSuccess;
}

template <typename T>
static cudaError_t scan_launch(const T* cm, int64_t ld, int32_t n, int32_t k, const BtWorkspace& W,
                               cudaStream_t st, int num_sms) {
  const BulkShape p = bulk_shape(k, (int)sizeof(T));
  if (p.row_bytes >= kBulkMinRowBytes) {
    const cudaError_t e = bulk_attr<T>();
    if (e != cudaSuccess) return e;
    bt_scan_bulk<T><<<num_sms, kBulkThreads, bulk_smem_bytes(p, k), st>>>(cm, ld, k, W.perm, W.cnt,
                                                                           W.t64, W.ctl, p);
  } else {
    bt_scan_rows<T><<<num_sms, kThreads, 0, st>>>(cm, ld, n, k, W.perm, W.items, W.t64, W.ctl);
  }
  return cudaSuccess;
}

// Returns a cudaError_t (cudaSuccess on success); argument checks are done
// by the caller.
cudaError_t best_transfer_run(int32_t n, int32_t k, const void* cm, int elem_bytes, int64_t ld,
                              const int32_t* assign, int32_t* tc, int32_t* td, void* ws,
                              cudaStream_t st, int num_sms) {
  void* base = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
  const BtWorkspace W = carve(base, n, k);
  const int nranges = stream_ranges(n, k, elem_bytes, num_sms);
  if (nranges > 0)
    return elem_bytes == 2
               ? stream_run(static_cast<const int16_t*>(cm), ld, n, k, assign, tc, td, W, nranges,
                            st, num_sms)
               : stream_run(static_cast<const int32_t*>(cm), ld, n, k, assign, tc, td, W, nranges,
                            st, num_sms);
  cudaError_t e = cudaMemsetAsync(W.ctl, 0, 4 * BT_CTL_WORDS + 4ull * (k + 1), st);
  if (e != cudaSuccess) return e;
  bt_count<<<kTiles, kTileThreads, 4 * (size_t)k, st>>>(assign, n, k, W.cnt, W.tile_rel);
  bt_plan<<<1, kThreads, 0, st>>>(W.cnt, k, num_sms, W.items, W.ctl);
  bt_place<<<kTiles, kTileThreads, 4 * (size_t)k, st>>>(assign, n, k, W.cnt, W.tile_rel, W.perm);
  bt_sort_items<<<num_sms * 4, kThreads, 0, st>>>(W.items, W.ctl, W.perm, k, W.t64);
  e = elem_bytes == 2
          ? scan_launch(static_cast<const int16_t*>(cm), ld, n, k, W, st, num_sms)
          : scan_launch(static_cast<const int32_t*>(cm), ld, n, k, W, st, num_sms);
  if (e != cudaSuccess) return e;
  bt_unpack<<<num_sms * 4, kThreads, 0, st>>>(W.t64, k, tc, td, W.ctl);
  return cudaGetLastError();
}

}  // namespace lbdd
