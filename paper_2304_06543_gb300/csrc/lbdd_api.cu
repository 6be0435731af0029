// Host side of the C ABI declared in include/lbdd.h.
//
// Owns device memory, validates inputs, picks launch shapes and launches the
// kernels of asral_solver.cu and best_transfer.cu.  No solver arithmetic runs
// on the host: every step of ASRAL executes in the CUDA kernels.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "lbdd_internal.h"

using namespace lbdd;

static char g_cuda_err[256] = "no error";
static std::mutex g_err_mu;

int lbdd::cuda_fail(cudaError_t e, const char* what) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  // the failure is reported here: clear the thread's last-error state, so that
  // the launch check of a later call does not report it a second time
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LBDD_ERR_OOM : LBDD_ERR_CUDA;
}

#define CK(call) LBDD_CK(call)

// Device memory of a solver comes from the stream-ordered pool on the
// solver's stream: allocating and freeing never waits for kernels running on
// other streams (a server admits and retires requests while others solve).
static int dev_alloc(lbdd_solver* s, void** p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 16);
  cudaError_t e = cudaMallocAsync(p, bytes, s->st);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMallocAsync");
  }
  s->allocs.push_back(*p);
  s->sizes.push_back(bytes);
  s->bytes += bytes;
  return LBDD_OK;
}

template <typename P>
static int dalloc(lbdd_solver* s, P** p, size_t count) {
  void* v = nullptr;
  int rc = dev_alloc(s, &v, count * sizeof(P));
  *p = static_cast<P*>(v);
  return rc;
}

static void dev_free(lbdd_solver* s, void* p) {
  for (size_t i = 0; i < s->allocs.size(); ++i) {
    if (s->allocs[i] == p) {
      cudaFreeAsync(p, s->st);
      s->bytes -= s->sizes[i];
      s->allocs.erase(s->allocs.begin() + i);
      s->sizes.erase(s->sizes.begin() + i);
      return;
    }
  }
}

static void free_all(lbdd_solver* s) {
  for (void* p : s->allocs) cudaFreeAsync(p, s->st);
  cudaStreamSynchronize(s->st);
  s->allocs.clear();
  s->sizes.clear();
  s->bytes = 0;
}

int lbdd::check_device(int* dev, int* sms) {
  CK(cudaGetDevice(dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, *dev));
  if (prop.major != 10 || prop.minor != 3) return LBDD_ERR_NODEV;
  *sms = prop.multiProcessorCount;
  return LBDD_OK;
}

// ------------------------------------------------------------ CM ingest ---

__global__ void cm_minmax(const void* cm, int elem, int64_t ld, int32_t n, int32_t k,
                          int* out_min, int* out_max) {
  int mn = INT32_MAX, mx = INT32_MIN;
  const int64_t total = (int64_t)n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = i / k, c = i - d * k;
    const int v = elem == 2 ? (int)static_cast<const int16_t*>(cm)[d * ld + c]
                            : static_cast<const int32_t*>(cm)[d * ld + c];
    mn = min(mn, v);
    mx = max(mx, v);
  }
  for (int off = 16; off > 0; off >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out_min, mn);
    atomicMax(out_max, mx);
  }
}

__global__ void cm_narrow(const int32_t* src, int64_t lds, int16_t* dst, int64_t ldd, int32_t n,
                          int32_t k) {
  const int64_t total = (int64_t)n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = i / k, c = i - d * k;
    dst[d * ldd + c] = (int16_t)src[d * lds + c];
  }
}

extern "C" int64_t lbdd_cm_pitch(int32_t k, int cm_dtype) {
  const int vpl = cm_dtype == LBDD_CM_I16 ? 8 : 4;
  return ((int64_t)k + vpl - 1) / vpl * vpl;
}

// Copy CM into padded device storage; returns storage, pitch and element size.
static int ingest_cm(lbdd_solver* s, const void* cm, int dtype, int is_device, int64_t src_ld) {
  const int32_t n = s->n, k = s->k;
  const int in_elem = dtype == LBDD_CM_I16 ? 2 : 4;
  const int64_t ld = lbdd_cm_pitch(k, dtype);
  const size_t bytes = ((size_t)n * ld + kColPad) * in_elem;
  void* store = nullptr;
  int rc = dev_alloc(s, &store, bytes);
  if (rc) return rc;
  CK(cudaMemsetAsync(store, 0, bytes, s->st));
  CK(cudaMemcpy2DAsync(store, ld * in_elem, cm, (size_t)src_ld * in_elem, (size_t)k * in_elem, n,
                       is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
  int* mm = nullptr;
  rc = dalloc(s, &mm, 2);
  if (rc) return rc;
  int init[2] = {INT32_MAX, INT32_MIN};
  CK(cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s->st));
  cm_minmax<<<s->num_sms * 4, 256, 0, s->st>>>(store, in_elem, ld, n, k, mm, mm + 1);
  CK(cudaGetLastError());
  int res[2];
  CK(cudaMemcpyAsync(res, mm, sizeof(res), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (res[0] < 1) return LBDD_ERR_ARG;   // CM entries are positive integers
  s->cm = store;
  s->ld = ld;
  s->elem = in_elem;
  if (in_elem == 4 && res[1] <= INT16_MAX) {
    const int64_t ld16 = lbdd_cm_pitch(k, LBDD_CM_I16);
    void* narrow = nullptr;
    rc = dev_alloc(s, &narrow, ((size_t)n * ld16 + kColPad) * 2);
    if (rc) return rc;
    CK(cudaMemsetAsync(narrow, 0, ((size_t)n * ld16 + kColPad) * 2, s->st));
    cm_narrow<<<s->num_sms * 8, 256, 0, s->st>>>(static_cast<const int32_t*>(store), ld,
                                                 static_cast<int16_t*>(narrow), ld16, n, k);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->st));
    // release the wide copy
    dev_free(s, store);
    s->cm = narrow;
    s->ld = ld16;
    s->elem = 2;
  }
  return LBDD_OK;
}

// --------------------------------------------------------------- create ---

static int pick_cluster(const lbdd_solver* s) {
  if (s->cluster > 0) return s->cluster;
  // about 32 owned columns per CTA: relaxation work and the exchange per
  // Bellman-Ford sweep stay small; powers of two split the columns evenly
  int C = (s->k + 31) / 32;
  C = std::min(16, std::max(1, C));
  int p = 1;
  while (p < C) p <<= 1;
  return std::min(16, p);
}

// Dynamic shared memory for a launch: with the owned cost slice when it fits.
size_t lbdd::launch_smem(int32_t k, int C, int elem) {
  const size_t full = solver_smem_bytes(k, C, elem, true);
  return full <= kMaxSmem ? full : solver_smem_bytes(k, C, elem, false);
}

bool lbdd::fits_k(int32_t k, int elem, int C) {
  const size_t smem = launch_smem(k, C, elem);
  if (smem > kMaxSmem) return false;
  const int32_t w = (k + C - 1) / C;
  if (w > solver_max_k(1, elem)) return false;
  if (solver_max_clusters(C, elem, smem) >= 1) return true;
  // a refused attribute or occupancy query only means "does not fit": clear
  // the error it left, which a later launch check would otherwise report
  (void)cudaGetLastError();
  return false;
}

// Largest k whose 16-CTA launch fits kMaxSmem for both stored CM widths
// (the replicas and the frontier grow with k; the cost slice then lives in
// global memory).  Host arithmetic only.
extern "C" int32_t lbdd_max_centers(void) {
  int32_t best = 65535;
  for (int elem = 2; elem <= 4; elem += 2) {
    int32_t lo = 1, hi = 65535;    // launch_smem(lo) fits; find the last k that does
    if (launch_smem(lo, 16, elem) > kMaxSmem) return 0;
    while (lo < hi) {
      const int32_t mid = lo + (hi - lo + 1) / 2;
      if (launch_smem(mid, 16, elem) <= kMaxSmem) lo = mid;
      else hi = mid - 1;
    }
    best = std::min(best, lo);
  }
  return best;
}

static int fits(const lbdd_solver* s, int C) { return fits_k(s->k, s->elem, C) ? 1 : 0; }

size_t lbdd::solver_footprint(int32_t n, int32_t k, int in_elem, int elem) {
  auto a = [](size_t b) { return (std::max<size_t>(b, 16) + 511) / 512 * 512; };
  const int dt_in = in_elem == 2 ? LBDD_CM_I16 : LBDD_CM_I32;
  const int dt = elem == 2 ? LBDD_CM_I16 : LBDD_CM_I32;
  size_t cm = a(((size_t)n * lbdd_cm_pitch(k, dt_in) + kColPad) * in_elem);
  if (elem != in_elem) cm += a(((size_t)n * lbdd_cm_pitch(k, dt) + kColPad) * elem);
  const size_t max_pages = ((size_t)n + kPage - 1) / kPage;
  const size_t npages = max_pages + k;
  size_t b = cm + a(8);                       // CM copies + min/max scratch
  b += 2 * a(4ull * k);                       // cap, pen
  b += 2 * a(4ull * n) + a(12ull * n);        // smin, order, sort_tmp
  b += 2 * a(4ull * n);                       // assign, pos
  b += 2 * a(4ull * k);                       // load, seg_size
  b += a(4ull * k * max_pages) + a(4ull * npages * kPageWords) + a(4ull * npages);
  b += 2 * a(4ull * k * k);                   // tc, td
  b += a(8ull * CTL_COUNT) + a(16) + a(sizeof(DevInst));
  return b;
}

static int create_impl(lbdd_solver** out, int32_t n, int32_t k, const void* cm, int cm_dtype,
                       int cm_is_device, int64_t cm_ld, const int32_t* cap, const int32_t* pen,
                       void* cuda_stream) {
  if (!out) return LBDD_ERR_ARG;
  *out = nullptr;
  if (n < 1 || k < 1 || !cm || !cap || !pen) return LBDD_ERR_ARG;
  if (k > 65535) return LBDD_ERR_ARG;   // Bellman-Ford packs node ids in 16 bits
  if (k > lbdd_max_centers()) return LBDD_ERR_ARG;   // the cluster's shared memory
  if (cm_dtype != LBDD_CM_I32 && cm_dtype != LBDD_CM_I16) return LBDD_ERR_ARG;
  for (int32_t i = 0; i < k; ++i)
    if (cap[i] < 1 || pen[i] < 1) return LBDD_ERR_ARG;
  lbdd_solver* s = new (std::nothrow) lbdd_solver();
  if (!s) return LBDD_ERR_OOM;
  s->n = n;
  s->n_cap = n;
  s->k = k;
  s->st = static_cast<cudaStream_t>(cuda_stream);
  int rc = check_device(&s->device, &s->num_sms);
  if (rc) { delete s; return rc; }
  rc = ingest_cm(s, cm, cm_dtype, cm_is_device, cm_ld);
  if (rc) { free_all(s); delete s; return rc; }
  if (launch_smem(k, 16, s->elem) > kMaxSmem) { free_all(s); delete s; return LBDD_ERR_ARG; }
  const int32_t max_pages = (int32_t)(((int64_t)n + kPage - 1) / kPage);
  const int32_t npages = max_pages + k;
  if (!rc) rc = dalloc(s, &s->cap, k);
  if (!rc) rc = dalloc(s, &s->pen, k);
  if (!rc) rc = dalloc(s, &s->smin, n);
  if (!rc) rc = dalloc(s, &s->order, n);
  if (!rc) rc = dalloc(s, &s->sort_tmp, 3ull * n);
  if (!rc) rc = dalloc(s, &s->assign, n);
  if (!rc) rc = dalloc(s, &s->pos, n);
  if (!rc) rc = dalloc(s, &s->load, k);
  if (!rc) rc = dalloc(s, &s->seg_size, k);
  if (!rc) rc = dalloc(s, &s->page_tab, (size_t)k * max_pages);
  if (!rc) rc = dalloc(s, &s->pool, (size_t)npages * kPageWords);
  if (!rc) rc = dalloc(s, &s->free_stack, npages);
  if (!rc) rc = dalloc(s, &s->tc, (size_t)k * k);
  if (!rc) rc = dalloc(s, &s->td, (size_t)k * k);
  if (!rc) rc = dalloc(s, &s->ctl, CTL_COUNT);
  if (!rc) rc = dalloc(s, &s->counter, 4);
  if (!rc) rc = dalloc(s, &s->d_inst, 1);
  if (rc) { free_all(s); delete s; return rc; }
  DevInst& I = s->h_inst;
  I.cm = s->cm; I.ld = s->ld; I.n = n; I.k = k; I.cap = s->cap; I.pen = s->pen; I.Q = 1;
  I.smin = s->smin; I.order = s->order; I.sort_tmp = s->sort_tmp; I.assign = s->assign;
  I.pos = s->pos; I.load = s->load; I.seg_size = s->seg_size; I.page_tab = s->page_tab;
  I.pool = s->pool; I.free_stack = s->free_stack; I.tc = s->tc; I.td = s->td; I.ctl = s->ctl;
  I.max_pages = max_pages; I.npages = npages;
  auto fail = [&](cudaError_t e, const char* w) { int r = cuda_fail(e, w); free_all(s); delete s; return r; };
  cudaError_t e;
  if ((e = cudaMemcpyAsync(s->cap, cap, 4ull * k, cudaMemcpyHostToDevice, s->st))) return fail(e, "cap");
  if ((e = cudaMemcpyAsync(s->pen, pen, 4ull * k, cudaMemcpyHostToDevice, s->st))) return fail(e, "pen");
  if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(int64_t) * CTL_COUNT, s->st))) return fail(e, "ctl");
  if ((e = cudaMemsetAsync(s->assign, 0xff, 4ull * n, s->st))) return fail(e, "assign");
  if ((e = cudaMemsetAsync(s->load, 0, 4ull * k, s->st))) return fail(e, "load");
  // defined contents everywhere, so that a corrupt index can never leave the pool
  if ((e = cudaMemsetAsync(s->page_tab, 0, 4ull * k * max_pages, s->st))) return fail(e, "pages");
  if ((e = cudaMemsetAsync(s->pool, 0, 4ull * npages * kPageWords, s->st))) return fail(e, "pool");
  if ((e = cudaMemsetAsync(s->pos, 0, 4ull * n, s->st))) return fail(e, "pos");
  if ((e = cudaMemcpyAsync(s->d_inst, &I, sizeof(DevInst), cudaMemcpyHostToDevice, s->st))) return fail(e, "inst");
  if ((e = cudaStreamSynchronize(s->st))) return fail(e, "sync");
  *out = s;
  return LBDD_OK;
}

extern "C" int lbdd_create(lbdd_solver** out, int32_t n, int32_t k, const void* cm, int cm_dtype,
                           int cm_is_device, const int32_t* cap, const int32_t* pen,
                           void* cuda_stream) {
  return create_impl(out, n, k, cm, cm_dtype, cm_is_device, k, cap, pen, cuda_stream);
}

// Extended cost matrix of Alg. 5: the caller's n x k costs widened to int32,
// plus (when K > k) a dummy center whose cost is max + 1 for every unit.
__global__ void strict_extend(const void* cm, int elem, int32_t n, int32_t k, int32_t K,
                              int32_t fill, int32_t* out) {
  const int64_t total = (int64_t)n * K;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = i / K, c = i - d * K;
    out[i] = c < k ? (elem == 2 ? (int32_t)static_cast<const int16_t*>(cm)[d * k + c]
                                : static_cast<const int32_t*>(cm)[d * k + c])
                   : fill;
  }
}

extern "C" int lbdd_create_strict(lbdd_solver** out, int32_t n, int32_t k, const void* cm,
                                  int cm_dtype, int cm_is_device, const int32_t* cap,
                                  void* cuda_stream) {
  if (!out) return LBDD_ERR_ARG;
  *out = nullptr;
  if (n < 1 || k < 1 || k > 65534 || !cm || !cap) return LBDD_ERR_ARG;
  if (cm_dtype != LBDD_CM_I32 && cm_dtype != LBDD_CM_I16) return LBDD_ERR_ARG;
  int64_t capsum = 0;
  for (int32_t i = 0; i < k; ++i) {
    if (cap[i] < 1) return LBDD_ERR_ARG;
    capsum += cap[i];
  }
  const int32_t K = capsum < n ? k + 1 : k;
  if (K > lbdd_max_centers()) return LBDD_ERR_ARG;   // with the dummy center, if any
  int dev = 0, sms = 0;
  int rc = check_device(&dev, &sms);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int elem = cm_dtype == LBDD_CM_I16 ? 2 : 4;
  const size_t in_bytes = (size_t)n * k * elem;
  void* src = nullptr;
  int32_t* ext = nullptr;
  int* mm = nullptr;
  auto cleanup = [&]() {
    if (src && !cm_is_device) cudaFreeAsync(src, st);
    if (ext) cudaFreeAsync(ext, st);
    if (mm) cudaFreeAsync(mm, st);
    cudaStreamSynchronize(st);
  };
  cudaError_t e = cudaSuccess;
  if (cm_is_device) {
    src = const_cast<void*>(cm);
  } else {
    e = cudaMallocAsync(&src, in_bytes, st);
    if (!e) e = cudaMemcpyAsync(src, cm, in_bytes, cudaMemcpyHostToDevice, st);
  }
  if (!e) e = cudaMallocAsync(reinterpret_cast<void**>(&ext), 4ull * n * K, st);
  if (!e) e = cudaMallocAsync(reinterpret_cast<void**>(&mm), 2 * sizeof(int), st);
  int res[2] = {INT32_MAX, INT32_MIN};
  if (!e) e = cudaMemcpyAsync(mm, res, sizeof(res), cudaMemcpyHostToDevice, st);
  if (!e) {
    cm_minmax<<<sms * 4, 256, 0, st>>>(src, elem, k, n, k, mm, mm + 1);
    e = cudaGetLastError();
  }
  if (!e) e = cudaMemcpyAsync(res, mm, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) { rc = cuda_fail(e, "lbdd_create_strict"); cleanup(); return rc; }
  if (res[0] < 1 || res[1] == INT32_MAX) { cleanup(); return LBDD_ERR_ARG; }
  strict_extend<<<sms * 8, 256, 0, st>>>(src, elem, n, k, K, res[1] + 1, ext);
  e = cudaGetLastError();
  if (e) { rc = cuda_fail(e, "strict_extend"); cleanup(); return rc; }
  std::vector<int32_t> capx(cap, cap + k), penx(K, 1);
  if (K > k) capx.push_back((int32_t)(n - capsum));
  lbdd_solver* s = nullptr;
  rc = create_impl(&s, n, K, ext, LBDD_CM_I32, 1, K, capx.data(), penx.data(), cuda_stream);
  cleanup();
  if (rc) return rc;
  s->strict = 1;
  *out = s;
  return LBDD_OK;
}

int lbdd::clone_solver(const lbdd_solver* src, lbdd_solver** out) {
  const int32_t Q = src->h_inst.Q;
  std::vector<int32_t> cap(src->k), q((size_t)src->k * Q), pen(src->k);
  CK(cudaMemcpyAsync(cap.data(), src->cap, 4ull * src->k, cudaMemcpyDeviceToHost, src->st));
  CK(cudaMemcpyAsync(q.data(), src->h_inst.pen, 4ull * src->k * Q, cudaMemcpyDeviceToHost,
                     src->st));
  CK(cudaStreamSynchronize(src->st));
  for (int32_t c = 0; c < src->k; ++c) pen[c] = q[(size_t)c * Q];
  int rc = create_impl(out, src->n, src->k, src->cm, src->elem == 2 ? LBDD_CM_I16 : LBDD_CM_I32,
                       1, src->ld, cap.data(), pen.data(), src->st);
  if (rc == LBDD_OK && Q > 1) rc = lbdd_set_penalty_table(*out, q.data(), Q);
  if (rc == LBDD_OK) { (*out)->strict = src->strict; }
  return rc;
}

int lbdd::clone_prefix(const lbdd_solver* src, int32_t n_sub, lbdd_solver** out) {
  if (!src || !out || n_sub < 1) return LBDD_ERR_ARG;
  n_sub = std::min(n_sub, src->n);
  const int32_t Q = src->h_inst.Q;
  std::vector<int32_t> cap(src->k), q((size_t)src->k * Q), pen(src->k);
  CK(cudaMemcpyAsync(cap.data(), src->cap, 4ull * src->k, cudaMemcpyDeviceToHost, src->st));
  CK(cudaMemcpyAsync(q.data(), src->h_inst.pen, 4ull * src->k * Q, cudaMemcpyDeviceToHost,
                     src->st));
  CK(cudaStreamSynchronize(src->st));
  for (int32_t c = 0; c < src->k; ++c) {
    pen[c] = q[(size_t)c * Q];
    cap[c] = std::max<int32_t>(1, (int32_t)((int64_t)cap[c] * n_sub / src->n));
  }
  int rc = create_impl(out, n_sub, src->k, src->cm, src->elem == 2 ? LBDD_CM_I16 : LBDD_CM_I32,
                       1, src->ld, cap.data(), pen.data(), src->st);
  if (rc == LBDD_OK && Q > 1) rc = lbdd_set_penalty_table(*out, q.data(), Q);
  return rc;
}

extern "C" int lbdd_set_penalty_table(lbdd_solver* s, const int32_t* qtab, int32_t Q) {
  if (!s || !qtab || Q < 1 || s->strict) return LBDD_ERR_ARG;
  for (int32_t c = 0; c < s->k; ++c)
    for (int32_t j = 0; j < Q; ++j) {
      const int32_t v = qtab[(size_t)c * Q + j];
      if (v < 1 || (j > 0 && v < qtab[(size_t)c * Q + j - 1])) return LBDD_ERR_ARG;
    }
  int64_t rounds = 0;
  CK(cudaMemcpyAsync(&rounds, s->ctl + CTL_PROLOGUE, sizeof(int64_t), cudaMemcpyDeviceToHost,
                     s->st));
  CK(cudaStreamSynchronize(s->st));
  if (rounds != 0) return LBDD_ERR_STATE;   // only before the first round (or after a reset)
  int32_t* table = nullptr;
  int rc = dalloc(s, &table, (size_t)s->k * Q);
  if (rc) return rc;
  CK(cudaMemcpyAsync(table, qtab, 4ull * s->k * Q, cudaMemcpyHostToDevice, s->st));
  s->h_inst.pen = table;
  s->h_inst.Q = Q;
  CK(cudaMemcpyAsync(s->d_inst, &s->h_inst, sizeof(DevInst), cudaMemcpyHostToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return LBDD_OK;
}

extern "C" int lbdd_set_option(lbdd_solver* s, int option, int64_t value) {
  if (!s) return LBDD_ERR_ARG;
  switch (option) {
    case LBDD_OPT_CLUSTER:
      // powers of two: the sizes the batch plans use and the tests cover
      if (value < 0 || value > 16 || (value & (value - 1)) != 0) return LBDD_ERR_ARG;
      if (value > 0 && !fits(s, (int)value)) return LBDD_ERR_ARG;
      s->cluster = (int)value;
      return LBDD_OK;
    case LBDD_OPT_NCYC_SKIP:
      if (value != 0 && value != 1) return LBDD_ERR_ARG;
      s->ncyc_skip = (int)value;
      return LBDD_OK;
    case LBDD_OPT_TC_SMEM:
      if (value != 0 && value != 1) return LBDD_ERR_ARG;
      s->tc_smem = (int)value;
      return LBDD_OK;
    case LBDD_OPT_NPATH_REUSE:
      if (value != 0 && value != 1) return LBDD_ERR_ARG;
      s->npath_reuse = (int)value;
      return LBDD_OK;
    case LBDD_OPT_PHASE_TIMERS:
      if (value != 0 && value != 1) return LBDD_ERR_ARG;
      s->phase_timers = (int)value;
      return LBDD_OK;
    default:
      return LBDD_ERR_ARG;
  }
}

// ---------------------------------------------------------------- solve ---

int lbdd::status_to_rc(int64_t st) {
  if (st == 0) return LBDD_OK;
  if (st == ST_ERR_INVARIANT) return LBDD_ERR_INVARIANT;
  if (st == ST_ERR_TIMEOUT) return LBDD_ERR_TIMEOUT;
  return LBDD_ERR_STATE;
}

static int set_target(lbdd_solver* s, int64_t max_rounds, cudaStream_t st) {
  int64_t h[2];
  CK(cudaMemcpyAsync(h, s->ctl + CTL_ROUNDS, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h + 1, s->ctl + CTL_STATUS, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h[1] != 0) return LBDD_ERR_STATE;
  const int64_t target = max_rounds < 0 ? (int64_t)s->n : std::min<int64_t>(s->n, h[0] + max_rounds);
  CK(cudaMemcpyAsync(s->ctl + CTL_TARGET, &target, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return LBDD_OK;
}

int lbdd::solver_flags(const lbdd_solver* s) {
  return (s->ncyc_skip ? 0 : OPT_NO_NCYC_SKIP) | (s->npath_reuse ? 0 : OPT_NO_NPATH_REUSE) |
         (s->tc_smem ? 0 : OPT_NO_TC_SMEM) | (s->phase_timers ? OPT_PHASE_TIMERS : 0) |
         (s->strict ? OPT_STRICT : 0);
}

int lbdd::choose_cluster(lbdd_solver* s) {
  int C = pick_cluster(s);
  while (C > 1 && !fits(s, C)) C >>= 1;
  return fits(s, C) ? C : 0;
}

extern "C" int lbdd_solve(lbdd_solver* s, int64_t max_rounds) {
  if (!s) return LBDD_ERR_ARG;
  int rc = set_target(s, max_rounds, s->st);
  if (rc) return rc;
  const int C = choose_cluster(s);
  if (C < 1) return LBDD_ERR_ARG;
  const size_t smem = launch_smem(s->k, C, s->elem);
  CK(cudaMemsetAsync(s->counter, 0, sizeof(int32_t), s->st));
  CK(launch_solver(s->d_inst, 1, s->counter, C, 1, s->elem, smem, solver_flags(s), s->st));
  int64_t st = 0;
  CK(cudaMemcpyAsync(&st, s->ctl + CTL_STATUS, sizeof(int64_t), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return status_to_rc(st);
}

int lbdd::solve_timed(lbdd_solver* s, int64_t max_rounds, int C, float* ms) {
  int rc = set_target(s, max_rounds, s->st);
  if (rc) return rc;
  if (C < 1 || !fits(s, C)) return LBDD_ERR_ARG;
  const size_t smem = launch_smem(s->k, C, s->elem);
  struct Events {   // destroyed on every return path
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  CK(cudaEventCreate(&ev.a));
  CK(cudaEventCreate(&ev.b));
  CK(cudaMemsetAsync(s->counter, 0, sizeof(int32_t), s->st));
  CK(prepare_solver(C, s->elem, smem));
  CK(cudaEventRecord(ev.a, s->st));
  CK(launch_solver(s->d_inst, 1, s->counter, C, 1, s->elem, smem, solver_flags(s), s->st, 0,
                   false));
  CK(cudaEventRecord(ev.b, s->st));
  int64_t st = 0;
  CK(cudaMemcpyAsync(&st, s->ctl + CTL_STATUS, sizeof(int64_t), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  CK(cudaEventElapsedTime(ms, ev.a, ev.b));
  return status_to_rc(st);
}

// ----------------------------------------------------------- insertion ---

// The unit appended as row d (the dynamic update of the paper's proof sketch:
// adding a demand unit is one more iteration of the loop of Alg. 2): its
// costs into the CM row (narrowed when the CM is stored as int16; the caller
// checked the range), its most suitable center (lowest index among the
// minima), its round at the end of the extraction order, not yet allotted.
__global__ void insert_unit(void* cm, int elem, int64_t ld, int32_t d, int32_t k,
                            const int32_t* __restrict__ row, int32_t* smin, int32_t* order,
                            int32_t* assign, int32_t* pos) {
  __shared__ int2 part[32];
  int32_t bv = INT32_MAX, bj = INT32_MAX;
  for (int32_t c = threadIdx.x; c < k; c += blockDim.x) {
    const int32_t v = row[c];
    if (elem == 2) static_cast<int16_t*>(cm)[(int64_t)d * ld + c] = (int16_t)v;
    else static_cast<int32_t*>(cm)[(int64_t)d * ld + c] = v;
    if (v < bv) { bv = v; bj = c; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const int32_t ov = __shfl_xor_sync(0xffffffffu, bv, off);
    const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, off);
    if (ov < bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
  }
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = make_int2(bv, bj);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (part[w].x < bv || (part[w].x == bv && part[w].y < bj)) { bv = part[w].x; bj = part[w].y; }
    smin[d] = bj;
    order[d] = d;
    assign[d] = -1;
    pos[d] = 0;
  }
}

// Room for cap_new units: the unit-indexed arrays, the CM rows and the
// member-list page table and pool are reallocated with their contents; the
// new pages join the free stack (if no round has run, the prologue builds
// the stack from all pages anyway).
static int grow_units(lbdd_solver* s, int32_t cap_new) {
  const int32_t n = s->n, k = s->k;
  const int64_t ld = s->ld;
  const int elem = s->elem;
  DevInst& I = s->h_inst;
  const int32_t mp_old = I.max_pages, np_old = I.npages;
  const int32_t mp_new = (int32_t)(((int64_t)cap_new + kPage - 1) / kPage);
  const int32_t np_new = mp_new + k;
  void* cm = nullptr;
  int32_t *smin = nullptr, *order = nullptr, *sort_tmp = nullptr, *assign = nullptr,
          *pos = nullptr, *page_tab = nullptr, *pool = nullptr, *free_stack = nullptr;
  const size_t cm_bytes = ((size_t)cap_new * ld + kColPad) * elem;
  int rc = dev_alloc(s, &cm, cm_bytes);
  if (!rc) rc = dalloc(s, &smin, cap_new);
  if (!rc) rc = dalloc(s, &order, cap_new);
  if (!rc) rc = dalloc(s, &sort_tmp, 3ull * cap_new);
  if (!rc) rc = dalloc(s, &assign, cap_new);
  if (!rc) rc = dalloc(s, &pos, cap_new);
  if (!rc) rc = dalloc(s, &page_tab, (size_t)k * mp_new);
  if (!rc) rc = dalloc(s, &pool, (size_t)np_new * kPageWords);
  if (!rc) rc = dalloc(s, &free_stack, np_new);
  if (rc) {   // the solver keeps its old arrays
    for (void* p : {cm, (void*)smin, (void*)order, (void*)sort_tmp, (void*)assign, (void*)pos,
                    (void*)page_tab, (void*)pool, (void*)free_stack})
      if (p) dev_free(s, p);
    return rc;
  }
  const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
  CK(cudaMemsetAsync(cm, 0, cm_bytes, s->st));
  CK(cudaMemcpyAsync(cm, s->cm, (size_t)n * ld * elem, dd, s->st));
  CK(cudaMemcpyAsync(smin, s->smin, 4ull * n, dd, s->st));
  CK(cudaMemcpyAsync(order, s->order, 4ull * n, dd, s->st));
  CK(cudaMemsetAsync(assign, 0xff, 4ull * cap_new, s->st));
  CK(cudaMemcpyAsync(assign, s->assign, 4ull * n, dd, s->st));
  CK(cudaMemsetAsync(pos, 0, 4ull * cap_new, s->st));
  CK(cudaMemcpyAsync(pos, s->pos, 4ull * n, dd, s->st));
  CK(cudaMemsetAsync(page_tab, 0, 4ull * k * mp_new, s->st));
  CK(cudaMemcpy2DAsync(page_tab, 4ull * mp_new, s->page_tab, 4ull * mp_old, 4ull * mp_old, k, dd,
                       s->st));
  CK(cudaMemsetAsync(pool, 0, 4ull * np_new * kPageWords, s->st));
  CK(cudaMemcpyAsync(pool, s->pool, 4ull * np_old * kPageWords, dd, s->st));
  CK(cudaMemcpyAsync(free_stack, s->free_stack, 4ull * np_old, dd, s->st));
  int64_t h[2];
  CK(cudaMemcpyAsync(h, s->ctl + CTL_PROLOGUE, sizeof(int64_t), cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(h + 1, s->ctl + CTL_FREE_TOP, sizeof(int64_t), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (h[0] != 0 && np_new > np_old) {
    std::vector<int32_t> ids(np_new - np_old);
    for (int32_t i = 0; i < np_new - np_old; ++i) ids[i] = np_old + i;
    const int64_t top = h[1] + (int64_t)ids.size();
    CK(cudaMemcpyAsync(free_stack + h[1], ids.data(), 4ull * ids.size(), cudaMemcpyHostToDevice,
                       s->st));
    CK(cudaMemcpyAsync(s->ctl + CTL_FREE_TOP, &top, sizeof(int64_t), cudaMemcpyHostToDevice,
                       s->st));
    CK(cudaStreamSynchronize(s->st));
  }
  for (void* p : {s->cm, (void*)s->smin, (void*)s->order, (void*)s->sort_tmp, (void*)s->assign,
                  (void*)s->pos, (void*)s->page_tab, (void*)s->pool, (void*)s->free_stack})
    dev_free(s, p);
  s->cm = cm; s->smin = smin; s->order = order; s->sort_tmp = sort_tmp; s->assign = assign;
  s->pos = pos; s->page_tab = page_tab; s->pool = pool; s->free_stack = free_stack;
  I.cm = cm; I.smin = smin; I.order = order; I.sort_tmp = sort_tmp; I.assign = assign;
  I.pos = pos; I.page_tab = page_tab; I.pool = pool; I.free_stack = free_stack;
  I.max_pages = mp_new;
  I.npages = np_new;
  s->n_cap = cap_new;
  return LBDD_OK;
}

extern "C" int lbdd_insert(lbdd_solver* s, const void* row, int cm_dtype, int32_t* unit_out) {
  if (!s || !row || !unit_out) return LBDD_ERR_ARG;
  if (cm_dtype != LBDD_CM_I32 && cm_dtype != LBDD_CM_I16) return LBDD_ERR_ARG;
  if (s->strict || s->in_batches > 0) return LBDD_ERR_STATE;
  if (s->n >= INT32_MAX - 1) return LBDD_ERR_ARG;
  const int32_t k = s->k;
  std::vector<int32_t> r(k);
  for (int32_t c = 0; c < k; ++c) {
    const int32_t v = cm_dtype == LBDD_CM_I16 ? (int32_t)static_cast<const int16_t*>(row)[c]
                                              : static_cast<const int32_t*>(row)[c];
    if (v < 1 || (s->elem == 2 && v > INT16_MAX)) return LBDD_ERR_ARG;
    r[c] = v;
  }
  int rc = LBDD_OK;
  if (!s->ins_row) rc = dalloc(s, &s->ins_row, k);
  if (rc) return rc;
  if (s->n + 1 > s->n_cap) {
    const int64_t want = (int64_t)s->n_cap + s->n_cap / 2 + 1024;
    rc = grow_units(s, (int32_t)std::min<int64_t>(want, INT32_MAX - 1));
    if (rc) return rc;
  }
  const int32_t d = s->n;
  CK(cudaMemcpyAsync(s->ins_row, r.data(), 4ull * k, cudaMemcpyHostToDevice, s->st));
  insert_unit<<<1, kThreads, 0, s->st>>>(s->cm, s->elem, s->ld, d, k, s->ins_row, s->smin,
                                         s->order, s->assign, s->pos);
  CK(cudaGetLastError());
  s->n = d + 1;
  s->h_inst.n = s->n;
  CK(cudaMemcpyAsync(s->d_inst, &s->h_inst, sizeof(DevInst), cudaMemcpyHostToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  *unit_out = d;
  return LBDD_OK;
}

extern "C" int lbdd_reset(lbdd_solver* s) {
  if (!s) return LBDD_ERR_ARG;
  CK(cudaMemsetAsync(s->ctl, 0, sizeof(int64_t) * CTL_COUNT, s->st));
  CK(cudaMemsetAsync(s->assign, 0xff, 4ull * s->n, s->st));
  CK(cudaMemsetAsync(s->load, 0, 4ull * s->k, s->st));
  return LBDD_OK;
}

// ------------------------------------------------------------ accessors ---

static int read_ctl(const lbdd_solver* s, int idx, int64_t* out) {
  CK(cudaMemcpyAsync(out, s->ctl + idx, sizeof(int64_t), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return LBDD_OK;
}

extern "C" int lbdd_objective(const lbdd_solver* s, int64_t* out) {
  if (!s || !out) return LBDD_ERR_ARG;
  return read_ctl(s, CTL_DELTA, out);
}

extern "C" int lbdd_rounds_done(const lbdd_solver* s, int64_t* out) {
  if (!s || !out) return LBDD_ERR_ARG;
  return read_ctl(s, CTL_ROUNDS, out);
}

extern "C" int lbdd_assignment(const lbdd_solver* s, int32_t* out, int out_is_device) {
  if (!s || !out) return LBDD_ERR_ARG;
  CK(cudaMemcpyAsync(out, s->assign, 4ull * s->n,
                     out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return LBDD_OK;
}

extern "C" int lbdd_loads(const lbdd_solver* s, int32_t* out) {
  if (!s || !out) return LBDD_ERR_ARG;
  CK(cudaMemcpyAsync(out, s->load, 4ull * s->k, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return LBDD_OK;
}

extern "C" int lbdd_get_stats(const lbdd_solver* s, lbdd_stats* out) {
  if (!s || !out) return LBDD_ERR_ARG;
  int64_t c[CTL_COUNT];
  CK(cudaMemcpyAsync(c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  out->rounds = c[CTL_ROUNDS];
  out->cycles_applied = c[CTL_CYCLES];
  out->paths_applied = c[CTL_PATHS];
  out->bf_calls = c[CTL_BF_CALLS];
  out->bf_sweeps = c[CTL_BF_SWEEPS];
  out->bf_max_sweeps = c[CTL_BF_MAX];
  out->moves = c[CTL_MOVES];
  out->ncyc_skipped = c[CTL_NCYC_SKIPPED];
  out->rows_scanned = c[CTL_ROWS_SCANNED];
  out->cm_elem_bytes = s->elem;
  out->prologue_ns = c[CTL_T_PROLOGUE];
  out->rounds_ns = c[CTL_T_TOTAL];
  // phase timers are SM cycles; scale by the measured ns per cycle of the loop
  const double ns_per_cycle = c[CTL_T_CYCLES] > 0 ? (double)c[CTL_T_TOTAL] / c[CTL_T_CYCLES] : 0.0;
  out->merge_ns = (int64_t)(c[CTL_T_MERGE] * ns_per_cycle);
  out->relax_ns = (int64_t)(c[CTL_T_RELAX] * ns_per_cycle);
  out->sync_ns = (int64_t)(c[CTL_T_SYNC] * ns_per_cycle);
  out->gather_ns = (int64_t)(c[CTL_T_GATHER] * ns_per_cycle);
  out->apply_ns = (int64_t)(c[CTL_T_APPLY] * ns_per_cycle);
  out->rescan_ns = (int64_t)(c[CTL_T_RESCAN] * ns_per_cycle);
  out->relax_loop_ns = (int64_t)(c[CTL_T_RLOOP] * ns_per_cycle);
  out->relax_reduce_ns = (int64_t)(c[CTL_T_RRED] * ns_per_cycle);
  out->cost_slice_in_smem = c[CTL_TSM_ON];
  out->npath_reused = c[CTL_NPATH_REUSED];
  out->col_rows = c[CTL_COL_ROWS];
  out->front_sum = c[CTL_FRONT_SUM];
  for (int h = 0; h < 6; ++h) out->front_hist[h] = c[CTL_FRONT_HIST + h];
  out->cluster_size = const_cast<lbdd_solver*>(s)->cluster ? s->cluster
                                                            : choose_cluster(const_cast<lbdd_solver*>(s));
  return LBDD_OK;
}

extern "C" int lbdd_best_transfer_table(const lbdd_solver* s, int32_t* tc, int32_t* td,
                                        int out_is_device) {
  if (!s || !tc || !td) return LBDD_ERR_ARG;
  const cudaMemcpyKind kind = out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(tc, s->tc, 4ull * s->k * s->k, kind, s->st));
  CK(cudaMemcpyAsync(td, s->td, 4ull * s->k * s->k, kind, s->st));
  CK(cudaStreamSynchronize(s->st));
  return LBDD_OK;
}

extern "C" int lbdd_solver_cm(const lbdd_solver* s, const void** cm_dev, int* cm_dtype,
                              int64_t* ld) {
  if (!s || !cm_dev || !cm_dtype || !ld) return LBDD_ERR_ARG;
  *cm_dev = s->cm;
  *cm_dtype = s->elem == 2 ? LBDD_CM_I16 : LBDD_CM_I32;
  *ld = s->ld;
  return LBDD_OK;
}

extern "C" void lbdd_destroy(lbdd_solver* s) {
  if (!s) return;
  cudaStreamSynchronize(s->st);
  free_all(s);
  delete s;
}

extern "C" const char* lbdd_strerror(int code) {
  switch (code) {
    case LBDD_OK: return "ok";
    case LBDD_ERR_ARG: return "invalid argument";
    case LBDD_ERR_OOM: return "out of memory";
    case LBDD_ERR_CUDA: return "CUDA runtime error";
    case LBDD_ERR_TIMEOUT: return "timed out";
    case LBDD_ERR_INVARIANT: return "invariant violated (negative cycle in Gamma)";
    case LBDD_ERR_STATE: return "invalid state";
    case LBDD_ERR_NODEV: return "no compute capability 10.3 device";
    case LBDD_ERR_BUDGET: return "request exceeds the memory budget";
    default: return "unknown status";
  }
}

extern "C" const char* lbdd_last_cuda_error(void) { return g_cuda_err; }

// ----------------------------------------------------- best transfer K2 ---

extern "C" size_t lbdd_best_transfer_workspace(int32_t n, int32_t k) {
  return bt_workspace_bytes(n, k);
}

extern "C" int lbdd_best_transfer(int32_t n, int32_t k, const void* cm_dev, int cm_dtype,
                                  int64_t ld, const int32_t* assign_dev, int32_t* tc_dev,
                                  int32_t* td_dev, void* workspace, size_t workspace_bytes,
                                  void* stream) {
  if (n < 1 || k < 1 || !cm_dev || !assign_dev || !tc_dev || !td_dev || !workspace)
    return LBDD_ERR_ARG;
  if (cm_dtype != LBDD_CM_I32 && cm_dtype != LBDD_CM_I16) return LBDD_ERR_ARG;
  const int elem = cm_dtype == LBDD_CM_I16 ? 2 : 4;
  if (ld < k || (ld * elem) % 16 != 0 || (reinterpret_cast<uintptr_t>(cm_dev) & 15) != 0)
    return LBDD_ERR_ARG;
  if (k > bt_max_k(elem)) return LBDD_ERR_ARG;
  if (workspace_bytes < bt_workspace_bytes(n, k)) return LBDD_ERR_ARG;
  int dev = 0, sms = 0;
  int rc = check_device(&dev, &sms);
  if (rc) return rc;
  CK(best_transfer_run(n, k, cm_dev, elem, ld, assign_dev, tc_dev, td_dev, workspace,
                       static_cast<cudaStream_t>(stream), sms));
  return LBDD_OK;
}
