// Cost matrix from a road network (Section 3.4 "Demand-service cost matrix
// construction"; Section 5: the paper's CM is the shortest road distance from
// every demand node to every service center of the New Delhi network).
//
// One CTA per center computes single-source shortest paths over the CSR graph
// by label correcting: the frontier of a sweep is the set of nodes whose
// label dropped in the previous sweep; every frontier node relaxes its edges
// with atomicMin on the labels, and a node whose label dropped is appended to
// the next frontier once per sweep (a per-node mark holds the last sweep it
// was appended in).  Labels only decrease and lengths are positive integers,
// so the sweeps end with the exact shortest distances whatever order the
// relaxations take; the CM is therefore bit-identical to a sequential
// Dijkstra.  The labels of all centers (k x V int32) stay L2-resident for
// road graphs of the paper's size (65,000 nodes, about 100 centers).
// A gather then writes CM[d][s] = dist_s(demand[d]), demand-major.
#include <algorithm>
#include <cstdint>

#include "lbdd_internal.h"

namespace lbdd {

constexpr int kRoadThreads = 512;
constexpr int32_t kRoadInf = INT32_MAX;

// err[0]: bad graph or ids; err[1]: largest length; err[2]: unreachable
// demand; err[3]: sweep limit reached (cannot happen with positive lengths).
__global__ void road_check(int32_t V, const int32_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col, const int32_t* __restrict__ w,
                           int32_t k, const int32_t* __restrict__ centers, int32_t n,
                           const int32_t* __restrict__ demand, int* err) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = g; v < V; v += gs)
    if (row_ptr[v] > row_ptr[v + 1] || row_ptr[v] < 0) atomicExch(err, 1);
  const int32_t E = row_ptr[V];
  if (row_ptr[0] != 0 || E < 0) atomicExch(err, 1);
  int mx = 0;
  for (int64_t e = g; e < E; e += gs) {
    if (w[e] < 1 || (uint32_t)col[e] >= (uint32_t)V) atomicExch(err, 1);
    mx = max(mx, w[e]);
  }
  atomicMax(err + 1, mx);
  for (int64_t s = g; s < k; s += gs)
    if ((uint32_t)centers[s] >= (uint32_t)V) atomicExch(err, 1);
  for (int64_t d = g; d < n; d += gs)
    if ((uint32_t)demand[d] >= (uint32_t)V) atomicExch(err, 1);
}

__global__ void __launch_bounds__(kRoadThreads)
road_sssp(int32_t V, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
          const int32_t* __restrict__ w, int32_t k, const int32_t* __restrict__ centers,
          int32_t* dist, int32_t* queues, int32_t* marks, int* err) {
  __shared__ int s_cnt[2];
  const int tid = threadIdx.x;
  int32_t* qa = queues + (int64_t)blockIdx.x * 2 * V;
  int32_t* qb = qa + V;
  int32_t* mk = marks + (int64_t)blockIdx.x * V;
  for (int32_t s = blockIdx.x; s < k; s += gridDim.x) {
    int32_t* d = dist + (int64_t)s * V;
    for (int32_t v = tid; v < V; v += kRoadThreads) {
      d[v] = kRoadInf;
      mk[v] = -1;
    }
    __syncthreads();
    if (tid == 0) {
      d[centers[s]] = 0;
      qa[0] = centers[s];
      s_cnt[0] = 0;
      s_cnt[1] = 0;
    }
    __syncthreads();
    int na = 1, cur = 0;
    for (int32_t sweep = 0; na > 0; ++sweep) {
      if (sweep > V) {        // positive lengths converge within V sweeps
        if (tid == 0) atomicExch(err + 3, 1);
        break;
      }
      const int32_t* qin = cur ? qb : qa;
      int32_t* qout = cur ? qa : qb;
      int* cnt_out = &s_cnt[cur ^ 1];
      for (int i = tid; i < na; i += kRoadThreads) {
        const int32_t u = qin[i];
        const int32_t du = __ldcg(d + u);
        const int32_t e1 = row_ptr[u + 1];
        for (int32_t e = row_ptr[u]; e < e1; ++e) {
          const int32_t v = col[e];
          const int32_t nd = du + w[e];
          if (nd < __ldcg(d + v) && nd < atomicMin(d + v, nd) && atomicExch(mk + v, sweep) != sweep)
            qout[atomicAdd(cnt_out, 1)] = v;
        }
      }
      __syncthreads();
      na = *cnt_out;
      if (tid == 0) s_cnt[cur] = 0;   // the consumed frontier's counter, reused next sweep
      cur ^= 1;
      __syncthreads();
    }
    __syncthreads();
  }
}

__global__ void road_gather(int32_t V, int32_t k, int32_t n, const int32_t* __restrict__ dist,
                            const int32_t* __restrict__ demand, int32_t* cm, int64_t ld,
                            int* err) {
  const int64_t total = (int64_t)n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dd = i / k, s = i - dd * k;
    const int32_t v = __ldcg(dist + s * V + demand[dd]);
    if (v == kRoadInf || v < 1) atomicExch(err + 2, 1);
    cm[dd * ld + s] = v;
  }
}

}  // namespace lbdd

using namespace lbdd;

extern "C" int lbdd_road_cm(int32_t V, const int32_t* row_ptr, const int32_t* col,
                            const int32_t* w, int32_t k, const int32_t* centers, int32_t n,
                            const int32_t* demand, int32_t* cm, int64_t ld, void* stream) {
  if (V < 1 || k < 1 || n < 1 || ld < k || !row_ptr || !col || !w || !centers || !demand || !cm)
    return LBDD_ERR_ARG;
  int dev = 0, sms = 0;
  int rc = check_device(&dev, &sms);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = std::min(k, sms);
  int32_t *dist = nullptr, *queues = nullptr, *marks = nullptr;
  int* err = nullptr;
  auto release = [&]() {
    cudaFreeAsync(dist, st);
    cudaFreeAsync(queues, st);
    cudaFreeAsync(marks, st);
    cudaFreeAsync(err, st);
    cudaStreamSynchronize(st);
  };
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&err), 4 * sizeof(int), st);
  if (!e) e = cudaMemsetAsync(err, 0, 4 * sizeof(int), st);
  if (!e) {
    road_check<<<sms * 4, 256, 0, st>>>(V, row_ptr, col, w, k, centers, n, demand, err);
    e = cudaGetLastError();
  }
  int h[4] = {0, 0, 0, 0};
  if (!e) e = cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) { rc = cuda_fail(e, "lbdd_road_cm check"); release(); return rc; }
  // labels are int32: every path length must fit
  if (h[0] != 0 || (int64_t)h[1] * (V - 1) >= (int64_t)kRoadInf) { release(); return LBDD_ERR_ARG; }
  e = cudaMallocAsync(reinterpret_cast<void**>(&dist), 4ull * k * V, st);
  if (!e) e = cudaMallocAsync(reinterpret_cast<void**>(&queues), 8ull * grid * V, st);
  if (!e) e = cudaMallocAsync(reinterpret_cast<void**>(&marks), 4ull * grid * V, st);
  if (!e) {
    road_sssp<<<grid, kRoadThreads, 0, st>>>(V, row_ptr, col, w, k, centers, dist, queues, marks,
                                             err);
    e = cudaGetLastError();
  }
  if (!e) {
    road_gather<<<sms * 8, 256, 0, st>>>(V, k, n, dist, demand, cm, ld, err);
    e = cudaGetLastError();
  }
  if (!e) e = cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) { rc = cuda_fail(e, "lbdd_road_cm"); release(); return rc; }
  release();
  if (h[2] != 0 || h[3] != 0) return LBDD_ERR_ARG;   // a demand node no center reaches
  return LBDD_OK;
}
