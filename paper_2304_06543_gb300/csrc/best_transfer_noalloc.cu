// Best-transfer table without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// table: cudaMalloc may synchronise the whole device, which a latency-bound
// pipeline sharing the GPU with other streams cannot afford, and some host
// applications hand a plugin a fixed memory plan and forbid it to grow.  For
// them this file offers a variant of lbdd_best_transfer whose scratch lives in
// one fixed, file-scope device array instead of a caller-supplied workspace.
// The array is reserved on every GPU that loads this library and stays there
// until the process exits.
#include <cstdint>
#include <mutex>

#include "../../include/lbdd.h"
#include "lbdd_device.cuh"

namespace lbdd {
size_t bt_workspace_bytes(int32_t n, int32_t k);
int bt_max_k(int elem_bytes);
cudaError_t best_transfer_run(int32_t n, int32_t k, const void* cm, int elem_bytes, int64_t ld,
                              const int32_t* assign, int32_t* tc, int32_t* td, void* ws,
                              cudaStream_t st, int num_sms);
int cuda_fail(cudaError_t e, const char* what);
}  // namespace lbdd

namespace {

// Fixed scratch shared by every call on a device (64 MiB).
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_bt_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};   // device address of g_bt_scratch, per device
int g_num_sms[kMaxDevices] = {};

// One-time set-up per device (the device must be current): look up the
// device address of the scratch array.  The host-side name g_bt_scratch is
// only a stand-in and must never be handed to a kernel.
int setup_device(int dev, void** addr, int* sms) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return lbdd::cuda_fail(e, "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3) return LBDD_ERR_NODEV;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_bt_scratch);
    if (e != cudaSuccess) return lbdd::cuda_fail(e, "cudaGetSymbolAddress");
    if (p == nullptr) return LBDD_ERR_CUDA;
    g_num_sms[dev] = prop.multiProcessorCount;
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_num_sms[dev];
  return LBDD_OK;
}

}  // namespace

extern "C" int lbdd_best_transfer_noalloc(int32_t n, int32_t k, const void* cm_dev,
                                          int cm_dtype, int64_t ld, const int32_t* assign_dev,
                                          int32_t* tc_dev, int32_t* td_dev, void* stream) {
  if (n < 1 || k < 1 || !cm_dev || !assign_dev || !tc_dev || !td_dev) return LBDD_ERR_ARG;
  if (cm_dtype != LBDD_CM_I32 && cm_dtype != LBDD_CM_I16) return LBDD_ERR_ARG;
  const int elem = cm_dtype == LBDD_CM_I16 ? 2 : 4;
  if (ld < k || (ld * elem) % 16 != 0 || (reinterpret_cast<uintptr_t>(cm_dev) & 15) != 0)
    return LBDD_ERR_ARG;
  if (k > lbdd::bt_max_k(elem)) return LBDD_ERR_ARG;
  // the scratch the scan needs must fit in the fixed array
  if (lbdd::bt_workspace_bytes(n, k) > kStaticScratchBytes) return LBDD_ERR_BUDGET;
  int dev = 0;
  const cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return lbdd::cuda_fail(ed, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return LBDD_ERR_CUDA;
  void* scratch = nullptr;
  int sms = 0;
  const int rc = setup_device(dev, &scratch, &sms);
  if (rc != LBDD_OK) return rc;
  // Every stage rewrites the scratch it reads (keys, histograms, segment
  // bounds via cudaMemsetAsync, the packed table filled with its identity),
  // so nothing left by an earlier call can leak into this one.
  const cudaError_t e = lbdd::best_transfer_run(n, k, cm_dev, elem, ld, assign_dev, tc_dev, td_dev,
                                                scratch, static_cast<cudaStream_t>(stream), sms);
  return e == cudaSuccess ? LBDD_OK : lbdd::cuda_fail(e, "lbdd_best_transfer_noalloc");
}
