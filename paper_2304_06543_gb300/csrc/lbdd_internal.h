// Host-side internals shared by the translation units of the C ABI
// (lbdd_api.cu: single solvers and the best-transfer call; lbdd_batch.cu:
// batched launches and the cluster-size autotuner; lbdd_server.cu: the
// request server).  Not part of the public interface.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/lbdd.h"
#include "lbdd_device.cuh"

namespace lbdd {
// asral_solver.cu
size_t solver_smem_bytes(int32_t k, int C, int elem_bytes, bool with_slice);
int solver_max_k(int C, int elem_bytes);
int solver_max_clusters(int C, int elem_bytes, size_t smem);
cudaError_t prepare_solver(int C, int elem_bytes, size_t smem);
cudaError_t launch_solver(const DevInst* d_insts, int ninst, int* d_counter, int C,
                          int nclusters, int elem_bytes, size_t smem, int flags,
                          cudaStream_t st, uint64_t quantum_ns = 0, bool set_attrs = true);
// best_transfer.cu
size_t bt_workspace_bytes(int32_t n, int32_t k);
int bt_max_k(int elem_bytes);
cudaError_t best_transfer_run(int32_t n, int32_t k, const void* cm, int elem_bytes, int64_t ld,
                              const int32_t* assign, int32_t* tc, int32_t* td, void* ws,
                              cudaStream_t st, int num_sms);

// Dynamic shared memory a solver CTA may request: the 227 KB a block may
// opt into, less 1 KB for the kernel's static shared variables (400 bytes
// at present), which count against the same limit.
constexpr size_t kMaxSmem = 227 * 1024 - 1024;
}  // namespace lbdd

struct lbdd_solver {
  int32_t n = 0, k = 0;
  int elem = 4;
  int64_t ld = 0;
  void* cm = nullptr;
  int32_t *cap = nullptr, *pen = nullptr, *smin = nullptr, *order = nullptr,
          *sort_tmp = nullptr, *assign = nullptr, *pos = nullptr, *load = nullptr,
          *seg_size = nullptr, *page_tab = nullptr, *pool = nullptr, *free_stack = nullptr,
          *tc = nullptr, *td = nullptr, *counter = nullptr;
  int64_t* ctl = nullptr;
  lbdd::DevInst* d_inst = nullptr;
  lbdd::DevInst h_inst;
  cudaStream_t st = nullptr;
  int cluster = 0;         // 0 = auto
  int ncyc_skip = 1;
  int npath_reuse = 1;
  int tc_smem = 1;
  int phase_timers = 0;
  int strict = 0;          // strict-LBDD instance (Alg. 5), k includes a dummy center if any
  int device = 0;
  int num_sms = 0;
  int32_t n_cap = 0;       // units the unit-indexed arrays and the page pool hold (>= n)
  int in_batches = 0;      // batches that hold a copy of this solver's device view
  int32_t* ins_row = nullptr;  // k costs of a unit being inserted (device staging)
  size_t bytes = 0;        // device bytes held now
  std::vector<void*> allocs;
  std::vector<size_t> sizes;
};

namespace lbdd {
// Records the CUDA error text for lbdd_last_cuda_error and maps it to a status.
int cuda_fail(cudaError_t e, const char* what);
int check_device(int* dev, int* sms);
// Dynamic shared memory of a launch for k centers on C-CTA clusters (with the
// owned cost slice when it fits).
size_t launch_smem(int32_t k, int C, int elem);
// Whether an instance with k centers and elem-byte costs runs on C-CTA clusters.
bool fits_k(int32_t k, int elem, int C);
// Latency-oriented default cluster size of one solver (largest that fits).
int choose_cluster(lbdd_solver* s);
int solver_flags(const lbdd_solver* s);
int status_to_rc(int64_t st);
// Device bytes lbdd_create allocates for an n x k instance whose costs are
// stored with elem-byte entries (in_elem: entry size of the caller's CM,
// which is held alongside the narrowed copy while it is made).
size_t solver_footprint(int32_t n, int32_t k, int in_elem, int elem);
// A new solver on the same device holding a copy of src's instance (costs,
// capacities, penalties), in the initial state.
int clone_solver(const lbdd_solver* src, lbdd_solver** out);
// A smaller instance shaped like src: its first n_sub units, capacities
// scaled by n_sub / n (at least 1), the same penalties.
int clone_prefix(const lbdd_solver* src, int32_t n_sub, lbdd_solver** out);
// Advances s by up to max_rounds rounds on C-CTA clusters; *ms is the
// kernel's device time.
int solve_timed(lbdd_solver* s, int64_t max_rounds, int C, float* ms);
}  // namespace lbdd

#define LBDD_CK(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return lbdd::cuda_fail(e_, #call); \
  } while (0)
