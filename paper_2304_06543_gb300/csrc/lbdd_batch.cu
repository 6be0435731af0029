// Batched solves: many independent LBDD instances advanced by one set of
// persistent launches, replayed as a single CUDA graph.
//
// Every instance is an independent run of Alg. 2, so a batch needs no
// communication between instances; the only decisions are how many CTAs each
// instance's cluster gets and how the GPU's SMs are shared between instances
// of different sizes.
//
//  * Cluster size per instance.  A cluster of C CTAs owns k/C columns of the
//    best-transfer table each (Bellman-Ford relaxation is split by column).
//    Larger C shortens a round (lower latency) but costs C SMs; for a batch
//    the SM-time per round, t(k, C) * C, decides throughput.  The autotuner
//    (lbdd_autotune) measures t(k, C) on a clone of one instance per
//    (cost width, k bucket) and keeps the table per device.  The plan starts
//    every instance at its throughput-best C and moves the instances that
//    would outlast the rest of the batch to faster (larger) clusters.
//  * Groups.  Instances with the same cost width and C form a group: one
//    persistent launch of that group's clusters, each cluster pulling the
//    next instance from a device-side counter, longest estimated solve
//    first.  The SMs are shared between the groups in proportion to their
//    estimated SM-time, and the groups run concurrently on forked streams.
//  * One graph.  Setting every instance's round target, resetting the
//    counters, the forked group launches and the status gather are captured
//    once into a CUDA graph; lbdd_batch_run replays it.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "lbdd_internal.h"

using namespace lbdd;

#define CK(call) LBDD_CK(call)

namespace lbdd {

// ------------------------------------------------------------- kernels ---

// Round target of every instance: max_rounds more rounds (all remaining if
// max_rounds < 0).  Instances in an error state keep their target.
__global__ void batch_set_targets(const DevInst* __restrict__ insts, int m,
                                  const int64_t* __restrict__ max_rounds) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t* c = insts[i].ctl;
  if (c[CTL_STATUS] != 0) return;
  const int64_t n = insts[i].n, mr = *max_rounds;
  c[CTL_TARGET] = mr < 0 ? n : min(n, c[CTL_ROUNDS] + mr);
}

// out[2i] = status, out[2i+1] = rounds done of instance i.
__global__ void batch_gather(const DevInst* __restrict__ insts, int m, int64_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t* c = insts[i].ctl;
  out[2 * i] = c[CTL_STATUS];
  out[2 * i + 1] = c[CTL_ROUNDS];
}

// --------------------------------------------------------- tuning table ---

constexpr int kMaxDevices = 64;
constexpr int kBuckets = 17;            // bucket b: 2^(b-1) < k <= 2^b
constexpr int kNC = 5;                  // cluster sizes 1, 2, 4, 8, 16
struct TuneTable {
  double ns[2][kBuckets][kNC];          // ns per round; 0 = not measured
};
static std::mutex g_tune_mu;
static TuneTable g_tune[kMaxDevices];

static int bucket_of(int32_t k) {
  int b = 0;
  while ((1 << b) < k && b < kBuckets - 1) ++b;
  return b;
}
static int cidx(int C) { return C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : C == 8 ? 3 : 4; }
static int wid(int elem) { return elem == 2 ? 0 : 1; }

// Default cluster size when nothing is measured: about 128 owned columns
// per CTA (fewer SMs per instance than a lone solve, which favours latency).
static int default_cluster(int32_t k, int elem) {
  int C = 1;
  while (C < 16 && (int64_t)C * 128 < k) C <<= 1;
  while (C < 16 && !fits_k(k, elem, C)) C <<= 1;
  return C;
}

// ------------------------------------------------------------------ plan ---

struct Group {
  int elem = 4, C = 1, ncl = 1;
  size_t smem = 0;
  int flags = 0;
  std::vector<int> idx;                 // instances, longest estimate first
  double work = 0, longest = 0;         // SM-ns, ns
};

struct Est {
  int C;
  double t;                             // ns per round (model units when untuned)
};

// Cluster size and per-round estimate of every instance.
using Cands = std::vector<std::vector<std::pair<int, double>>>;

// Cluster size and per-round estimate of every instance: the least SM-time
// per round among the measured sizes (the default rule when unmeasured).
// cands[i] lists instance i's measured (C, ns per round) pairs.
static int choose_sizes(lbdd_solver* const* v, int m, int forced_C, int dev,
                        std::vector<Est>* est, Cands* cands) {
  est->assign(m, Est{1, 1.0});
  cands->assign(m, {});
  TuneTable tab;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tab = g_tune[dev];
  }
  for (int i = 0; i < m; ++i) {
    const lbdd_solver* s = v[i];
    if (forced_C > 0) {
      if (!fits_k(s->k, s->elem, forced_C)) return LBDD_ERR_ARG;
      (*est)[i] = Est{forced_C, (double)s->k / forced_C + 1.0};
      continue;
    }
    const double* row = tab.ns[wid(s->elem)][bucket_of(s->k)];
    for (int C = 1; C <= 16; C <<= 1)
      if (row[cidx(C)] > 0 && fits_k(s->k, s->elem, C)) (*cands)[i].push_back({C, row[cidx(C)]});
    if ((*cands)[i].empty()) {
      const int C = default_cluster(s->k, s->elem);
      if (!fits_k(s->k, s->elem, C)) return LBDD_ERR_ARG;
      (*est)[i] = Est{C, (double)s->k / C + 1.0};
      continue;
    }
    // throughput-best: least SM-time per round; ties go to the larger cluster
    Est best{0, 0};
    for (auto& c : (*cands)[i])
      if (best.C == 0 || c.second * c.first <= best.t * best.C) best = Est{c.first, c.second};
    (*est)[i] = best;
  }
  return LBDD_OK;
}

// Order of instances inside a group's work queue.
enum Order { LONGEST_FIRST = 0, SHORTEST_FIRST = 1 };

// Groups of instances with equal (cost width, cluster size, options).
static int build_groups(lbdd_solver* const* v, const int64_t* rem, int m,
                        const std::vector<Est>& est, Order order, const uint8_t* first,
                        std::vector<Group>* groups) {
  groups->clear();
  for (int i = 0; i < m; ++i) {
    Group* g = nullptr;
    const int fl = solver_flags(v[i]);
    for (auto& x : *groups)
      if (x.elem == v[i]->elem && x.C == est[i].C && x.flags == fl) g = &x;
    if (!g) {
      groups->push_back(Group{});
      g = &groups->back();
      g->elem = v[i]->elem;
      g->C = est[i].C;
      g->flags = fl;
    }
    g->idx.push_back(i);
    const double len = (double)rem[i] * est[i].t;
    g->work += len * est[i].C;
    g->longest = std::max(g->longest, len);
  }
  // heaviest group first; inside a group the instances marked `first`, then
  // longest (or shortest) instance first
  std::stable_sort(groups->begin(), groups->end(),
                   [](const Group& a, const Group& b) { return a.work > b.work; });
  for (auto& g : *groups) {
    std::stable_sort(g.idx.begin(), g.idx.end(), [&](int a, int b) {
      const bool fa = first && first[a], fb = first && first[b];
      if (fa != fb) return fa;
      const double la = (double)rem[a] * est[a].t, lb = (double)rem[b] * est[b].t;
      return order == LONGEST_FIRST ? la > lb : la < lb;
    });
    int32_t kmax = 0;
    for (int i : g.idx) kmax = std::max(kmax, v[i]->k);
    g.smem = launch_smem(kmax, g.C, g.elem);
    if (g.smem > kMaxSmem) return LBDD_ERR_ARG;
  }
  return LBDD_OK;
}

// Upper bound on a group's clusters: its instances, co-residency, the SMs.
static int group_cap(const Group& g, int max_clusters, int sms, int* cap) {
  const int fit = solver_max_clusters(g.C, g.elem, g.smem);
  if (fit < 1) {
    (void)cudaGetLastError();   // the refused query's error is reported as LBDD_ERR_ARG
    return LBDD_ERR_ARG;
  }
  *cap = std::min<int>((int)g.idx.size(), fit);
  if (max_clusters > 0) *cap = std::min(*cap, max_clusters);
  *cap = std::max(1, std::min(*cap, sms / g.C));
  return LBDD_OK;
}

// SMs in proportion to each group's estimated SM-time.
static int allocate_proportional(std::vector<Group>* groups, int max_clusters, int sms) {
  double total = 0;
  for (auto& g : *groups) total += g.work;
  int used = 0;
  std::vector<int> cap(groups->size());
  for (size_t gi = 0; gi < groups->size(); ++gi) {
    Group& g = (*groups)[gi];
    int rc = group_cap(g, max_clusters, sms, &cap[gi]);
    if (rc) return rc;
    const double share = total > 0 ? sms * g.work / total : sms;
    g.ncl = std::max(1, std::min(cap[gi], (int)std::floor(share / g.C)));
    used += g.ncl * g.C;
  }
  auto need = [&](const Group& g) { return g.work / (g.ncl * g.C); };
  while (used > sms) {
    int best = -1;
    for (size_t gi = 0; gi < groups->size(); ++gi)
      if ((*groups)[gi].ncl > 1 && (best < 0 || need((*groups)[gi]) < need((*groups)[best])))
        best = (int)gi;
    if (best < 0) break;
    (*groups)[best].ncl--;
    used -= (*groups)[best].C;
  }
  for (;;) {
    int best = -1;
    for (size_t gi = 0; gi < groups->size(); ++gi) {
      const Group& g = (*groups)[gi];
      if (g.ncl < cap[gi] && used + g.C <= sms && (best < 0 || need(g) > need((*groups)[best])))
        best = (int)gi;
    }
    if (best < 0) break;
    (*groups)[best].ncl++;
    used += (*groups)[best].C;
  }
  return LBDD_OK;
}

// rem[i]: rounds instance i has left.  Groups, their cluster counts and
// queue orders for one pass over the instances: sizes by least SM-time per
// round, long instances moved to faster clusters, SMs shared in proportion
// to estimated SM-time.
static int make_plan(lbdd_solver* const* v, const int64_t* rem, int m, int forced_C,
                     int max_clusters, int dev, int sms, Order order, const uint8_t* first,
                     std::vector<Group>* groups, std::vector<int>* cluster_of) {
  std::vector<Est> est;
  Cands cands;
  int rc = choose_sizes(v, m, forced_C, dev, &est, &cands);
  if (rc) return rc;
  // instances longer than the plan's SM-time per SM get faster clusters,
  // longest first, while that lowers their own time
  for (int iter = 0; iter < 4 * m && forced_C == 0; ++iter) {
    double total = 0, top_len = 0;
    int top = -1;
    for (int i = 0; i < m; ++i) {
      const double len = (double)rem[i] * est[i].t;
      total += len * est[i].C;
      if (!cands[i].empty() && len > top_len) { top_len = len; top = i; }
    }
    if (top < 0 || top_len <= total / std::max(1, sms)) break;
    Est next{0, 0};
    for (auto& c : cands[top])
      if (c.first > est[top].C && c.second < est[top].t && (next.C == 0 || c.second < next.t))
        next = Est{c.first, c.second};
    if (next.C == 0) { cands[top].clear(); continue; }
    est[top] = next;
  }
  rc = build_groups(v, rem, m, est, order, first, groups);
  if (!rc) rc = allocate_proportional(groups, max_clusters, sms);
  if (rc) return rc;
  cluster_of->assign(m, 0);
  for (int i = 0; i < m; ++i) (*cluster_of)[i] = est[i].C;
  return LBDD_OK;
}

}  // namespace lbdd

// ----------------------------------------------------------- the batch ---

constexpr int kMaxGroups = 16;          // one per (cost width, cluster size, solver options)

struct lbdd_batch {
  int capacity = 0;                 // instances the buffers hold
  std::vector<lbdd_solver*> solvers;
  std::vector<Group> groups;
  std::vector<int> cluster_of;      // per instance (caller's order)
  std::vector<int> slot_of;         // caller's index -> position in d_insts
  std::vector<int> offset;          // per group: first position in d_insts
  cudaStream_t st = nullptr;
  cudaStream_t side[kMaxGroups - 1] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kMaxGroups - 1] = {};
  DevInst* d_insts = nullptr;
  DevInst* h_insts = nullptr;       // pinned staging of d_insts
  int* d_counters = nullptr;
  int64_t* d_params = nullptr;
  int64_t* d_out = nullptr;
  int64_t* h_params = nullptr;      // pinned
  int64_t* h_out = nullptr;         // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t quantum_ns = 0;
  int dev = 0, sms = 0;
};

static void batch_free(lbdd_batch* b) {
  for (lbdd_solver* x : b->solvers) x->in_batches--;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->st) cudaStreamSynchronize(b->st);
  for (auto s : b->side)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  cudaFree(b->d_insts);
  cudaFree(b->d_counters);
  cudaFree(b->d_params);
  cudaFree(b->d_out);
  cudaFreeHost(b->h_insts);
  cudaFreeHost(b->h_params);
  cudaFreeHost(b->h_out);
  delete b;
}

// Issues one pass of the batch on b->st (asynchronous).
static int batch_enqueue(lbdd_batch* b) {
  const int m = (int)b->solvers.size();
  CK(cudaMemcpyAsync(b->d_params, b->h_params, sizeof(int64_t), cudaMemcpyHostToDevice, b->st));
  batch_set_targets<<<(m + 255) / 256, 256, 0, b->st>>>(b->d_insts, m, b->d_params);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->groups.size(), b->st));
  CK(cudaEventRecord(b->fork, b->st));
  for (size_t g = 0; g < b->groups.size(); ++g) {
    const Group& G = b->groups[g];
    cudaStream_t s = g == 0 ? b->st : b->side[g - 1];
    if (g > 0) CK(cudaStreamWaitEvent(s, b->fork, 0));
    CK(launch_solver(b->d_insts + b->offset[g], (int)G.idx.size(), b->d_counters + g, G.C, G.ncl,
                     G.elem, G.smem, G.flags, s, b->quantum_ns, false));
    if (g > 0) {
      CK(cudaEventRecord(b->join[g - 1], s));
      CK(cudaStreamWaitEvent(b->st, b->join[g - 1], 0));
    }
  }
  batch_gather<<<(m + 255) / 256, 256, 0, b->st>>>(b->d_insts, m, b->d_out);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(b->h_out, b->d_out, sizeof(int64_t) * 2 * m, cudaMemcpyDeviceToHost, b->st));
  return LBDD_OK;
}

namespace lbdd {

// Launch state for up to `capacity` instances on `stream` (no plan yet).
int batch_alloc(lbdd_batch** out, int capacity, uint64_t quantum_ns, void* stream) {
  if (!out || capacity < 1) return LBDD_ERR_ARG;
  *out = nullptr;
  int dev = 0, sms = 0;
  int rc = check_device(&dev, &sms);
  if (rc) return rc;
  if (dev >= kMaxDevices) return LBDD_ERR_NODEV;
  lbdd_batch* b = new (std::nothrow) lbdd_batch();
  if (!b) return LBDD_ERR_OOM;
  b->capacity = capacity;
  b->st = static_cast<cudaStream_t>(stream);
  b->quantum_ns = quantum_ns;
  b->dev = dev;
  b->sms = sms;
  cudaError_t e;
  auto cf = [&](cudaError_t err, const char* w) { batch_free(b); return cuda_fail(err, w); };
  if ((e = cudaMalloc(&b->d_insts, sizeof(DevInst) * capacity))) return cf(e, "batch insts");
  if ((e = cudaMalloc(&b->d_counters, sizeof(int) * kMaxGroups))) return cf(e, "batch counters");
  if ((e = cudaMalloc(&b->d_params, sizeof(int64_t) * 2))) return cf(e, "batch params");
  if ((e = cudaMalloc(&b->d_out, sizeof(int64_t) * 2 * capacity))) return cf(e, "batch out");
  if ((e = cudaMallocHost(&b->h_insts, sizeof(DevInst) * capacity))) return cf(e, "batch insts (host)");
  if ((e = cudaMallocHost(&b->h_params, sizeof(int64_t) * 2))) return cf(e, "batch params (host)");
  if ((e = cudaMallocHost(&b->h_out, sizeof(int64_t) * 2 * capacity))) return cf(e, "batch out (host)");
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming))) return cf(e, "event");
  for (int g = 0; g < kMaxGroups - 1; ++g) {
    if ((e = cudaStreamCreateWithFlags(&b->side[g], cudaStreamNonBlocking))) return cf(e, "stream");
    if ((e = cudaEventCreateWithFlags(&b->join[g], cudaEventDisableTiming))) return cf(e, "event");
  }
  *out = b;
  return LBDD_OK;
}

// Plans a pass over solvers[0..m) (rem: rounds each has left; NULL = all n)
// and stages their instance records on b->st.  Every solver must live on
// the batch's device.
int batch_set(lbdd_batch* b, lbdd_solver* const* solvers, const int64_t* rem, int m,
              int cluster_size, int max_clusters, bool shortest_first, const uint8_t* first) {
  if (!b || !solvers || m < 1 || m > b->capacity || cluster_size < 0 || cluster_size > 16 ||
      max_clusters < 0 || (cluster_size & (cluster_size - 1)) != 0)
    return LBDD_ERR_ARG;
  std::vector<int64_t> r(m);
  for (int i = 0; i < m; ++i) {
    if (!solvers[i] || solvers[i]->device != b->dev) return LBDD_ERR_ARG;
    r[i] = rem ? std::max<int64_t>(rem[i], 1) : solvers[i]->n;
  }
  for (lbdd_solver* old : b->solvers) old->in_batches--;
  b->solvers.assign(solvers, solvers + m);
  for (lbdd_solver* x : b->solvers) x->in_batches++;
  int rc = make_plan(solvers, r.data(), m, cluster_size, max_clusters, b->dev, b->sms,
                     shortest_first ? SHORTEST_FIRST : LONGEST_FIRST, first, &b->groups,
                     &b->cluster_of);
  if (rc) return rc;
  if (b->groups.size() > (size_t)kMaxGroups) return LBDD_ERR_ARG;
  b->slot_of.assign(m, 0);
  b->offset.clear();
  int pos = 0;
  for (auto& g : b->groups) {
    b->offset.push_back(pos);
    for (int i : g.idx) {
      b->slot_of[i] = pos;
      b->h_insts[pos++] = solvers[i]->h_inst;
    }
  }
  CK(cudaMemcpyAsync(b->d_insts, b->h_insts, sizeof(DevInst) * m, cudaMemcpyHostToDevice, b->st));
  for (auto& g : b->groups) CK(prepare_solver(g.C, g.elem, g.smem));
  return LBDD_OK;
}

// Captures one pass of the current plan into a CUDA graph.
int batch_capture(lbdd_batch* b) {
  // a private stream for capture, so that work already queued on the
  // caller's stream stays out of the graph
  cudaStream_t cap_st;
  CK(cudaStreamSynchronize(b->st));
  CK(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
  cudaStream_t user = b->st;
  b->st = cap_st;
  cudaError_t e = cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal);
  int rc = e ? cuda_fail(e, "begin capture") : batch_enqueue(b);
  cudaGraph_t graph = nullptr;
  if (!e) e = cudaStreamEndCapture(cap_st, &graph);
  cudaStreamDestroy(cap_st);
  b->st = user;
  if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
  if (e) return cuda_fail(e, "end capture");
  b->graph = graph;
  CK(cudaGraphInstantiate(&b->exec, graph, 0));
  return LBDD_OK;
}

// Starts one pass (max_rounds more rounds for every instance) on b->st.
int batch_launch(lbdd_batch* b, int64_t max_rounds) {
  b->h_params[0] = max_rounds;
  for (auto& g : b->groups) CK(prepare_solver(g.C, g.elem, g.smem));
  if (b->exec) {
    CK(cudaGraphLaunch(b->exec, b->st));
    return LBDD_OK;
  }
  return batch_enqueue(b);
}

// Waits for the pass; *first_rc = the first failing instance's status.
int batch_wait(lbdd_batch* b, int* first_rc) {
  CK(cudaStreamSynchronize(b->st));
  int first = LBDD_OK;
  for (size_t i = 0; i < b->solvers.size(); ++i) {
    const int r = status_to_rc(b->h_out[2 * b->slot_of[i]]);
    if (r && first == LBDD_OK) first = r;
  }
  if (first_rc) *first_rc = first;
  return LBDD_OK;
}

int batch_launches(const lbdd_batch* b) { return 2 + (int)b->groups.size(); }
int64_t batch_rounds(const lbdd_batch* b, int i) { return b->h_out[2 * b->slot_of[i] + 1]; }
int64_t batch_status(const lbdd_batch* b, int i) { return b->h_out[2 * b->slot_of[i]]; }
void batch_destroy(lbdd_batch* b) {
  if (b) batch_free(b);
}

}  // namespace lbdd

// ------------------------------------------------------------- C ABI ---

extern "C" int lbdd_batch_create(lbdd_batch** out, lbdd_solver* const* solvers, int m,
                                 int cluster_size, int max_clusters, void* stream) {
  if (!out) return LBDD_ERR_ARG;
  *out = nullptr;
  if (!solvers || m < 1) return LBDD_ERR_ARG;
  lbdd_batch* b = nullptr;
  int rc = batch_alloc(&b, m, 0, stream);
  if (rc) return rc;
  rc = batch_set(b, solvers, nullptr, m, cluster_size, max_clusters, false, nullptr);
  if (!rc) rc = batch_capture(b);
  if (rc) { batch_free(b); return rc; }
  *out = b;
  return LBDD_OK;
}

extern "C" int lbdd_batch_run(lbdd_batch* b, int64_t max_rounds) {
  if (!b) return LBDD_ERR_ARG;
  int first = LBDD_OK;
  int rc = batch_launch(b, max_rounds);
  if (!rc) rc = batch_wait(b, &first);
  return rc ? rc : first;
}

extern "C" int lbdd_batch_plan(const lbdd_batch* b, int32_t* cluster_of, int32_t* ngroups,
                               int32_t* group_cluster, int32_t* group_clusters,
                               int32_t* group_size, int max_groups) {
  if (!b) return LBDD_ERR_ARG;
  if (cluster_of)
    for (size_t i = 0; i < b->cluster_of.size(); ++i) cluster_of[i] = b->cluster_of[i];
  if (ngroups) *ngroups = (int32_t)b->groups.size();
  for (int g = 0; g < (int)b->groups.size() && g < max_groups; ++g) {
    if (group_cluster) group_cluster[g] = b->groups[g].C;
    if (group_clusters) group_clusters[g] = b->groups[g].ncl;
    if (group_size) group_size[g] = (int32_t)b->groups[g].idx.size();
  }
  return LBDD_OK;
}

extern "C" void lbdd_batch_destroy(lbdd_batch* b) { batch_destroy(b); }

extern "C" int lbdd_solve_batch(lbdd_solver* const* solvers, int m, int64_t max_rounds,
                                int cluster_size, int max_clusters, void* stream) {
  if (!solvers || m < 1) return LBDD_ERR_ARG;
  lbdd_batch* b = nullptr;
  int rc = batch_alloc(&b, m, 0, stream);
  if (rc) return rc;
  rc = batch_set(b, solvers, nullptr, m, cluster_size, max_clusters, false, nullptr);
  int first = LBDD_OK;
  if (!rc) rc = batch_launch(b, max_rounds);
  if (!rc) rc = batch_wait(b, &first);
  batch_free(b);
  return rc ? rc : first;
}

// --------------------------------------------------------- autotuning ---

extern "C" int lbdd_autotune(lbdd_solver* const* solvers, int m, int probe_rounds, void* stream) {
  (void)stream;
  if (!solvers || m < 1 || probe_rounds < 1) return LBDD_ERR_ARG;
  int dev = 0, sms = 0;
  int rc = check_device(&dev, &sms);
  if (rc) return rc;
  if (dev >= kMaxDevices) return LBDD_ERR_NODEV;
  // one representative per (cost width, k bucket): the instance with most units
  std::vector<int> rep(2 * kBuckets, -1);
  for (int i = 0; i < m; ++i) {
    if (!solvers[i]) return LBDD_ERR_ARG;
    const int key = wid(solvers[i]->elem) * kBuckets + bucket_of(solvers[i]->k);
    if (rep[key] < 0 || solvers[i]->n > solvers[rep[key]]->n) rep[key] = i;
  }
  for (int key = 0; key < 2 * kBuckets; ++key) {
    if (rep[key] < 0) continue;
    // a whole solve of a scaled-down copy (first probe_rounds units,
    // capacities scaled alike) passes through the filling and the overload
    // phases in proportion, unlike the first rounds of the instance itself
    lbdd_solver* tmp = nullptr;
    rc = clone_prefix(solvers[rep[key]], probe_rounds, &tmp);
    if (rc) return rc;
    double row[kNC] = {0, 0, 0, 0, 0};
    const int64_t rounds = tmp->n;
    for (int C = 1; C <= 16 && rc == LBDD_OK; C <<= 1) {
      if (!fits_k(tmp->k, tmp->elem, C)) continue;
      float ms = 0;
      rc = lbdd_reset(tmp);
      if (!rc) rc = solve_timed(tmp, 0, C, &ms);          // prologue only
      if (!rc) rc = solve_timed(tmp, rounds, C, &ms);
      if (!rc) row[cidx(C)] = ms * 1e6 / (double)rounds;
    }
    lbdd_destroy(tmp);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::memcpy(g_tune[dev].ns[key / kBuckets][key % kBuckets], row, sizeof(row));
  }
  return LBDD_OK;
}

extern "C" int lbdd_tune_get(int cm_dtype, int32_t k, int cluster_size, double* ns_per_round) {
  if (!ns_per_round || k < 1 || cluster_size < 1 || cluster_size > 16 ||
      (cluster_size & (cluster_size - 1)) != 0)
    return LBDD_ERR_ARG;
  if (cm_dtype != LBDD_CM_I16 && cm_dtype != LBDD_CM_I32) return LBDD_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();     // reported as LBDD_ERR_NODEV; leave no stale error
    return LBDD_ERR_NODEV;
  }
  if (dev >= kMaxDevices) return LBDD_ERR_NODEV;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  *ns_per_round = g_tune[dev].ns[cm_dtype == LBDD_CM_I16 ? 0 : 1][bucket_of(k)][cidx(cluster_size)];
  return LBDD_OK;
}

extern "C" int lbdd_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::memset(g_tune, 0, sizeof(g_tune));
  return LBDD_OK;
}
