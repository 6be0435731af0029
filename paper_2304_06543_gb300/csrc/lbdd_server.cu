// Request server: continuous batching of LBDD solves on one GPU.
//
// Requests (an instance plus a host buffer for its allotment) are queued by
// lbdd_server_submit from any thread.  Three threads own all device work:
//
//  * admission takes queued requests in arrival order while the server's
//    device-memory budget and active-slot limit allow, and creates their
//    solvers (stream-ordered allocation and the host-to-device copy of CM,
//    which overlap the running pass);
//  * retirement copies a finished request's allotment and objective back,
//    frees its solver and releases its budget, on a stream of its own;
//  * the pass engine repeatedly runs one time-sliced pass over every active
//    request: a batch plan (cluster size per request, SM shares per group in
//    proportion to remaining work, shortest remaining work first inside a
//    group) and the persistent launches of lbdd_batch.cu with a quantum,
//    after which every cluster stops at its next quantum check.  A request
//    that made no progress in kAgePasses passes in a row (its group had
//    fewer clusters than instances and shorter ones kept them) moves to the
//    front of its group until it runs again, so no request waits without
//    bound.  Solver state stays on the device between passes, so a request
//    resumes exactly where it stopped; requests admitted during a pass join
//    the next one.
//
// A request's result does not depend on what it shares the GPU with: each
// solve is a deterministic function of its own instance (canonical
// tie-breaking), and a pass boundary only splits its rounds between
// launches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lbdd_internal.h"

using namespace lbdd;

namespace lbdd {
int batch_alloc(lbdd_batch** out, int capacity, uint64_t quantum_ns, void* stream);
int batch_set(lbdd_batch* b, lbdd_solver* const* solvers, const int64_t* rem, int m,
              int cluster_size, int max_clusters, bool shortest_first, const uint8_t* first);
int batch_launch(lbdd_batch* b, int64_t max_rounds);
int batch_wait(lbdd_batch* b, int* first_rc);
int batch_launches(const lbdd_batch* b);
int64_t batch_rounds(const lbdd_batch* b, int i);
int64_t batch_status(const lbdd_batch* b, int i);
void batch_destroy(lbdd_batch* b);
}  // namespace lbdd

namespace {

enum State { QUEUED = 0, ACTIVE = 1, DONE = 2, FAILED = 3 };

// Passes without progress after which a request goes first in its group.
constexpr int kAgePasses = 8;

struct Request {
  int64_t id = 0;
  int32_t n = 0, k = 0;
  const void* cm = nullptr;
  int dtype = LBDD_CM_I32;
  int cm_is_device = 0;
  std::vector<int32_t> cap, pen;
  int32_t* assign_out = nullptr;
  size_t footprint = 0;
  lbdd_solver* solver = nullptr;
  int64_t rounds = 0;
  int stalled = 0;        // passes in a row without progress
  int state = QUEUED;
  int status = LBDD_OK;
  int64_t objective = 0;
  int64_t t_submit = 0, t_admit = -1, t_done = -1;
};

int64_t now_ns(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
      .count();
}

}  // namespace

struct lbdd_server {
  lbdd_server_config cfg{};
  int dev = 0, sms = 0;
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_admit;   // admission: new submissions or freed budget
  std::condition_variable cv_retire;  // retirement: finished requests
  std::condition_variable cv_engine;  // engine: newly admitted requests
  std::condition_variable cv_done;    // pollers
  std::deque<Request*> queue;         // submitted, not admitted
  std::vector<Request*> ready;        // admitted, waiting for the next pass
  std::vector<Request*> finished;     // out of the pass, waiting to be retired
  std::unordered_map<int64_t, Request*> all;
  int64_t next_id = 1;
  size_t bytes = 0;                   // budget held by admitted requests
  int held = 0;                       // admitted and not yet retired
  bool stop = false;

  // counters (under mu)
  int64_t passes = 0, admitted = 0, completed = 0, failed = 0, launches = 0;
  size_t peak_bytes = 0;
  int64_t busy_ns = 0;                // time with a pass in flight
  int peak_active = 0;

  std::thread admit, retire, engine;
  cudaStream_t run_st = nullptr, admit_st = nullptr, retire_st = nullptr;
  lbdd_batch* batch = nullptr;
};

// Device bytes a request may hold: int32 input is narrowed to int16 when
// every cost fits, and both copies exist while the narrow one is made.
static size_t request_footprint(int32_t n, int32_t k, int dtype) {
  return solver_footprint(n, k, dtype == LBDD_CM_I16 ? 2 : 4, 2);
}

static void finish(lbdd_server* S, Request* r, int state, int status) {
  // caller holds S->mu
  r->state = state;
  r->status = status;
  r->t_done = now_ns(S->t0);
  if (state == DONE) S->completed++;
  else S->failed++;
}

// Retires finished requests: result copies on their own stream, so that a
// large admission copy in flight never delays them.
static void retire_loop(lbdd_server* S) {
  cudaSetDevice(S->dev);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    if (S->finished.empty()) {
      if (S->stop) break;
      S->cv_retire.wait(lk);
      continue;
    }
    std::vector<Request*> fin;
    fin.swap(S->finished);
    lk.unlock();
    for (Request* r : fin) {
      r->solver->st = S->retire_st;
      int rc = r->status;
      int64_t obj = 0;
      if (rc == LBDD_OK) rc = lbdd_assignment(r->solver, r->assign_out, 0);
      if (rc == LBDD_OK) rc = lbdd_objective(r->solver, &obj);
      lbdd_destroy(r->solver);
      lk.lock();
      r->solver = nullptr;
      r->objective = obj;
      S->bytes -= r->footprint;
      S->held--;
      finish(S, r, rc == LBDD_OK ? DONE : FAILED, rc);
      S->cv_admit.notify_all();
      S->cv_done.notify_all();
      lk.unlock();
    }
    lk.lock();
  }
}

// Admits queued requests in arrival order while budget and slots allow.
static void admit_loop(lbdd_server* S) {
  cudaSetDevice(S->dev);
  std::unique_lock<std::mutex> lk(S->mu);
  const int max_active = S->cfg.max_active > 0 ? S->cfg.max_active : S->sms;
  for (;;) {
    if (S->stop) break;
    Request* r = nullptr;
    if (!S->queue.empty()) {
      Request* h = S->queue.front();
      if (h->footprint > S->cfg.budget_bytes) {
        S->queue.pop_front();
        finish(S, h, FAILED, LBDD_ERR_BUDGET);
        S->cv_done.notify_all();
        continue;
      }
      if (S->held < max_active && S->bytes + h->footprint <= S->cfg.budget_bytes) {
        S->queue.pop_front();
        S->bytes += h->footprint;
        S->held++;
        S->peak_bytes = std::max(S->peak_bytes, S->bytes);
        r = h;
      }
    }
    if (!r) {
      S->cv_admit.wait(lk);
      continue;
    }
    lk.unlock();
    lbdd_solver* s = nullptr;
    const int rc = lbdd_create(&s, r->n, r->k, r->cm, r->dtype, r->cm_is_device, r->cap.data(),
                               r->pen.data(), S->admit_st);
    lk.lock();
    if (rc) {
      S->bytes -= r->footprint;
      S->held--;
      finish(S, r, FAILED, rc);
      S->cv_done.notify_all();
      continue;
    }
    r->solver = s;
    r->state = ACTIVE;
    r->t_admit = now_ns(S->t0);
    S->admitted++;
    S->ready.push_back(r);
    S->cv_engine.notify_all();
  }
}

static void engine_loop(lbdd_server* S) {
  cudaSetDevice(S->dev);
  std::vector<Request*> active;
  std::vector<lbdd_solver*> v;
  std::vector<int64_t> rem;
  std::vector<uint8_t> aged;
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    if (S->stop) break;   // unfinished requests are released by lbdd_server_destroy
    for (Request* r : S->ready) active.push_back(r);
    S->ready.clear();
    if (active.empty()) {
      S->cv_engine.wait(lk);
      continue;
    }
    S->peak_active = std::max(S->peak_active, (int)active.size());
    lk.unlock();
    v.clear();
    rem.clear();
    aged.clear();
    for (Request* r : active) {
      v.push_back(r->solver);
      rem.push_back(r->n - r->rounds);
      aged.push_back(r->stalled >= kAgePasses ? 1 : 0);
    }
    const int64_t t_a = now_ns(S->t0);
    int rc = batch_set(S->batch, v.data(), rem.data(), (int)v.size(), S->cfg.cluster_size, 0, true,
                       aged.data());
    if (!rc) rc = batch_launch(S->batch, -1);
    int first = LBDD_OK;
    if (!rc) rc = batch_wait(S->batch, &first);
    const int64_t t_b = now_ns(S->t0);
    lk.lock();
    S->passes++;
    if (!rc) S->launches += batch_launches(S->batch);
    S->busy_ns += t_b - t_a;
    std::vector<Request*> keep;
    for (size_t i = 0; i < active.size(); ++i) {
      Request* r = active[i];
      int st = rc;
      if (!rc) {
        const int64_t before = r->rounds;
        r->rounds = batch_rounds(S->batch, (int)i);
        r->stalled = r->rounds > before ? 0 : r->stalled + 1;
        st = status_to_rc(batch_status(S->batch, (int)i));
      }
      if (st != LBDD_OK || r->rounds >= r->n) {
        r->status = st;
        S->finished.push_back(r);
      } else {
        keep.push_back(r);
      }
    }
    active.swap(keep);
    if (!S->finished.empty()) S->cv_retire.notify_all();
  }
}

extern "C" int lbdd_server_create(lbdd_server** out, const lbdd_server_config* cfg) {
  if (!out || !cfg) return LBDD_ERR_ARG;
  *out = nullptr;
  if (cfg->budget_bytes == 0 || cfg->max_active < 0 || cfg->quantum_us < 0 ||
      cfg->cluster_size < 0 || cfg->cluster_size > 16 ||
      (cfg->cluster_size & (cfg->cluster_size - 1)) != 0)
    return LBDD_ERR_ARG;
  lbdd_server* S = new (std::nothrow) lbdd_server();
  if (!S) return LBDD_ERR_OOM;
  S->cfg = *cfg;
  if (S->cfg.quantum_us == 0) S->cfg.quantum_us = 20000;
  S->t0 = std::chrono::steady_clock::now();
  int rc = check_device(&S->dev, &S->sms);
  if (rc) { delete S; return rc; }
  cudaError_t e = cudaSuccess;
  cudaStream_t* sts[3] = {&S->run_st, &S->admit_st, &S->retire_st};
  for (auto* p : sts)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(p, cudaStreamNonBlocking);
  const int cap = S->cfg.max_active > 0 ? S->cfg.max_active : S->sms;
  rc = e ? cuda_fail(e, "server streams")
         : batch_alloc(&S->batch, cap, (uint64_t)S->cfg.quantum_us * 1000, S->run_st);
  if (rc) {
    for (auto* p : sts)
      if (*p) cudaStreamDestroy(*p);
    delete S;
    return rc;
  }
  S->admit = std::thread(admit_loop, S);
  S->retire = std::thread(retire_loop, S);
  S->engine = std::thread(engine_loop, S);
  *out = S;
  return LBDD_OK;
}

extern "C" int lbdd_server_submit(lbdd_server* S, int32_t n, int32_t k, const void* cm,
                                  int cm_dtype, const int32_t* cap, const int32_t* pen,
                                  int32_t* assign_out, int64_t* ticket) {
  return lbdd_server_submit_ex(S, n, k, cm, cm_dtype, 0, cap, pen, assign_out, ticket);
}

extern "C" int lbdd_server_submit_ex(lbdd_server* S, int32_t n, int32_t k, const void* cm,
                                     int cm_dtype, int cm_is_device, const int32_t* cap,
                                     const int32_t* pen, int32_t* assign_out, int64_t* ticket) {
  if (!S || !ticket || n < 1 || k < 1 || k > lbdd_max_centers() || !cm || !cap || !pen ||
      !assign_out)
    return LBDD_ERR_ARG;
  if (cm_dtype != LBDD_CM_I32 && cm_dtype != LBDD_CM_I16) return LBDD_ERR_ARG;
  if (cm_is_device != 0 && cm_is_device != 1) return LBDD_ERR_ARG;
  for (int32_t i = 0; i < k; ++i)
    if (cap[i] < 1 || pen[i] < 1) return LBDD_ERR_ARG;
  Request* r = new (std::nothrow) Request();
  if (!r) return LBDD_ERR_OOM;
  r->n = n;
  r->k = k;
  r->cm = cm;
  r->dtype = cm_dtype;
  r->cm_is_device = cm_is_device;
  r->cap.assign(cap, cap + k);
  r->pen.assign(pen, pen + k);
  r->assign_out = assign_out;
  r->footprint = request_footprint(n, k, cm_dtype);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) { delete r; return LBDD_ERR_STATE; }
  r->id = S->next_id++;
  r->t_submit = now_ns(S->t0);
  S->all[r->id] = r;
  S->queue.push_back(r);
  *ticket = r->id;
  S->cv_admit.notify_all();
  return LBDD_OK;
}

extern "C" int lbdd_server_poll(lbdd_server* S, int64_t ticket, int64_t timeout_ms,
                                lbdd_request_info* out) {
  if (!S || !out) return LBDD_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return LBDD_ERR_ARG;
  Request* r = it->second;
  auto done = [&] { return r->state == DONE || r->state == FAILED; };
  if (!done() && timeout_ms != 0) {
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
  }
  out->state = r->state;
  out->status = r->status;
  out->objective = r->objective;
  out->rounds = r->rounds;
  out->submit_ns = r->t_submit;
  out->admit_ns = r->t_admit;
  out->done_ns = r->t_done;
  return done() ? LBDD_OK : LBDD_ERR_TIMEOUT;
}

extern "C" int lbdd_server_release(lbdd_server* S, int64_t ticket) {
  if (!S) return LBDD_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return LBDD_ERR_ARG;
  if (it->second->state != DONE && it->second->state != FAILED) return LBDD_ERR_STATE;
  delete it->second;
  S->all.erase(it);
  return LBDD_OK;
}

extern "C" int lbdd_server_get_stats(lbdd_server* S, lbdd_server_stats* out) {
  if (!S || !out) return LBDD_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  out->passes = S->passes;
  out->admitted = S->admitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = (int64_t)S->queue.size();
  out->bytes_in_use = (int64_t)S->bytes;
  out->peak_bytes = (int64_t)S->peak_bytes;
  out->busy_ns = S->busy_ns;
  out->uptime_ns = now_ns(S->t0);
  out->peak_active = S->peak_active;
  out->launches = S->launches;
  return LBDD_OK;
}

extern "C" void lbdd_server_destroy(lbdd_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    // queued requests are dropped; active ones finish their current pass
    for (Request* r : S->queue) finish(S, r, FAILED, LBDD_ERR_STATE);
    S->queue.clear();
    S->cv_admit.notify_all();
    S->cv_retire.notify_all();
    S->cv_engine.notify_all();
    S->cv_done.notify_all();
  }
  S->engine.join();
  S->admit.join();
  S->retire.join();
  // nothing runs on the device any more: release what is left
  for (auto& kv : S->all) {
    if (kv.second->solver) lbdd_destroy(kv.second->solver);
    delete kv.second;
  }
  batch_destroy(S->batch);
  cudaStreamDestroy(S->run_st);
  cudaStreamDestroy(S->admit_st);
  cudaStreamDestroy(S->retire_st);
  delete S;
}
