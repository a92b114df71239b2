// Serving loop: continuous batching of independent simulations on one GPU.
//
// Requests (a problem handle, an initial BDF history, a number of steps) queue FIFO until the
// device-memory budget admits them; admitted requests get their state (BDF history, matrix,
// Krylov and preconditioner workspace) resident on the device and their own CUDA stream.
// A pool of host worker threads steps admitted simulations round-robin, one step at a time, so
// the kernels of different simulations overlap on the device; a finished simulation's result
// is copied out, its memory released, and waiting requests are admitted as memory frees up.
// Every step's latency (wall time of lfx_step) is recorded for p50/p99 reporting.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lfx_internal.h"

using namespace lfx;

namespace {

struct Request {
  int64_t ticket = 0;
  lfx_problem *pb = nullptr;
  int64_t V = 0;
  int sigma = 1;
  std::vector<double> u_hist, p_hist;
  double t0 = 0.0;
  int n_steps = 0, done_steps = 0;
  lfx_state *st = nullptr;
  cudaStream_t stream = nullptr;
  int64_t bytes = 0;
  bool admitted = false, finished = false;
  lfx_status status = LFX_OK;
  std::string error;
  std::vector<double> u_out, p_out;
  lfx_step_stats last{};
};

}  // namespace

struct lfx_server {
  int64_t budget = 0, used = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> waiting, ready;
  std::map<int64_t, std::unique_ptr<Request>> all;
  std::vector<std::thread> workers;
  std::vector<float> latency_ms;
  int64_t next_ticket = 1;
  int64_t admitted_total = 0, max_active = 0, active = 0;
  bool stop = false;
};

// Problem-side facts the estimate needs (defined in api.cu).
int64_t lfx_internal_state_bytes_estimate(const lfx_problem *pb, int64_t *V, int *sigma);

// Admission.  Under the lock, the waiting requests that fit the budget leave the queue in FIFO
// order with their bytes reserved; their states and streams are then created without the lock
// (state creation allocates and uploads, and cudaMalloc may synchronise the device), so workers
// keep stepping meanwhile; finally, under the lock again, each goes to the ready queue or, if its
// creation failed, finishes with the error and gives its bytes back (which may admit more).
// The caller's current device is restored before returning.
static void admit(lfx_server *sv) {
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  for (;;) {
    std::vector<Request *> take;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      while (!sv->waiting.empty()) {
        Request *r = sv->waiting.front();
        if (sv->used + r->bytes > sv->budget) break;
        sv->waiting.pop_front();
        sv->used += r->bytes;
        take.push_back(r);
      }
    }
    if (take.empty()) break;
    cudaSetDevice(sv->device);
    struct Made {
      lfx_state *st = nullptr;
      cudaStream_t stream = nullptr;
      lfx_status rc = LFX_OK;
      std::string err;
    };
    std::vector<Made> made(take.size());
    for (size_t i = 0; i < take.size(); ++i) {
      Request *r = take[i];
      Made &m = made[i];
      m.rc = lfx_state_create(r->pb, r->u_hist.data(), r->p_hist.data(), r->t0, &m.st);
      if (m.rc == LFX_OK) {
        if (cudaStreamCreateWithFlags(&m.stream, cudaStreamNonBlocking) == cudaSuccess)
          m.rc = lfx_set_stream(m.st, m.stream);
        else
          m.rc = LFX_ERR_CUDA;
      }
      if (m.rc != LFX_OK) {
        m.err = lfx_last_error();
        if (m.st) lfx_state_destroy(m.st);
        if (m.stream) cudaStreamDestroy(m.stream);
        m.st = nullptr;
        m.stream = nullptr;
      }
    }
    bool freed = false;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (size_t i = 0; i < take.size(); ++i) {
        Request *r = take[i];
        const Made &m = made[i];
        if (m.rc != LFX_OK) {
          r->status = m.rc;
          r->error = m.err;
          r->finished = true;
          sv->used -= r->bytes;
          freed = true;
          continue;
        }
        r->st = m.st;
        r->stream = m.stream;
        r->admitted = true;
        sv->admitted_total += 1;
        sv->active += 1;
        if (sv->active > sv->max_active) sv->max_active = sv->active;
        sv->ready.push_back(r);
      }
    }
    sv->cv.notify_all();
    if (!freed) break;
  }
  if (prev >= 0) cudaSetDevice(prev);
}

static void worker_loop(lfx_server *sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] { return sv->stop || !sv->ready.empty(); });
      if (sv->stop) return;
      r = sv->ready.front();
      sv->ready.pop_front();
    }
    lfx_step_stats stats{};
    const auto t0 = std::chrono::steady_clock::now();
    lfx_status rc = lfx_step(r->st, &stats);
    const auto t1 = std::chrono::steady_clock::now();
    const float ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
    std::string err = rc == LFX_OK ? std::string() : std::string(lfx_last_error());
    bool finish = false;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->latency_ms.push_back(ms);
      r->done_steps += 1;
      r->last = stats;
      if (rc != LFX_OK && rc != LFX_ERR_NOT_CONVERGED) {
        r->status = rc;
        r->error = err;
        finish = true;
      } else if (r->done_steps >= r->n_steps) {
        if (rc == LFX_ERR_NOT_CONVERGED) r->status = rc;
        finish = true;
      }
    }
    if (!finish) {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->ready.push_back(r);
      sv->cv.notify_one();
      continue;
    }
    // copy the result out and release the device memory (outside the lock)
    r->u_out.resize(3 * r->V);
    r->p_out.resize(r->V);
    lfx_status gr = lfx_state_get(r->st, r->u_out.data(), r->p_out.data());
    lfx_state_destroy(r->st);
    cudaStreamDestroy(r->stream);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (gr != LFX_OK && r->status == LFX_OK) r->status = gr;
      r->st = nullptr;
      r->stream = nullptr;
      r->finished = true;
      sv->used -= r->bytes;
      sv->active -= 1;
    }
    admit(sv);
    sv->cv.notify_all();
  }
}

extern "C" {

lfx_status lfx_server_create(int64_t hbm_budget_bytes, int32_t n_workers, lfx_server **out) {
  clear_error();
  if (!out || hbm_budget_bytes <= 0 || n_workers < 1 || n_workers > 64) {
    set_error("lfx_server_create: invalid argument");
    return LFX_ERR_INVALID_ARG;
  }
  std::unique_ptr<lfx_server> sv(new (std::nothrow) lfx_server);
  if (!sv) return LFX_ERR_OOM;
  sv->budget = hbm_budget_bytes;
  LFX_CUDA_TRY(cudaGetDevice(&sv->device));
  for (int i = 0; i < n_workers; ++i) sv->workers.emplace_back(worker_loop, sv.get());
  *out = sv.release();
  return LFX_OK;
}

lfx_status lfx_server_submit(lfx_server *sv, lfx_problem *pb, const double *u_hist, const double *p_hist,
                             double t0, int32_t n_steps, int64_t *ticket) {
  clear_error();
  if (!sv || !pb || !u_hist || !p_hist || !ticket || n_steps < 1) {
    set_error("lfx_server_submit: invalid argument");
    return LFX_ERR_INVALID_ARG;
  }
  std::unique_ptr<Request> r(new (std::nothrow) Request);
  if (!r) return LFX_ERR_OOM;
  r->pb = pb;
  r->bytes = lfx_internal_state_bytes_estimate(pb, &r->V, &r->sigma);
  if (r->bytes > sv->budget) {
    set_error("lfx_server_submit: request needs %lld bytes, budget is %lld", (long long)r->bytes,
              (long long)sv->budget);
    return LFX_ERR_BUDGET;
  }
  r->u_hist.assign(u_hist, u_hist + (size_t)r->sigma * 3 * r->V);
  r->p_hist.assign(p_hist, p_hist + (size_t)r->sigma * r->V);
  r->t0 = t0;
  r->n_steps = n_steps;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    *ticket = r->ticket;
    sv->waiting.push_back(r.get());
    sv->all[r->ticket] = std::move(r);
  }
  admit(sv);
  sv->cv.notify_all();
  return LFX_OK;
}

lfx_status lfx_server_poll(lfx_server *sv, int64_t ticket, int32_t *done, int32_t *steps_done,
                           lfx_step_stats *last) {
  if (!sv) {
    set_error("lfx_server_poll: NULL server");
    return LFX_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) {
    set_error("lfx_server_poll: unknown ticket %lld", (long long)ticket);
    return LFX_ERR_INVALID_ARG;
  }
  Request *r = it->second.get();
  if (done) *done = r->finished ? 1 : 0;
  if (steps_done) *steps_done = r->done_steps;
  if (last) *last = r->last;
  if (r->finished && r->status != LFX_OK && r->status != LFX_ERR_NOT_CONVERGED) {
    set_error("%s", r->error.c_str());
    return r->status;
  }
  return LFX_OK;
}

lfx_status lfx_server_result(lfx_server *sv, int64_t ticket, double *u, double *p) {
  if (!sv || !u || !p) {
    set_error("lfx_server_result: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end() || !it->second->finished) {
    set_error("lfx_server_result: ticket %lld unknown or not finished", (long long)ticket);
    return LFX_ERR_INVALID_ARG;
  }
  Request *r = it->second.get();
  const lfx_status status = r->status;
  if (!r->u_out.empty()) {
    memcpy(u, r->u_out.data(), sizeof(double) * r->u_out.size());
    memcpy(p, r->p_out.data(), sizeof(double) * r->p_out.size());
  }
  sv->all.erase(it);
  return status == LFX_ERR_NOT_CONVERGED ? LFX_OK : status;
}

lfx_status lfx_server_stats(lfx_server *sv, float *latency_ms, int64_t capacity, int64_t *n_latencies,
                            int64_t *used_bytes, int64_t *n_waiting, int64_t *max_active) {
  if (!sv) {
    set_error("lfx_server_stats: NULL server");
    return LFX_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  const int64_t n = (int64_t)sv->latency_ms.size();
  if (latency_ms && capacity > 0) memcpy(latency_ms, sv->latency_ms.data(), sizeof(float) * std::min(n, capacity));
  if (n_latencies) *n_latencies = n;
  if (used_bytes) *used_bytes = sv->used;
  if (n_waiting) *n_waiting = (int64_t)sv->waiting.size();
  if (max_active) *max_active = sv->max_active;
  return LFX_OK;
}

lfx_status lfx_batch_step(lfx_state *const *states, int32_t n, lfx_step_stats *stats) {
  clear_error();
  if (n < 0 || (n > 0 && !states)) {
    set_error("lfx_batch_step: invalid argument");
    return LFX_ERR_INVALID_ARG;
  }
  for (int32_t i = 0; i < n; ++i) {
    if (!states[i]) {
      set_error("lfx_batch_step: state %d is NULL", i);
      return LFX_ERR_INVALID_ARG;
    }
    for (int32_t j = 0; j < i; ++j)
      if (states[j] == states[i]) {
        set_error("lfx_batch_step: state %d appears twice", i);
        return LFX_ERR_INVALID_ARG;
      }
  }
  if (n == 0) return LFX_OK;
  int dev = 0;
  LFX_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<lfx_status> rc((size_t)n, LFX_OK);
  std::vector<std::string> err((size_t)n);
  // one host thread per state: each state's step runs on its own stream, so the kernels of the n
  // simulations overlap on the device while every thread waits only for its own solver's flags
  std::vector<std::thread> th;
  th.reserve((size_t)n);
  for (int32_t i = 0; i < n; ++i)
    th.emplace_back([&, i] {
      cudaSetDevice(dev);
      rc[i] = lfx_step(states[i], stats ? stats + i : nullptr);
      if (rc[i] != LFX_OK) err[i] = lfx_last_error();
    });
  for (auto &t : th) t.join();
  lfx_status out = LFX_OK;
  for (int32_t i = 0; i < n; ++i) {
    if (rc[i] == LFX_OK) continue;
    if (out == LFX_OK || (out == LFX_ERR_NOT_CONVERGED && rc[i] != LFX_ERR_NOT_CONVERGED)) {
      out = rc[i];
      set_error("lfx_batch_step: state %d: %s", i, err[i].c_str());
    }
  }
  return out;
}

void lfx_server_destroy(lfx_server *sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto &t : sv->workers) t.join();
  for (auto &kv : sv->all) {
    Request *r = kv.second.get();
    if (r->st) lfx_state_destroy(r->st);
    if (r->stream) cudaStreamDestroy(r->stream);
  }
  delete sv;
}

}  // extern "C"
