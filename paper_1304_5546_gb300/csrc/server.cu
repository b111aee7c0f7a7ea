// Solve server (dg_server_* of the C ABI): continuous batching of wave
// propagation solves on one GPU.
//
// A worker thread owns a batch (dg_batch) and a stream.  Callers submit
// requests (an operator, a final time, an optional point source, initial
// fields) from any thread; the worker, in a loop:
//   1. completes requests whose results have reached host memory;
//   2. admits queued requests, oldest first, into the batch while their
//      order's pool has a free range (the memory budget is the pools'
//      capacity; a request that does not fit waits, later smaller ones may
//      pass it) and, with a work limit, while the running requests' nodal
//      values stay within it (there the queue is first come, first served);
//   3. advances every admitted request by a chunk of LSRK steps (the
//      smallest number of steps any of them has left, at most kChunk) with
//      one dg_batch_step, so requests that arrive while others run join at
//      the next chunk boundary and share its launches;
//   4. retires requests that reached their final time: their fields go to
//      host memory asynchronously (through pinned buffers), their pool
//      range is freed for the next admission.
// The host runs at most kAhead chunks ahead of the device.  Each request
// keeps its own time step (dg_solve's rule: ceil(T / dt_cfl) steps, landing
// on T) and its own source clock, so its result does not depend on what
// else is in the batch.  With DG_SERVER_SEQUENTIAL the worker admits a
// request only when none is running: plain one-at-a-time solves through the
// same code, the baseline continuous batching is measured against.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "staging.h"

using dgw::fail;

namespace {

constexpr int kChunk = 4;  // steps per dg_batch_step at most
constexpr int kAhead = 2;  // chunks the host may enqueue ahead of the device

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t id = 0;
  const dg_op* op = nullptr;
  double T = 0.0, dt = 0.0;
  int64_t nsteps = 0, done_steps = 0;
  bool has_src = false;
  dg_point_source src{};
  const void* q0 = nullptr;
  void* out = nullptr;
  int32_t slot = -1;
  int32_t state = DG_REQUEST_QUEUED;
  dg_status status = DG_OK;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0, t_retired = 0.0;
  size_t staging_idx = 0;  // pinned buffer holding the result on its way out
  bool staged = false;     // staging_idx is held for this request
  bool cancel = false;     // dg_server_cancel asked for it (under the server lock)
  cudaEvent_t out_ev = nullptr;
};

}  // namespace

struct dg_server {
  int device = 0;
  int flags = 0;
  dg_batch* batch = nullptr;
  cudaStream_t stream = nullptr;
  dgw::Staging out_staging;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work;  // submissions or stop
  std::condition_variable cv_done;  // a request completed
  bool stop = false;
  int64_t next_id = 1;
  std::deque<Request*> queue;                     // submitted, not admitted (worker pops)
  std::unordered_map<int64_t, Request*> requests;  // every request not yet released
  // worker-only state
  std::vector<Request*> running;
  std::vector<Request*> finishing;
  std::deque<cudaEvent_t> inflight;
  std::vector<cudaEvent_t> spare_events;
  int64_t completed = 0, failed = 0, cancelled = 0;
  std::atomic<int64_t> steps{0}, launches{0};
  std::atomic<int64_t> max_nodes{0};  // work limit (dg_server_set_work_limit); 0: none
};

namespace {

cudaEvent_t take_event(dg_server* s) {
  if (!s->spare_events.empty()) {
    cudaEvent_t e = s->spare_events.back();
    s->spare_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

void finish(dg_server* s, Request* r, int32_t state, dg_status status) {
  std::lock_guard<std::mutex> lock(s->mu);
  r->state = state;
  r->status = status;
  r->t_done = now_s();
  if (state == DG_REQUEST_DONE)
    ++s->completed;
  else if (state == DG_REQUEST_FAILED)
    ++s->failed;
  else
    ++s->cancelled;
  s->cv_done.notify_all();
}

// requests whose results reached host memory
void poll_finishing(dg_server* s) {
  for (size_t i = 0; i < s->finishing.size();) {
    Request* r = s->finishing[i];
    if (cudaEventQuery(r->out_ev) != cudaSuccess) {
      ++i;
      continue;
    }
    if (r->staged) {
      const int Np = r->op->Np;
      std::memcpy(r->out, s->out_staging.ptr(r->staging_idx),
                  3 * static_cast<size_t>(r->op->K) * Np * sizeof(float));
      s->out_staging.unhold(r->staging_idx);
      r->staged = false;
    }
    s->spare_events.push_back(r->out_ev);
    r->out_ev = nullptr;
    finish(s, r, DG_REQUEST_DONE, DG_OK);
    s->finishing[i] = s->finishing.back();
    s->finishing.pop_back();
  }
}

// queued requests, oldest first, while they fit
void admit(dg_server* s) {
  std::vector<Request*> cand;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    cand.assign(s->queue.begin(), s->queue.end());
  }
  const bool seq = (s->flags & DG_SERVER_SEQUENTIAL) != 0;
  const int64_t limit = s->max_nodes.load(std::memory_order_relaxed);
  int64_t nodes = 0;  // K * Np of the running requests
  for (const Request* r : s->running) nodes += r->op->K * r->op->Np;
  for (Request* r : cand) {
    bool cancelled = false;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (r->cancel) {
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
          if (*it == r) {
            s->queue.erase(it);
            break;
          }
        cancelled = true;
      }
    }
    if (cancelled) {
      finish(s, r, DG_REQUEST_CANCELLED, DG_OK);
      continue;
    }
    if (seq && (!s->running.empty() || !s->finishing.empty())) break;
    const int64_t r_nodes = r->op->K * r->op->Np;
    if (limit > 0 && !s->running.empty() && nodes + r_nodes > limit) break;
    int32_t slot = -1;
    dg_status st = dg_batch_add(s->batch, r->op, r->dt, r->has_src ? &r->src : nullptr, s->stream,
                                &slot);
    if (st == DG_ERR_OOM) {
      if (seq) break;
      continue;  // no room now; later requests may fit
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (*it == r) {
          s->queue.erase(it);
          break;
        }
    }
    if (st == DG_OK) {
      const int64_t stride = r->op->K * r->op->Np;
      st = dg_batch_set_fields(s->batch, slot, r->q0, stride, s->stream);
    }
    if (st != DG_OK) {
      if (slot >= 0) dg_batch_remove(s->batch, slot);
      finish(s, r, DG_REQUEST_FAILED, st);
      continue;
    }
    r->slot = slot;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      r->t_admit = now_s();
      r->state = DG_REQUEST_RUNNING;
    }
    s->running.push_back(r);
    nodes += r_nodes;
    if (seq) break;
  }
}

// running requests that were cancelled leave the batch, without results
void drop_cancelled(dg_server* s) {
  for (size_t i = 0; i < s->running.size();) {
    Request* r = s->running[i];
    bool cancel;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      cancel = r->cancel;
    }
    if (!cancel) {
      ++i;
      continue;
    }
    dg_batch_remove(s->batch, r->slot);
    s->running[i] = s->running.back();
    s->running.pop_back();
    finish(s, r, DG_REQUEST_CANCELLED, DG_OK);
  }
}

// requests at their final time: results out (through pinned memory), range freed
dg_status retire(dg_server* s) {
  for (size_t i = 0; i < s->running.size();) {
    Request* r = s->running[i];
    if (r->done_steps < r->nsteps) {
      ++i;
      continue;
    }
    dg_status st = DG_OK;
    if (r->out) {
      const int64_t n = r->op->K * r->op->Np;
      void* h = s->out_staging.get(3 * static_cast<size_t>(n) * sizeof(float), &r->staging_idx);
      if (h) {
        s->out_staging.hold(r->staging_idx);
        r->staged = true;
      }
      st = h ? dg_batch_get_fields(s->batch, r->slot, h, n, s->stream) : DG_ERR_OOM;
    }
    r->out_ev = take_event(s);
    if (st == DG_OK) {
      cudaError_t err = r->out ? s->out_staging.mark(r->staging_idx, s->stream)
                               : cudaEventRecord(r->out_ev, s->stream);
      if (r->out && err == cudaSuccess) err = cudaEventRecord(r->out_ev, s->stream);
      if (err != cudaSuccess) st = DG_ERR_CUDA;
    }
    dg_batch_remove(s->batch, r->slot);
    s->running[i] = s->running.back();
    s->running.pop_back();
    {
      std::lock_guard<std::mutex> lock(s->mu);
      r->t_retired = now_s();
    }
    if (st != DG_OK) {
      if (r->staged) s->out_staging.unhold(r->staging_idx);
      r->staged = false;
      s->spare_events.push_back(r->out_ev);
      r->out_ev = nullptr;
      finish(s, r, DG_REQUEST_FAILED, st);
      continue;
    }
    s->finishing.push_back(r);
  }
  return DG_OK;
}

void worker_loop(dg_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    poll_finishing(s);
    drop_cancelled(s);
    admit(s);
    if (!s->running.empty()) {
      if (static_cast<int>(s->inflight.size()) >= kAhead) {
        cudaEventSynchronize(s->inflight.front());
        s->spare_events.push_back(s->inflight.front());
        s->inflight.pop_front();
        continue;
      }
      int64_t k = kChunk;
      for (Request* r : s->running) k = std::min<int64_t>(k, r->nsteps - r->done_steps);
      if (k > 0) {
        const dg_status st = dg_batch_step(s->batch, static_cast<int32_t>(k), s->stream);
        if (st != DG_OK) {
          for (Request* r : s->running) {
            dg_batch_remove(s->batch, r->slot);
            finish(s, r, DG_REQUEST_FAILED, st);
          }
          s->running.clear();
          continue;
        }
        s->steps += k;
        s->launches.store(dg_batch_launch_count(s->batch));
        cudaEvent_t e = take_event(s);
        cudaEventRecord(e, s->stream);
        s->inflight.push_back(e);
        for (Request* r : s->running) r->done_steps += k;
      }
      retire(s);
      continue;
    }
    if (!s->finishing.empty()) {
      cudaEventSynchronize(s->finishing.front()->out_ev);
      continue;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->stop && s->queue.empty()) break;
    // a queued request that fits nowhere although nothing runs can never be
    // admitted: fail it rather than wait forever
    if (!s->queue.empty()) {
      lock.unlock();
      admit(s);
      if (s->running.empty()) {
        Request* r = nullptr;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          if (!s->queue.empty()) {
            r = s->queue.front();
            s->queue.pop_front();
          }
        }
        if (r) finish(s, r, DG_REQUEST_FAILED, DG_ERR_OOM);
      }
      continue;
    }
    s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty(); });
  }
  for (cudaEvent_t e : s->inflight) cudaEventDestroy(e);
  s->inflight.clear();
}

}  // namespace

// ============================================================ C ABI
extern "C" double dg_server_clock(void) { return now_s(); }

extern "C" dg_status dg_server_create(const int64_t* capacity, int32_t flags, dg_server** out) {
  dgw::clear_error();
  if (!capacity || !out) return fail(DG_ERR_ARG, "dg_server_create: NULL argument");
  if (flags & ~DG_SERVER_SEQUENTIAL)
    return fail(DG_ERR_ARG, "dg_server_create: unknown flags 0x%x", flags);
  dg_server* s = new (std::nothrow) dg_server;
  if (!s) return fail(DG_ERR_OOM, "dg_server_create: out of host memory");
  s->flags = flags;
  cudaError_t err = cudaGetDevice(&s->device);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (err != cudaSuccess) {
    delete s;
    return fail(DG_ERR_CUDA, "dg_server_create: %s", cudaGetErrorString(err));
  }
  const dg_status st = dg_batch_create(capacity, 0, &s->batch);
  if (st != DG_OK) {
    cudaStreamDestroy(s->stream);
    delete s;
    return st;
  }
  try {
    s->worker = std::thread(worker_loop, s);
  } catch (...) {
    dg_batch_destroy(s->batch);
    cudaStreamDestroy(s->stream);
    delete s;
    return fail(DG_ERR_OOM, "dg_server_create: cannot start the worker thread");
  }
  *out = s;
  return DG_OK;
}

extern "C" void dg_server_destroy(dg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  for (auto& kv : s->requests) {
    if (kv.second->out_ev) cudaEventDestroy(kv.second->out_ev);
    delete kv.second;
  }
  for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
  s->out_staging.release();
  dg_batch_destroy(s->batch);
  cudaStreamDestroy(s->stream);
  delete s;
}

extern "C" dg_status dg_server_submit(dg_server* s, const dg_op* op, double T,
                                      const dg_point_source* src, const void* q0, void* out,
                                      int64_t* request_id) {
  dgw::clear_error();
  if (!s || !op || !request_id) return fail(DG_ERR_ARG, "dg_server_submit: NULL argument");
  if (op->precision != DG_FP32)
    return fail(DG_ERR_ARG, "dg_server_submit: the server computes in FP32; use a DG_FP32 operator");
  if (!(T > 0.0) || !std::isfinite(T)) return fail(DG_ERR_ARG, "dg_server_submit: bad final time");
  Request* r = new (std::nothrow) Request;
  if (!r) return fail(DG_ERR_OOM, "dg_server_submit: out of host memory");
  // dg_solve's step rule with the CFL step of the operator
  const double dt_cfl = (2.0 / 3.0) * op->min_inradius_over_c * op->ref.lgl_gap;
  const double ns = std::ceil(T / dt_cfl - 1e-12);
  if (!(ns >= 1.0) || ns > 2147483647.0) {
    delete r;
    return fail(DG_ERR_ARG, "dg_server_submit: step count out of range");
  }
  r->op = op;
  r->T = T;
  r->nsteps = static_cast<int64_t>(ns);
  r->dt = T / static_cast<double>(r->nsteps);
  r->has_src = src != nullptr;
  if (src) r->src = *src;
  r->q0 = q0;
  r->out = out;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) {
      delete r;
      return fail(DG_ERR_ARG, "dg_server_submit: the server is stopping");
    }
    r->id = s->next_id++;
    s->requests[r->id] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_one();
  *request_id = r->id;
  return DG_OK;
}

namespace {

void fill_info(const Request* r, dg_request_info* info) {
  info->state = r->state;
  info->status = r->status;
  info->N = r->op->N;
  info->K = r->op->K;
  info->nsteps = r->nsteps;
  info->dt = r->dt;
  info->t_submit = r->t_submit;
  info->t_admit = r->t_admit;
  info->t_done = r->t_done;
  info->t_retired = r->t_retired;
}

}  // namespace

extern "C" dg_status dg_server_wait(dg_server* s, int64_t request_id, double timeout_s,
                                    dg_request_info* info) {
  dgw::clear_error();
  if (!s) return fail(DG_ERR_ARG, "dg_server_wait: NULL server");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end())
    return fail(DG_ERR_ARG, "dg_server_wait: unknown request %lld", static_cast<long long>(request_id));
  Request* r = it->second;
  auto done = [&] {
    return r->state == DG_REQUEST_DONE || r->state == DG_REQUEST_FAILED ||
           r->state == DG_REQUEST_CANCELLED;
  };
  if (timeout_s < 0)
    s->cv_done.wait(lock, done);
  else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), done))
    return fail(DG_ERR_TIMEOUT, "dg_server_wait: request %lld not done after %g s",
                static_cast<long long>(request_id), timeout_s);
  if (info) fill_info(r, info);
  return DG_OK;
}

extern "C" dg_status dg_server_info(dg_server* s, int64_t request_id, dg_request_info* info) {
  dgw::clear_error();
  if (!s || !info) return fail(DG_ERR_ARG, "dg_server_info: NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end())
    return fail(DG_ERR_ARG, "dg_server_info: unknown request %lld", static_cast<long long>(request_id));
  fill_info(it->second, info);
  return DG_OK;
}

extern "C" dg_status dg_server_release(dg_server* s, int64_t request_id) {
  dgw::clear_error();
  if (!s) return fail(DG_ERR_ARG, "dg_server_release: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end())
    return fail(DG_ERR_ARG, "dg_server_release: unknown request %lld", static_cast<long long>(request_id));
  Request* r = it->second;
  if (r->state != DG_REQUEST_DONE && r->state != DG_REQUEST_FAILED &&
      r->state != DG_REQUEST_CANCELLED)
    return fail(DG_ERR_ARG, "dg_server_release: request %lld has not finished",
                static_cast<long long>(request_id));
  s->requests.erase(it);
  delete r;
  return DG_OK;
}

extern "C" dg_status dg_server_cancel(dg_server* s, int64_t request_id) {
  dgw::clear_error();
  if (!s) return fail(DG_ERR_ARG, "dg_server_cancel: NULL server");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->requests.find(request_id);
    if (it == s->requests.end())
      return fail(DG_ERR_ARG, "dg_server_cancel: unknown request %lld",
                  static_cast<long long>(request_id));
    Request* r = it->second;
    if (r->state != DG_REQUEST_QUEUED && r->state != DG_REQUEST_RUNNING)
      return fail(DG_ERR_ARG, "dg_server_cancel: request %lld has already finished",
                  static_cast<long long>(request_id));
    r->cancel = true;
  }
  s->cv_work.notify_one();
  return DG_OK;
}

extern "C" dg_status dg_server_stats(dg_server* s, int64_t* completed, int64_t* failed,
                                     int64_t* steps, int64_t* launches) {
  dgw::clear_error();
  if (!s) return fail(DG_ERR_ARG, "dg_server_stats: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (completed) *completed = s->completed;
  if (failed) *failed = s->failed;
  if (steps) *steps = s->steps.load();
  if (launches) *launches = s->launches.load();
  return DG_OK;
}

extern "C" dg_status dg_server_set_work_limit(dg_server* server, int64_t max_nodes) {
  dgw::clear_error();
  if (!server) return fail(DG_ERR_ARG, "dg_server_set_work_limit: NULL server");
  if (max_nodes < 0)
    return fail(DG_ERR_ARG, "dg_server_set_work_limit: max_nodes = %lld < 0",
                static_cast<long long>(max_nodes));
  server->max_nodes.store(max_nodes, std::memory_order_relaxed);
  return DG_OK;
}
