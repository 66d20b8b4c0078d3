// Continuous-batching request server (host side).
//
// Requests (a model, a batch of per-trajectory inputs in host memory, a seed and a
// trajectory-id base) are submitted without blocking.  A scheduler thread admits them in
// arrival order as soon as an in-flight slot and enough of the device-memory budget are
// free, copies their inputs into a device arena, launches the simulation on the slot's
// own stream and copies the results back; requests admitted while others are running
// execute concurrently on the GPU.  Completion is observed through CUDA events, after
// which the request's arena block and slot are reused by the next waiting request.
// Because every trajectory's random numbers are keyed by its id, a request's results do
// not depend on what else is in flight.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "matleap.h"
#include "ml_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kPending = 0, kRunning = 1, kDone = 2, kFailed = 3 };

// First-fit allocator over one device allocation, 256-byte granules.
class Arena {
 public:
  bool init(size_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return false;
    }
    size_ = bytes;
    free_[0] = bytes;
    return true;
  }
  void release() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  // Returns offset or SIZE_MAX.
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_ += bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void free(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* ptr(size_t off) const { return static_cast<char*>(base_) + off; }
  size_t size() const { return size_; }
  size_t used() const { return used_; }

 private:
  void* base_ = nullptr;
  size_t size_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

}  // namespace

struct ml_request {
  const ml_model* model = nullptr;
  int32_t N = 0, M = 0;
  int64_t n = 0;
  int32_t x0_per = 0, T_per = 0;
  uint64_t seed = 0, id_base = 0;
  // pinned host staging: inputs then outputs
  char* host = nullptr;
  size_t in_bytes = 0, out_bytes = 0, dev_bytes = 0;
  size_t off_theta = 0, off_x0 = 0, off_T = 0;  // offsets of inputs (0 theta bytes if none)
  bool has_theta = false;
  size_t dev_off = SIZE_MAX;
  int slot = -1;
  cudaEvent_t done = nullptr;
  std::atomic<int> state{kPending};
  int error = ML_OK;
  char message[256] = {0};
  Clock::time_point t_submit, t_admit, t_done;
};

struct ml_server {
  int device = 0;
  ml_sim_params params;
  Arena arena;
  int max_inflight = 0;
  std::vector<cudaStream_t> streams;
  std::vector<int> slot_free;
  std::deque<ml_request*> pending;
  std::vector<ml_request*> running;
  std::mutex mu;
  std::condition_variable cv;       // wakes the scheduler
  std::condition_variable done_cv;  // wakes waiters
  bool stop = false;
  std::thread worker;
  // statistics
  int64_t admitted = 0, completed = 0, trajectories = 0;
  size_t peak_bytes = 0;
  int peak_inflight = 0;
};

namespace {

size_t request_device_bytes(const ml_request& r) {
  const size_t n = (size_t)r.n, N = (size_t)r.N, M = (size_t)r.M;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t b = 0;
  b += r.has_theta ? up(n * M * 8) : 0;
  b += up((r.x0_per ? n : 1) * N * 8);
  b += up((r.T_per ? n : 1) * 8);
  b += up(n * N * 8) + up(n * M * 8) + up(n * M * 8) + up(n * 4) + up(n * 32);
  return b;
}

// Launches one admitted request on its slot's stream (scheduler thread, lock held).
void launch_request(ml_server* s, ml_request* r) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t n = (size_t)r->n, N = (size_t)r->N, M = (size_t)r->M;
  cudaStream_t st = s->streams[r->slot];
  char* d = s->arena.ptr(r->dev_off);
  char* p = d;
  double* d_theta = nullptr;
  if (r->has_theta) {
    d_theta = reinterpret_cast<double*>(p);
    p += up(n * M * 8);
  }
  int64_t* d_x0 = reinterpret_cast<int64_t*>(p);
  p += up((r->x0_per ? n : 1) * N * 8);
  double* d_T = reinterpret_cast<double*>(p);
  p += up((r->T_per ? n : 1) * 8);
  int64_t* d_X = reinterpret_cast<int64_t*>(p);
  p += up(n * N * 8);
  int64_t* d_r = reinterpret_cast<int64_t*>(p);
  p += up(n * M * 8);
  double* d_G = reinterpret_cast<double*>(p);
  p += up(n * M * 8);
  uint32_t* d_st = reinterpret_cast<uint32_t*>(p);
  p += up(n * 4);
  int64_t* d_c = reinterpret_cast<int64_t*>(p);
  const char* h = r->host;
  cudaError_t e = cudaSuccess;
  if (r->has_theta) e = cudaMemcpyAsync(d_theta, h + r->off_theta, n * M * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_x0, h + r->off_x0, (r->x0_per ? n : 1) * N * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_T, h + r->off_T, (r->T_per ? n : 1) * 8, cudaMemcpyHostToDevice, st);
  int rc = ML_OK;
  if (e == cudaSuccess) {
    rc = ml_simulate(r->model, r->n, d_theta, d_x0, r->x0_per, d_T, r->T_per, &s->params,
                     r->seed, r->id_base, d_X, d_r, d_G, d_st, d_c, st);
  }
  char* out = r->host + r->in_bytes;
  if (e == cudaSuccess && rc == ML_OK) {
    e = cudaMemcpyAsync(out, d_X, n * N * 8, cudaMemcpyDeviceToHost, st);
    out += n * N * 8;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_r, n * M * 8, cudaMemcpyDeviceToHost, st);
    out += n * M * 8;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_G, n * M * 8, cudaMemcpyDeviceToHost, st);
    out += n * M * 8;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_st, n * 4, cudaMemcpyDeviceToHost, st);
    out += n * 4;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_c, n * 32, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(r->done, st);
  }
  if (e != cudaSuccess || rc != ML_OK) {
    r->error = rc != ML_OK ? rc : ML_ERR_CUDA;
    std::snprintf(r->message, sizeof r->message, "%s",
                  rc != ML_OK ? ml_last_error() : cudaGetErrorString(e));
    cudaEventRecord(r->done, st);  // complete it in stream order so the slot is reusable
  }
}

void scheduler(ml_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // retire finished requests
    bool changed = false;
    for (size_t k = 0; k < s->running.size();) {
      ml_request* r = s->running[k];
      const cudaError_t q = cudaEventQuery(r->done);
      if (q == cudaErrorNotReady) {
        ++k;
        continue;
      }
      if (q != cudaSuccess && r->error == ML_OK) {
        r->error = ML_ERR_CUDA;
        std::snprintf(r->message, sizeof r->message, "%s", cudaGetErrorString(q));
      }
      r->t_done = Clock::now();
      s->arena.free(r->dev_off, r->dev_bytes);
      s->slot_free.push_back(r->slot);
      s->completed++;
      r->state.store(r->error == ML_OK ? kDone : kFailed);
      s->running[k] = s->running.back();
      s->running.pop_back();
      changed = true;
    }
    if (changed) s->done_cv.notify_all();
    if (s->stop && s->pending.empty() && s->running.empty()) break;
    // admit in arrival order while a slot and enough of the budget are free
    while (!s->stop && !s->pending.empty() && !s->slot_free.empty()) {
      ml_request* r = s->pending.front();
      const size_t off = s->arena.alloc(r->dev_bytes);
      if (off == SIZE_MAX) break;
      s->pending.pop_front();
      r->dev_off = off;
      r->slot = s->slot_free.back();
      s->slot_free.pop_back();
      r->t_admit = Clock::now();
      r->state.store(kRunning);
      s->running.push_back(r);
      s->admitted++;
      s->trajectories += r->n;
      if (s->arena.used() > s->peak_bytes) s->peak_bytes = s->arena.used();
      if ((int)s->running.size() > s->peak_inflight) s->peak_inflight = (int)s->running.size();
      launch_request(s, r);
    }
    if (s->stop && !s->pending.empty()) {
      // shutting down: cancel requests that were never admitted
      for (ml_request* r : s->pending) {
        r->error = ML_ERR_BUSY;
        std::snprintf(r->message, sizeof r->message, "server destroyed before admission");
        r->t_done = Clock::now();
        r->state.store(kFailed);
      }
      s->pending.clear();
      s->done_cv.notify_all();
    }
    // poll running work every 20 us, or sleep until a submit
    if (!s->running.empty())
      s->cv.wait_for(lk, std::chrono::microseconds(20));
    else if (!s->stop && s->pending.empty())
      s->cv.wait_for(lk, std::chrono::milliseconds(50));
    else if (!s->stop)
      s->cv.wait_for(lk, std::chrono::microseconds(20));
  }
}

int set_err(int code, const char* msg) { return mlk::set_error(code, msg); }

}  // namespace

extern "C" {

int ml_server_create(size_t hbm_budget_bytes, int32_t max_inflight, const ml_sim_params* p,
                     ml_server** out) {
  if (!out) return set_err(ML_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes < (1u << 20)) return set_err(ML_ERR_ARG, "budget below 1 MiB");
  if (max_inflight < 1 || max_inflight > 64) return set_err(ML_ERR_ARG, "max_inflight must be in [1, 64]");
  ml_server* s = new (std::nothrow) ml_server;
  if (!s) return set_err(ML_ERR_OOM, "host allocation failed");
  if (p) s->params = *p;
  else ml_default_params(&s->params);
  s->params.use_graph = 0;  // concurrent launches: no shared graph executable
  s->params.queue_order = nullptr;  // requests differ in size: no shared order
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return set_err(ML_ERR_CUDA, "no CUDA device");
  }
  if (!s->arena.init(hbm_budget_bytes)) {
    delete s;
    return set_err(ML_ERR_OOM, "cannot reserve the device-memory budget");
  }
  s->max_inflight = max_inflight;
  for (int k = 0; k < max_inflight; ++k) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      s->arena.release();
      delete s;
      return set_err(ML_ERR_CUDA, "stream creation failed");
    }
    s->streams.push_back(st);
    s->slot_free.push_back(max_inflight - 1 - k);
  }
  s->worker = std::thread(scheduler, s);
  *out = s;
  return ML_OK;
}

int ml_server_submit(ml_server* s, const ml_model* model, int64_t n_traj, const double* theta,
                     const int64_t* x0, int32_t x0_per_traj, const double* T, int32_t T_per_traj,
                     uint64_t seed, uint64_t traj_id_base, ml_request** out) {
  if (!s || !model || !out || !x0 || !T) return set_err(ML_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (n_traj < 1) return set_err(ML_ERR_ARG, "n_traj must be >= 1");
  if (traj_id_base > 0xffffffffULL || (uint64_t)n_traj > 0x100000000ULL - traj_id_base)
    return set_err(ML_ERR_ARG, "trajectory ids must stay below 2^32");
  const int N = ml_model_num_species(model), M = ml_model_num_reactions(model);
  if (N < 1 || M < 1) return set_err(ML_ERR_ARG, "bad model");
  ml_request* r = new (std::nothrow) ml_request;
  if (!r) return set_err(ML_ERR_OOM, "host allocation failed");
  r->model = model;
  r->N = N;
  r->M = M;
  r->n = n_traj;
  r->x0_per = x0_per_traj ? 1 : 0;
  r->T_per = T_per_traj ? 1 : 0;
  r->seed = seed;
  r->id_base = traj_id_base;
  r->has_theta = theta != nullptr;
  const size_t n = (size_t)n_traj;
  const size_t b_theta = r->has_theta ? n * M * 8 : 0;
  const size_t b_x0 = (r->x0_per ? n : 1) * N * 8, b_T = (r->T_per ? n : 1) * 8;
  r->off_theta = 0;
  r->off_x0 = b_theta;
  r->off_T = b_theta + b_x0;
  r->in_bytes = (b_theta + b_x0 + b_T + 15) / 16 * 16;
  r->out_bytes = n * ((size_t)N * 8 + (size_t)M * 16 + 4 + 32);
  r->dev_bytes = request_device_bytes(*r);
  if (r->dev_bytes > s->arena.size()) {
    delete r;
    return set_err(ML_ERR_BUSY, "request needs more device memory than the whole budget");
  }
  void* h = nullptr;
  if (cudaHostAlloc(&h, r->in_bytes + r->out_bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    delete r;
    return set_err(ML_ERR_OOM, "pinned host staging allocation failed");
  }
  r->host = static_cast<char*>(h);
  if (b_theta) std::memcpy(r->host + r->off_theta, theta, b_theta);
  std::memcpy(r->host + r->off_x0, x0, b_x0);
  std::memcpy(r->host + r->off_T, T, b_T);
  if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(h);
    delete r;
    return set_err(ML_ERR_CUDA, "event creation failed");
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      cudaEventDestroy(r->done);
      cudaFreeHost(h);
      delete r;
      return set_err(ML_ERR_BUSY, "server is shutting down");
    }
    s->pending.push_back(r);
  }
  s->cv.notify_one();
  *out = r;
  return ML_OK;
}

int ml_request_wait(ml_server* s, ml_request* r, int32_t timeout_ms) {
  if (!s || !r) return set_err(ML_ERR_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return r->state.load() >= kDone; };
  if (timeout_ms < 0) s->done_cv.wait(lk, ready);
  else if (!s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return set_err(ML_ERR_TIMEOUT, "request not finished within the timeout");
  if (r->state.load() == kFailed) return set_err(r->error, r->message);
  return ML_OK;
}

int ml_request_result(const ml_request* r, int64_t* X, int64_t* rr, double* G, uint32_t* status,
                      int64_t* counters, double* latency_s, double* queue_s) {
  if (!r) return set_err(ML_ERR_ARG, "NULL request");
  if (r->state.load() != kDone) return set_err(ML_ERR_BUSY, "request not finished");
  const size_t n = (size_t)r->n, N = (size_t)r->N, M = (size_t)r->M;
  const char* o = r->host + r->in_bytes;
  if (X) std::memcpy(X, o, n * N * 8);
  o += n * N * 8;
  if (rr) std::memcpy(rr, o, n * M * 8);
  o += n * M * 8;
  if (G) std::memcpy(G, o, n * M * 8);
  o += n * M * 8;
  if (status) std::memcpy(status, o, n * 4);
  o += n * 4;
  if (counters) std::memcpy(counters, o, n * 32);
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  if (queue_s) *queue_s = std::chrono::duration<double>(r->t_admit - r->t_submit).count();
  return ML_OK;
}

int ml_request_free(ml_server* s, ml_request* r) {
  if (!r) return ML_OK;
  if (s) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->state.load() < kDone) return set_err(ML_ERR_BUSY, "request still pending or running");
  }
  if (r->done) cudaEventDestroy(r->done);
  if (r->host) cudaFreeHost(r->host);
  delete r;
  return ML_OK;
}

int ml_server_stats(ml_server* s, int64_t* admitted, int64_t* completed, int64_t* trajectories,
                    size_t* peak_bytes, int32_t* peak_inflight) {
  if (!s) return set_err(ML_ERR_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (admitted) *admitted = s->admitted;
  if (completed) *completed = s->completed;
  if (trajectories) *trajectories = s->trajectories;
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  if (peak_inflight) *peak_inflight = s->peak_inflight;
  return ML_OK;
}

int ml_server_destroy(ml_server* s) {
  if (!s) return ML_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  s->arena.release();
  delete s;
  return ML_OK;
}

}  // extern "C"
