// chhs_serve.cu -- the request loop: continuous batching of independent CHHS
// runs on one GPU (declared in include/chhs.h, chhs_server_*).
//
// A worker thread owns the device work.  Submitted runs wait in a FIFO
// queue; a run is admitted as soon as an active slot is free and its
// hierarchy (chhs_workspace_bytes) fits in the device memory pool, which is
// allocated once and carved by a first-fit allocator, so admission and
// retirement never call cudaMalloc or cudaFree (cudaFree synchronises the
// whole device).  Every active run has its own stream and advances in slices
// of a few time steps (one CUDA-graph launch per step); runs therefore
// overlap on the GPU, and between slices finished runs are retired and
// waiting ones admitted -- a run never waits for the others to finish.
// Results (phi at the last step, status, V-cycles, timestamps) stay with the
// server until the caller releases them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/chhs.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device buffer, 256-byte granules.
class Pool {
 public:
  bool init(size_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return false;
    }
    free_[0] = bytes;
    size_ = bytes;
    return true;
  }
  ~Pool() {
    if (base_) cudaFree(base_);
  }
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes) {
        size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_[off] = bytes;
        return static_cast<char*>(base_) + off;
      }
    return nullptr;
  }
  void release(void* p) {
    size_t off = static_cast<char*>(p) - static_cast<char*>(base_);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t len = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && next->first == off + len) {  // merge with the following block
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {  // merge with the preceding block
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += len;
        return;
      }
    }
    free_[off] = len;
  }
  size_t in_use() const {
    size_t s = 0;
    for (auto& u : used_) s += u.second;
    return s;
  }

 private:
  void* base_ = nullptr;
  size_t size_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  std::map<size_t, size_t> used_;
};

struct Job {
  long long id = 0;
  chhs_request req{};
  std::vector<double> phi0, phi_prev;
  // live state
  chhs_t* run = nullptr;
  void* arena = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t slice_done = nullptr;
  int steps_left = 0;
  int vcycles = 0;
  // result
  int status = CHHS_OK;
  bool done = false;
  std::vector<double> phi_out;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct chhs_server {
  size_t budget = 0;
  int device = 0;
  int max_active = 1;
  int slice = 1;
  Pool pool;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job*> queue;           // submitted, not admitted
  std::vector<Job*> active;         // admitted, running
  std::map<long long, Job*> all;    // every job not yet released
  long long next_id = 1;
  int n_done = 0;
  bool stop = false;
  std::thread worker;

  // Admit waiting jobs while a slot is free and the next job fits (FIFO).
  void admit_locked(std::unique_lock<std::mutex>& lk) {
    while (!queue.empty() && (int)active.size() < max_active) {
      Job* j = queue.front();
      chhs_opts o;
      chhs_default_opts(&o);
      o.precision = j->req.precision;
      size_t need = chhs_workspace_bytes(j->req.dim, j->req.n, &o);
      void* arena = need ? pool.alloc(need) : nullptr;
      if (!arena) {
        if (active.empty() && need) {  // can never fit: fail it rather than block the queue
          queue.pop_front();
          j->t_admit = now_s();
          teardown(j);  // no device resources yet: frees the host copies only
          record_locked(j, CHHS_ERR_OOM);
          cv.notify_all();
          continue;
        }
        return;  // wait for memory to free up
      }
      queue.pop_front();
      lk.unlock();
      j->t_admit = now_s();
      j->arena = arena;
      chhs_status s = CHHS_OK;
      if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&j->slice_done, cudaEventDisableTiming) != cudaSuccess)
        s = CHHS_ERR_CUDA;
      if (s == CHHS_OK)
        s = chhs_create_ext(j->req.dim, j->req.n, j->req.h, j->req.eps, j->req.gamma, j->req.dt, &o, j->stream,
                            arena, need, &j->run);
      if (s == CHHS_OK)
        s = chhs_set_phi(j->run, j->phi0.data(), j->phi_prev.empty() ? nullptr : j->phi_prev.data(), 0);
      j->steps_left = j->req.nsteps;
      if (s == CHHS_OK) s = launch_slice(j);
      if (s != CHHS_OK) teardown(j);
      lk.lock();
      if (s != CHHS_OK) {
        record_locked(j, s);
        cv.notify_all();
        continue;
      }
      active.push_back(j);
    }
  }

  chhs_status launch_slice(Job* j) {
    int k = std::min(slice, j->steps_left);
    chhs_status s = chhs_step_async(j->run, k);
    if (s != CHHS_OK) return s;
    j->steps_left -= k;
    if (cudaEventRecord(j->slice_done, j->stream) != cudaSuccess) return CHHS_ERR_CUDA;
    return CHHS_OK;
  }

  // A finished job's device side: copy phi out, destroy its handle, stream
  // and event.  Called without the lock (only the worker thread, or the
  // destroying thread once the worker has stopped, touches a job's device
  // resources), so a long copy-out does not hold up the other runs' slices
  // or the callers of submit, stats and result.
  void teardown(Job* j) {
    if (j->run) {
      size_t n = (size_t)j->req.n[0] * j->req.n[1] * (j->req.dim == 3 ? j->req.n[2] : 1);
      j->phi_out.resize(n);
      chhs_get_phi(j->run, j->phi_out.data(), 0);
      chhs_destroy(j->run);
      j->run = nullptr;
    }
    if (j->slice_done) cudaEventDestroy(j->slice_done);
    if (j->stream) cudaStreamDestroy(j->stream);
    j->slice_done = nullptr;
    j->stream = nullptr;
    j->phi0.clear();
    j->phi0.shrink_to_fit();
    j->phi_prev.clear();
    j->phi_prev.shrink_to_fit();
  }

  // Return a torn-down job's memory to the pool and publish its result (lock held).
  void record_locked(Job* j, int status) {
    j->status = status;
    if (j->arena) pool.release(j->arena);
    j->arena = nullptr;
    j->done = true;
    j->t_done = now_s();
    ++n_done;
  }

  // Tear a job down and record it, dropping the lock for the device work.
  void finish(std::unique_lock<std::mutex>& lk, Job* j, int status) {
    lk.unlock();
    teardown(j);
    lk.lock();
    record_locked(j, status);
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      admit_locked(lk);
      bool progressed = false;
      for (size_t q = 0; q < active.size();) {
        Job* j = active[q];
        cudaError_t ready = cudaEventQuery(j->slice_done);
        if (ready == cudaErrorNotReady) {
          ++q;
          continue;
        }
        progressed = true;
        int v = 0;
        chhs_status s = ready == cudaSuccess ? chhs_wait(j->run, &v, nullptr) : CHHS_ERR_CUDA;
        j->vcycles += v;
        if (s == CHHS_OK && j->steps_left > 0) {
          s = launch_slice(j);
          if (s == CHHS_OK) {  // next slice in flight
            ++q;
            continue;
          }
        }
        // the last slice has completed, or a call failed: out of the active
        // set first, then torn down without the lock
        active.erase(active.begin() + q);
        finish(lk, j, s);
        cv.notify_all();
      }
      if (progressed) continue;
      if (active.empty() && queue.empty()) {
        cv.wait(lk, [&] { return stop || !queue.empty(); });
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
};

extern "C" {

chhs_status chhs_server_create(size_t pool_bytes, int max_active, int steps_per_slice, chhs_server_t** out) {
  if (!out || pool_bytes == 0 || max_active < 1 || steps_per_slice < 1) return CHHS_ERR_INVALID_ARG;
  *out = nullptr;
  chhs_server_t* sv = new (std::nothrow) chhs_server_t();
  if (!sv) return CHHS_ERR_OOM;
  sv->budget = pool_bytes;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return CHHS_ERR_CUDA;
  }
  sv->max_active = max_active;
  sv->slice = steps_per_slice;
  if (!sv->pool.init(pool_bytes)) {
    delete sv;
    return CHHS_ERR_OOM;
  }
  sv->worker = std::thread([sv] { sv->loop(); });
  *out = sv;
  return CHHS_OK;
}

chhs_status chhs_server_submit(chhs_server_t* sv, const chhs_request* req, long long* id_out) {
  if (!sv || !req || !id_out || !req->phi0 || req->nsteps < 0) return CHHS_ERR_INVALID_ARG;
  chhs_opts o;
  chhs_default_opts(&o);
  o.precision = req->precision;
  if (chhs_workspace_bytes(req->dim, req->n, &o) == 0 || !(req->h > 0) || !(req->eps > 0) || !(req->dt > 0) ||
      !(req->gamma >= 0))
    return CHHS_ERR_INVALID_ARG;
  Job* j = new (std::nothrow) Job();
  if (!j) return CHHS_ERR_OOM;
  j->req = *req;
  size_t n = (size_t)req->n[0] * req->n[1] * (req->dim == 3 ? req->n[2] : 1);
  j->phi0.assign(req->phi0, req->phi0 + n);
  if (req->phi_prev) j->phi_prev.assign(req->phi_prev, req->phi_prev + n);
  j->req.phi0 = nullptr;
  j->req.phi_prev = nullptr;
  j->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    j->id = sv->next_id++;
    sv->all[j->id] = j;
    sv->queue.push_back(j);
  }
  sv->cv.notify_all();
  *id_out = j->id;
  return CHHS_OK;
}

chhs_status chhs_server_stats(chhs_server_t* sv, int* queued, int* active, int* done, size_t* pool_in_use) {
  if (!sv) return CHHS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (queued) *queued = (int)sv->queue.size();
  if (active) *active = (int)sv->active.size();
  if (done) *done = sv->n_done;
  if (pool_in_use) *pool_in_use = sv->pool.in_use();
  return CHHS_OK;
}

chhs_status chhs_server_wait(chhs_server_t* sv, long long id, double timeout_s) {
  if (!sv || !(timeout_s >= 0)) return CHHS_ERR_INVALID_ARG;  // negative or NaN
  std::unique_lock<std::mutex> lk(sv->mu);
  if (sv->all.find(id) == sv->all.end()) return CHHS_ERR_INVALID_ARG;
  // Looked up again at every wake-up: another thread may release the run
  // (which needs it done) between the worker's notify and this thread
  // taking the lock back, and the Job is then gone.
  auto done = [&] {
    auto f = sv->all.find(id);
    return f == sv->all.end() || f->second->done;
  };
  // A limit past kNoLimitS (about 11.6 days; infinity included) waits without
  // one: converting a larger one to the clock's integer ticks could overflow.
  constexpr double kNoLimitS = 1e6;
  if (timeout_s > kNoLimitS) {
    sv->cv.wait(lk, done);
    return CHHS_OK;
  }
  bool ok = sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
  return ok ? CHHS_OK : CHHS_ERR_NOT_CONVERGED;
}

chhs_status chhs_server_result(chhs_server_t* sv, long long id, int* done, int* status, int* vcycles,
                               double* phi_out, double* times3) {
  if (!sv) return CHHS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(id);
  if (it == sv->all.end()) return CHHS_ERR_INVALID_ARG;
  Job* j = it->second;
  if (done) *done = j->done ? 1 : 0;
  if (!j->done) return CHHS_OK;
  if (status) *status = j->status;
  if (vcycles) *vcycles = j->vcycles;
  if (phi_out) {
    if (!j->phi_out.empty()) {
      memcpy(phi_out, j->phi_out.data(), sizeof(double) * j->phi_out.size());
    } else {  // refused before it held a state (admission): no phi to report
      size_t n = (size_t)j->req.n[0] * j->req.n[1] * (j->req.dim == 3 ? j->req.n[2] : 1);
      std::fill(phi_out, phi_out + n, std::numeric_limits<double>::quiet_NaN());
    }
  }
  if (times3) {
    times3[0] = j->t_submit;
    times3[1] = j->t_admit;
    times3[2] = j->t_done;
  }
  return CHHS_OK;
}

chhs_status chhs_server_release(chhs_server_t* sv, long long id) {
  if (!sv) return CHHS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(id);
  if (it == sv->all.end() || !it->second->done) return CHHS_ERR_INVALID_ARG;
  delete it->second;
  sv->all.erase(it);
  return CHHS_OK;
}

void chhs_server_destroy(chhs_server_t* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  std::lock_guard<std::mutex> lk(sv->mu);
  for (Job* j : sv->active) {
    cudaStreamSynchronize(j->stream);
    sv->teardown(j);
    sv->record_locked(j, CHHS_ERR_INVALID_ARG);
  }
  for (auto& kv : sv->all) delete kv.second;
  sv->all.clear();
  delete sv;
}

}  // extern "C"
