// Serving engine: a request loop that admits retrieval and join jobs by an
// HBM budget and overlaps them on the device (dpg_server_* in include/dpg.h).
//
// Continuous batching: a dispatcher thread owns `slots` execution slots, each
// a context (lent scratch, no device-wide allocation) and a CUDA stream.  Jobs
// queue in arrival order; the head job is admitted as soon as a slot is free
// and the memory held by running jobs and unreleased results plus the job's
// own footprint fits the budget; when the head does not fit, a later job
// that does may be admitted ahead of it, at most max_bypass times per head
// (backfilling with an aging bound).  Admitted jobs run concurrently on their
// slots' streams.  Device memory comes from a private stream-ordered pool
// (cudaMallocFromPoolAsync), so admitting or retiring a job never synchronizes
// the device.  A job's result stays allocated until dpg_server_release.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dpg_internal.h"
#include "dpg_launch.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  dpg_job spec{};
  Clock::time_point submitted, finished;
  size_t work_bytes = 0, out_bytes = 0;
  void* work = nullptr;
  void* out = nullptr;
  int slot = -1;
  cudaEvent_t done_ev = nullptr;
  dpg_status status = DPG_OK;
  bool complete = false;
  bool released = false;
  uint32_t bypassed = 0;  // jobs admitted ahead of this one while it headed the queue
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct dpg_server {
  int device = 0;
  size_t budget = 0;
  size_t held = 0;  // bytes of running jobs' work space and unreleased results
  cudaMemPool_t pool = nullptr;
  std::vector<dpg_ctx*> ctx;
  std::vector<cudaStream_t> stream;
  std::vector<uint64_t> running;  // ticket per slot, 0 = free
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  uint32_t max_bypass = 0;  // jobs that may be admitted ahead of a queue head that does not fit
};

namespace {

// Work-space and result bytes of a job, from the same layouts the kernels use.
int footprint(dpg_server& s, const dpg_job& j, size_t* work, size_t* out, size_t* scratch_part) {
  const dpg_ctx& c = *s.ctx[0];
  if (j.kind == DPG_JOB_RETRIEVE) {
    if (j.rec_bytes == 0 || j.rec_bytes > dpg::kMaxDpgRecBytes || j.n > 0x7fffffffULL || j.n_src > 0x7fffffffULL)
      return DPG_EINVAL;
    dpg::Retrieval r{static_cast<const uint8_t*>(j.src), j.n_src, (uint32_t)j.rec_bytes, j.n,
                     dpg::RidSpec{reinterpret_cast<const uint8_t*>(j.rids), 4}, nullptr, nullptr};
    *scratch_part = al256(dpg::retrieve_scratch_need(c, r));
    *work = *scratch_part;
    *out = al256(j.n * j.rec_bytes);
    return DPG_OK;
  }
  if (j.kind == DPG_JOB_JOIN) {
    if (j.fact_bytes < 4 || j.dim_bytes < 8 || j.n_fact > 0x7fffffffULL || j.n_dim > 0x7fffffffULL ||
        j.join_mode < 0 || j.join_mode > 2)
      return DPG_EINVAL;
    *out = al256(j.n_fact * (j.fact_bytes + j.dim_bytes));
    size_t scratch = 0, aux = 0;
    if (j.join_mode == DPG_JOIN_MOVE) {
      dpg::JoinSpec js{};
      dpg::Retrieval r{static_cast<const uint8_t*>(j.dim), j.n_dim, (uint32_t)j.dim_bytes, j.n_fact,
                       dpg::RidSpec{static_cast<const uint8_t*>(j.fact) + j.fk_off, (uint32_t)j.fact_bytes},
                       nullptr, nullptr};
      r.join = &js;
      scratch = dpg::retrieve_scratch_need(c, r);
    } else if (j.join_mode == DPG_JOIN_SORT) {
      dpg::JoinSpec js{};
      js.mode = 1;
      dpg::Retrieval r{static_cast<const uint8_t*>(j.fact), j.n_fact, (uint32_t)j.fact_bytes, j.n_fact,
                       dpg::RidSpec{nullptr, 8}, nullptr, nullptr};
      r.join = &js;
      scratch = dpg::retrieve_scratch_need(c, r);
      aux = 2 * al256(j.n_fact * 8) + dpg::sort_scan_bytes(j.n_fact);
    }
    *scratch_part = al256(scratch);
    *work = *scratch_part + al256(aux);
    return DPG_OK;
  }
  return DPG_EINVAL;
}

// Enqueue a job on its slot (dispatcher thread, lock held).
void launch(dpg_server& s, Job& job, int slot) {
  dpg_ctx& c = *s.ctx[slot];
  cudaStream_t st = s.stream[slot];
  size_t work = 0, out = 0, scratch_part = 0;
  footprint(s, job.spec, &work, &out, &scratch_part);
  job.slot = slot;
  job.status = DPG_OK;
  cudaError_t e = cudaSuccess;
  if (work) e = cudaMallocFromPoolAsync(&job.work, work, s.pool, st);
  if (e == cudaSuccess && out) e = cudaMallocFromPoolAsync(&job.out, out, s.pool, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    job.status = DPG_ENOMEM;
  }
  if (job.status == DPG_OK) {
    c.scratch = job.work;
    c.scratch_bytes = scratch_part;
    c.aux = static_cast<uint8_t*>(job.work) + scratch_part;
    c.aux_bytes = work - scratch_part;
    const dpg_job& j = job.spec;
    if (j.kind == DPG_JOB_RETRIEVE)
      job.status = dpg_retrieve(&c, j.src, j.n_src, j.rec_bytes, j.n, j.rids, job.out, st);
    else
      job.status = dpg_fk_join(&c, j.fact, j.n_fact, j.fact_bytes, j.fk_off, j.dim, j.n_dim, j.dim_bytes, j.pk_off,
                               job.out, j.join_mode, st);
  }
  cudaEventRecord(job.done_ev, st);
  s.running[slot] = job.ticket;
}

// Retire a finished job (lock held): its status, timing and work space.
void retire(dpg_server& s, Job& job) {
  const int slot = job.slot;
  dpg_ctx& c = *s.ctx[slot];
  const dpg_status async = dpg_sync(&c, s.stream[slot]);  // the stream is done: returns at once
  if (job.status == DPG_OK) job.status = async;
  if (job.work) {
    cudaFreeAsync(job.work, s.stream[slot]);
    job.work = nullptr;
  }
  s.held -= job.work_bytes;
  job.work_bytes = 0;
  c.scratch = nullptr;
  c.scratch_bytes = 0;
  c.aux = nullptr;
  c.aux_bytes = 0;
  job.finished = Clock::now();
  job.complete = true;
  s.running[slot] = 0;
}

void dispatch(dpg_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progress = false;
    for (size_t k = 0; k < s->running.size(); ++k) {
      if (!s->running[k]) continue;
      Job& job = *s->jobs[s->running[k]];
      if (cudaEventQuery(job.done_ev) == cudaSuccess) {
        retire(*s, job);
        progress = true;
      }
    }
    if (progress) s->cv_done.notify_all();
    while (!s->queue.empty()) {
      int slot = -1;
      for (size_t k = 0; k < s->running.size(); ++k)
        if (!s->running[k]) {
          slot = (int)k;
          break;
        }
      if (slot < 0) break;
      // the head if it fits; else the first queued job that fits, while the
      // head has been passed fewer than max_bypass times (then the queue
      // waits for memory in order, so the head is not starved)
      Job& head = *s->jobs[s->queue.front()];
      auto fits = [&](const Job& j) { return s->held + j.work_bytes + j.out_bytes <= s->budget; };
      size_t pick = s->queue.size();
      if (fits(head)) {
        pick = 0;
      } else if (head.bypassed < s->max_bypass) {
        for (size_t q = 1; q < s->queue.size(); ++q)
          if (fits(*s->jobs[s->queue[q]])) {
            pick = q;
            break;
          }
      }
      if (pick == s->queue.size()) break;  // wait for memory
      Job& job = *s->jobs[s->queue[pick]];
      if (pick) head.bypassed++;
      s->queue.erase(s->queue.begin() + (std::ptrdiff_t)pick);
      s->held += job.work_bytes + job.out_bytes;
      launch(*s, job, slot);
      progress = true;
    }
    if (s->stop && !s->queue.empty()) {  // shutting down: queued jobs are not run
      for (uint64_t t : s->queue) {
        Job& j = *s->jobs[t];
        j.status = DPG_EBUSY;
        j.finished = Clock::now();
        j.complete = true;
      }
      s->queue.clear();
      s->cv_done.notify_all();
    }
    bool busy = false;
    for (uint64_t t : s->running) busy |= t != 0;
    if (s->stop && !busy && s->queue.empty()) break;
    if (!progress) {
      if (busy) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      }
    }
  }
}

}  // namespace

extern "C" {

dpg_status dpg_server_create(dpg_server** out, int device, int slots, size_t budget_bytes) {
  if (!out || slots < 1 || slots > 64 || budget_bytes == 0) return DPG_EINVAL;
  *out = nullptr;
  std::unique_ptr<dpg_server> s(new dpg_server());
  s->device = device;
  s->budget = budget_bytes;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return DPG_EINVAL;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  dpg_status rc = DPG_OK;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) rc = DPG_ECUDA;
  if (rc == DPG_OK) {
    uint64_t keep = budget_bytes;  // keep freed memory in the pool for the next job
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  for (int k = 0; rc == DPG_OK && k < slots; ++k) {
    dpg_ctx* c = nullptr;
    rc = dpg_ctx_create(&c, device);
    if (rc != DPG_OK) break;
    c->external_memory = true;
    s->ctx.push_back(c);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      rc = DPG_ECUDA;
      break;
    }
    s->stream.push_back(st);
  }
  if (rc != DPG_OK) {
    cudaGetLastError();
    for (dpg_ctx* c : s->ctx) {
      c->external_memory = false;
      dpg_ctx_destroy(c);
    }
    for (cudaStream_t st : s->stream) cudaStreamDestroy(st);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
  }
  s->running.assign(slots, 0);
  // backfilling bound: by default four jobs per slot may pass a head that
  // waits for memory (DPG_SERVE_BYPASS overrides; 0 keeps strict arrival order)
  s->max_bypass = (uint32_t)std::max(0, dpg::env_int("DPG_SERVE_BYPASS", 4 * slots));
  s->worker = std::thread(dispatch, s.get());
  if (prev >= 0) cudaSetDevice(prev);
  *out = s.release();
  return DPG_OK;
}

dpg_status dpg_server_submit(dpg_server* s, const dpg_job* job, uint64_t* ticket) {
  if (!s || !job || !ticket) return DPG_EINVAL;
  std::unique_ptr<Job> j(new Job());
  j->spec = *job;
  size_t work = 0, out = 0, scratch_part = 0;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  int rc;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rc = footprint(*s, *job, &work, &out, &scratch_part);
  }
  if (rc == DPG_OK && work + out > s->budget) rc = DPG_EBUSY;  // could never be admitted
  if (rc == DPG_OK && cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming) != cudaSuccess) rc = DPG_ECUDA;
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  if (rc != DPG_OK) return (dpg_status)rc;
  j->work_bytes = work;
  j->out_bytes = out;
  j->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    j->ticket = s->next_ticket++;
    *ticket = j->ticket;
    s->queue.push_back(j->ticket);
    s->jobs.emplace(j->ticket, std::move(j));
  }
  s->cv_work.notify_one();
  return DPG_OK;
}

dpg_status dpg_server_result(dpg_server* s, uint64_t ticket, int wait, void** out, size_t* out_bytes,
                             double* latency_ms) {
  if (!s) return DPG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return DPG_EINVAL;
  Job& j = *it->second;
  if (!j.complete) {
    if (!wait) return DPG_EBUSY;
    s->cv_done.wait(lk, [&] { return j.complete; });
  }
  if (out) *out = j.out;
  if (out_bytes) *out_bytes = j.out_bytes;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j.finished - j.submitted).count();
  return j.status;
}

dpg_status dpg_server_release(dpg_server* s, uint64_t ticket) {
  if (!s) return DPG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end() || !it->second->complete) return DPG_EINVAL;
  Job& j = *it->second;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  if (j.out) cudaFreeAsync(j.out, s->stream[j.slot >= 0 ? j.slot : 0]);
  s->held -= j.out_bytes;
  if (j.done_ev) cudaEventDestroy(j.done_ev);
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  s->jobs.erase(it);
  s->cv_work.notify_one();
  return DPG_OK;
}

size_t dpg_server_held_bytes(dpg_server* s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  return s->held;
}

void dpg_server_destroy(dpg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (cudaStream_t st : s->stream) cudaStreamSynchronize(st);
  for (auto& kv : s->jobs) {
    Job& j = *kv.second;
    if (j.out) cudaFreeAsync(j.out, s->stream[0]);
    if (j.work) cudaFreeAsync(j.work, s->stream[0]);
    if (j.done_ev) cudaEventDestroy(j.done_ev);
  }
  for (cudaStream_t st : s->stream) cudaStreamSynchronize(st);
  for (dpg_ctx* c : s->ctx) {
    c->scratch = nullptr;
    c->aux = nullptr;
    c->external_memory = false;
    dpg_ctx_destroy(c);
  }
  for (cudaStream_t st : s->stream) cudaStreamDestroy(st);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
}

}  // extern "C"
