// Native request loop for serving rollouts with continuous batching over a job pool
// (mg_server_*).
//
// Requests are submitted as job specs and wait in a FIFO queue.  Each poll runs one round of the
// loop: admit queued jobs in order while the trajectory budget and a free arena range allow
// (each job's trajectory record is a stream-ordered allocation on the pool's stream, from a
// memory pool of the server's own that keeps freed memory for the next jobs), issue one tick of
// the pool (every running job advances min(k, horizon - done) sub-steps in one launch), record an
// event after it, and hand back the jobs whose last tick has completed.  At most max_inflight
// ticks stay queued beyond the oldest incomplete one: a poll that would exceed that waits for the
// oldest, spinning on the event (never longer than wait_timeout_s), so the host stays a bounded
// distance ahead of the device and notices a finished job within microseconds.  Only pool ABI
// calls touch the pool.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <deque>
#include <thread>
#include <vector>

#include "mg_internal.h"

using namespace mg;

namespace {

enum JobState { QUEUED = 0, RUNNING = 1, DONE = 2, RELEASED = 3 };

struct ServeJob {
  mg_job_spec spec;
  std::vector<float> xh;     // off-diagonal extension records [n_envs][MG_NXPARAM], or empty
  double submit_s = 0.0, admit_s = -1.0, done_s = -1.0;
  int32_t job_id = -1;       // pool handle while admitted
  float *traj = nullptr;     // trajectory record (stream-ordered allocation) or null
  double traj_bytes = 0.0;
  bool last_tick_issued = false;
  JobState state = QUEUED;
};

struct Inflight {
  cudaEvent_t ev;
  std::vector<int64_t> finishing;  // tickets whose last tick precedes ev
};

double traj_bytes_of(const mg_job_spec &s) {
  return (double)s.horizon * MG_NTRAJ * 4.0 * (double)s.n_envs;
}

}  // namespace

struct mg_server {
  mg_pool *pool = nullptr;
  cudaStream_t stream = nullptr;
  cudaMemPool_t mempool = nullptr;  // trajectory records
  int64_t capacity = 0;             // envs of the pool's arena
  mg_server_config cfg{};
  std::chrono::steady_clock::time_point t0;
  std::vector<ServeJob> jobs;  // indexed by ticket
  std::deque<int64_t> queue;
  std::vector<int64_t> running;
  std::deque<Inflight> inflight;
  std::vector<cudaEvent_t> spare_events;
  double used = 0.0, peak = 0.0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

mg_status sfail(mg_status st, const char *msg) { return set_error(st, msg); }

mg_status sfail_cuda(cudaError_t e, const char *what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return set_error(e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA, buf);
}

#define SK(call)                                       \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return sfail_cuda(_e, #call); \
  } while (0)

// Hand back the jobs of the oldest in-flight tick (which has completed).
mg_status finish_front(mg_server *s) {
  Inflight f = s->inflight.front();
  s->inflight.pop_front();
  const double t = s->now();
  for (int64_t tk : f.finishing) {
    ServeJob &j = s->jobs[tk];
    j.done_s = t;
    j.state = DONE;
    s->running.erase(std::find(s->running.begin(), s->running.end(), tk));
    if (!s->cfg.keep_done) {
      mg_status st = mg_pool_release(s->pool, j.job_id);
      if (st != MG_OK) return st;
      if (j.traj) SK(cudaFreeAsync(j.traj, s->stream));
      j.traj = nullptr;
      s->used -= j.traj_bytes;
      j.state = RELEASED;
    }
  }
  s->spare_events.push_back(f.ev);
  return MG_OK;
}

// Wait (spinning, then yielding) for the oldest in-flight tick, at most wait_timeout_s.
mg_status wait_front(mg_server *s) {
  const double start = s->now();
  for (;;) {
    const cudaError_t q = cudaEventQuery(s->inflight.front().ev);
    if (q == cudaSuccess) return finish_front(s);
    if (q != cudaErrorNotReady) return sfail_cuda(q, "cudaEventQuery");
    const double t = s->now();
    if (t - start > s->cfg.wait_timeout_s)
      return sfail(MG_ETIMEOUT, "a serving tick did not complete within wait_timeout_s");
    if (t - start > 1e-3) std::this_thread::yield();
  }
}

// FIFO admission while the budget and a free range allow (serial: only into an empty server).
mg_status admit_queued(mg_server *s) {
  while (!s->queue.empty() && (!s->cfg.serial || s->running.empty())) {
    const int64_t tk = s->queue.front();
    ServeJob &j = s->jobs[tk];
    const double need = s->cfg.record ? traj_bytes_of(j.spec) : 0.0;
    if (s->used + need > s->cfg.budget_bytes) break;
    float *traj = nullptr;
    if (s->cfg.record) {
      const cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&traj),
                                                    (size_t)need, s->mempool, s->stream);
      if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        break;  // the device itself is out of memory: wait for running jobs to leave
      }
      if (e != cudaSuccess) return sfail_cuda(e, "cudaMallocFromPoolAsync(trajectory record)");
    }
    int32_t jid = -1;
    const mg_status st =
        j.xh.empty() ? mg_pool_admit(s->pool, &j.spec, traj, &jid)
                     : mg_pool_admit_offdiag(s->pool, &j.spec, traj, j.xh.data(), &jid);
    if (st == MG_ENOMEM) {  // no free arena range large enough yet
      if (traj) SK(cudaFreeAsync(traj, s->stream));
      break;
    }
    if (st != MG_OK) {
      if (traj) cudaFreeAsync(traj, s->stream);
      return st;
    }
    j.job_id = jid;
    j.traj = traj;
    std::vector<float>().swap(j.xh);  // uploaded by the admission
    j.traj_bytes = need;
    j.admit_s = s->now();
    j.state = RUNNING;
    s->used += need;
    if (s->used > s->peak) s->peak = s->used;
    s->queue.pop_front();
    s->running.push_back(tk);
  }
  return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_server_create(mg_pool *pool, const mg_server_config *cfg, mg_server **out) {
  if (!pool || !cfg || !out) return sfail(MG_EINVAL, "NULL argument");
  *out = nullptr;
  if (!(cfg->budget_bytes >= 0.0) || cfg->k < 1 || cfg->max_inflight < 1 ||
      !(cfg->wait_timeout_s > 0.0))
    return sfail(MG_EINVAL, "need budget_bytes >= 0, k >= 1, max_inflight >= 1, "
                            "wait_timeout_s > 0");
  int dev = 0;
  SK(cudaGetDevice(&dev));
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t mp = nullptr;
  SK(cudaMemPoolCreate(&mp, &props));
  uint64_t keep = UINT64_MAX;  // keep freed records for the next jobs
  cudaError_t e = cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e != cudaSuccess) {
    cudaMemPoolDestroy(mp);
    return sfail_cuda(e, "cudaMemPoolSetAttribute");
  }
  mg_server *s = new mg_server();
  s->pool = pool;
  s->stream = pool_stream(pool);
  s->capacity = pool_capacity(pool);
  s->mempool = mp;
  s->cfg = *cfg;
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return MG_OK;
}

mg_status mg_server_destroy(mg_server *s) {
  if (!s) return MG_OK;
  cudaStreamSynchronize(s->stream);
  for (ServeJob &j : s->jobs) {
    if (j.state == RUNNING || j.state == DONE) mg_pool_release(s->pool, j.job_id);
    if (j.traj) cudaFreeAsync(j.traj, s->stream);
  }
  cudaStreamSynchronize(s->stream);
  for (Inflight &f : s->inflight) cudaEventDestroy(f.ev);
  for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
  cudaMemPoolDestroy(s->mempool);
  delete s;
  return MG_OK;
}

}  // extern "C"

namespace {

mg_status submit_job(mg_server *s, const mg_job_spec *spec, const float *xh, int64_t *ticket) {
  if (!s || !spec || !ticket) return sfail(MG_EINVAL, "NULL argument");
  if (spec->n_envs < 1 || spec->n_envs > s->capacity || spec->horizon < 1 ||
      spec->hold_steps < 1)
    return sfail(MG_EINVAL, "bad job spec (n_envs outside [1, pool capacity], horizon or hold < 1)");
  if (s->cfg.record && traj_bytes_of(*spec) > s->cfg.budget_bytes)
    return sfail(MG_EINVAL, "the job's trajectory record alone exceeds the budget");
  ServeJob j;
  j.spec = *spec;
  if (xh) {  // a copy of the records, kept until the job is admitted
    j.xh.resize((size_t)spec->n_envs * MG_NXPARAM);
    SK(cudaMemcpy(j.xh.data(), xh, j.xh.size() * sizeof(float), cudaMemcpyDefault));
  }
  j.submit_s = s->now();
  *ticket = (int64_t)s->jobs.size();
  s->jobs.push_back(std::move(j));
  s->queue.push_back(*ticket);
  return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_server_submit(mg_server *s, const mg_job_spec *spec, int64_t *ticket) {
  return submit_job(s, spec, nullptr, ticket);
}

mg_status mg_server_submit_offdiag(mg_server *s, const mg_job_spec *spec, const float *xh,
                                   int64_t *ticket) {
  return submit_job(s, spec, xh, ticket);
}

mg_status mg_server_poll(mg_server *s, int32_t *n_queued, int32_t *n_running,
                         int32_t *n_inflight) {
  if (!s) return sfail(MG_EINVAL, "NULL server");
  NvtxRange nvtx("mg_server_poll");
  mg_status st = admit_queued(s);
  if (st != MG_OK) return st;
  std::vector<int64_t> finishing;
  bool advance = false;
  for (int64_t tk : s->running) {
    ServeJob &j = s->jobs[tk];
    int32_t done = 0, horizon = 0;
    if ((st = mg_pool_job_progress(s->pool, j.job_id, &done, &horizon)) != MG_OK) return st;
    if (done < horizon) advance = true;
  }
  if (advance && (st = mg_pool_tick(s->pool, s->cfg.k, nullptr)) != MG_OK) return st;
  for (int64_t tk : s->running) {
    ServeJob &j = s->jobs[tk];
    if (j.last_tick_issued) continue;
    int32_t done = 0, horizon = 0;
    if ((st = mg_pool_job_progress(s->pool, j.job_id, &done, &horizon)) != MG_OK) return st;
    if (done >= horizon) {
      j.last_tick_issued = true;
      finishing.push_back(tk);
    }
  }
  if (advance || !finishing.empty()) {
    cudaEvent_t ev = nullptr;
    if (!s->spare_events.empty()) {
      ev = s->spare_events.back();
      s->spare_events.pop_back();
    } else {
      SK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    SK(cudaEventRecord(ev, s->stream));
    s->inflight.push_back(Inflight{ev, finishing});
  }
  // Completed ticks are handed back; beyond max_inflight the oldest is waited for.
  while (!s->inflight.empty()) {
    if ((int32_t)s->inflight.size() > s->cfg.max_inflight) {
      if ((st = wait_front(s)) != MG_OK) return st;
      continue;
    }
    const cudaError_t q = cudaEventQuery(s->inflight.front().ev);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) return sfail_cuda(q, "cudaEventQuery");
    if ((st = finish_front(s)) != MG_OK) return st;
  }
  // Nothing left to advance: wait for the oldest tick, whose jobs leave (and may make room for
  // queued ones).
  if (!advance && !s->inflight.empty())
    if ((st = wait_front(s)) != MG_OK) return st;
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  if (n_running) *n_running = (int32_t)s->running.size();
  if (n_inflight) *n_inflight = (int32_t)s->inflight.size();
  return MG_OK;
}

mg_status mg_server_job(mg_server *s, int64_t ticket, double *submit_s, double *admit_s,
                        double *done_s) {
  if (!s || ticket < 0 || ticket >= (int64_t)s->jobs.size())
    return sfail(MG_EINVAL, "no such ticket");
  const ServeJob &j = s->jobs[ticket];
  if (submit_s) *submit_s = j.submit_s;
  if (admit_s) *admit_s = j.admit_s;
  if (done_s) *done_s = j.done_s;
  return MG_OK;
}

mg_status mg_server_job_result(mg_server *s, int64_t ticket, float *state, float *traj) {
  if (!s || ticket < 0 || ticket >= (int64_t)s->jobs.size())
    return sfail(MG_EINVAL, "no such ticket");
  const ServeJob &j = s->jobs[ticket];
  if (j.state != DONE) return sfail(MG_ESTATE, "the job is not finished and kept");
  mg_status st = MG_OK;
  if (state && (st = mg_pool_get_job_state(s->pool, j.job_id, state)) != MG_OK) return st;
  if (traj) {
    if (!j.traj) return sfail(MG_ESTATE, "the server does not record trajectories");
    SK(cudaMemcpyAsync(traj, j.traj, (size_t)j.traj_bytes, cudaMemcpyDefault, s->stream));
    SK(cudaStreamSynchronize(s->stream));
  }
  return MG_OK;
}

mg_status mg_server_release(mg_server *s, int64_t ticket) {
  if (!s || ticket < 0 || ticket >= (int64_t)s->jobs.size())
    return sfail(MG_EINVAL, "no such ticket");
  ServeJob &j = s->jobs[ticket];
  if (j.state != DONE) return sfail(MG_ESTATE, "the job is not finished and kept");
  mg_status st = mg_pool_release(s->pool, j.job_id);
  if (st != MG_OK) return st;
  if (j.traj) SK(cudaFreeAsync(j.traj, s->stream));
  j.traj = nullptr;
  s->used -= j.traj_bytes;
  j.state = RELEASED;
  return MG_OK;
}

mg_status mg_server_info(mg_server *s, double *now_s, double *used_bytes, double *peak_bytes) {
  if (!s) return sfail(MG_EINVAL, "NULL server");
  if (now_s) *now_s = s->now();
  if (used_bytes) *used_bytes = s->used;
  if (peak_bytes) *peak_bytes = s->peak;
  return MG_OK;
}

}  // extern "C"
