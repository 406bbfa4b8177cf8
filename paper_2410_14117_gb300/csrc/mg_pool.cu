// Job pool for serving rollouts with continuous batching.
//
// A pool owns an env arena (the same SoA planes as a sim) of fixed capacity.  A job is a block of
// envs of one vehicle type with its own parameter seed, procedural command seed, hold and
// horizon; admission takes a contiguous free range of the arena (first fit, freed ranges merge
// back), randomises the job's parameters and resets its envs with counter-based draws keyed by
// the job's seeds and job-local env ids, so a job's result does not depend on where it sits or
// what else runs.  Each tick is one launch of k_serve over every running job: a job advances
// min(k, horizon - done) sub-steps, recording its trajectory into a caller-owned device buffer.
// Jobs that arrive while others run join at the next tick.  Jobs admitted with the off-diagonal
// hydrodynamic extension (full M_A and D_l) run in a second launch of the same tick, on the
// general path with each block's coefficients staged in shared memory.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "mg_advance.cuh"

namespace mg {

struct JobDesc {
  int64_t env0;     // arena index of the job's first env
  float *traj;      // [horizon][MG_NTRAJ][n] or null
  uint64_t cmd_seed;
  int32_t n;
  int32_t type;
  int32_t n_thr;
  int32_t hold;
  int32_t step0;    // sub-steps done before this tick
  int32_t steps;    // sub-steps this tick
};

struct ServeBlock {
  int32_t job;      // index into the tick's job table
  int32_t first;    // job-local env index of the block's first env
  int32_t count;
  int32_t pad;
};

namespace {

constexpr int kServeThreads = 128;
// Register cap of the tick kernel for ticks of many blocks: the diagonal-mass step coefficients
// do not fit 128 registers beside the trajectory record without spilling; 144 (three blocks per
// SM) served the 200 req/s job mix at p99 2.0 ms against 2.25 ms at 128, and the 10x stream at
// 6.7 against 8.4 ms.
constexpr int kRegsServe = 144;

// WIDE (diagonal mass): 200 registers, for ticks whose blocks all fit at two per SM.  Few envs
// (a warp per scheduler or fewer) run latency-bound and gain from the extra registers; a tick of
// more blocks keeps more per SM resident with kRegsServe.  Measured on the 200 req/s job mix: p50
// 0.60 -> 0.56 ms with this choice per tick; the wide kernel for every tick gave the same p50 but
// p99 2.0 -> 2.3 ms (the 65,536-env jobs).
// XH (general path): the off-diagonal hydrodynamic coefficients of the block's envs, read from
// the pool's [MG_NXPARAM][capacity] planes into dynamic shared memory [kServeThreads][MG_NXPARAM].
template <bool DIAG, int NH, bool WIDE = false, bool XH = false>
__global__ void __maxnreg__(XH ? kRegsXH : !DIAG ? kRegsGeneral : WIDE ? kRegsWide : kRegsServe)
    k_serve(const FleetView fv, const JobDesc *__restrict__ jobs,
            const ServeBlock *__restrict__ blocks) {
  static_assert(!XH || !DIAG, "the off-diagonal extension runs on the general path");
  constexpr int MT = MG_MAX_THR;
  __shared__ float4 sdir[MG_MAX_THR], sarm[MG_MAX_THR];
  extern __shared__ float sxh[];
  const ServeBlock b = blocks[blockIdx.x];
  const JobDesc jd = jobs[b.job];
  if (threadIdx.x < MG_MAX_THR) {
    sdir[threadIdx.x] = fv.geo[jd.type].dir[threadIdx.x];
    sarm[threadIdx.x] = fv.geo[jd.type].arm[threadIdx.x];
  }
  if constexpr (XH) stage_xh(fv.xh, fv.n, jd.env0 + b.first, b.count, sxh);
  __syncthreads();
  if ((int)threadIdx.x >= b.count || jd.steps <= 0) return;
  const int64_t el = (int64_t)b.first + threadIdx.x;  // job-local env
  const int64_t e = jd.env0 + el;                     // arena env
  const int nt = jd.n_thr;
  const bool current_accel = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);

  St<MT> s;
  load_state<MT>(fv.st, e, s);
  Coef<DIAG> P;
  {
    Par<DIAG> raw;
    load_par<DIAG>(fv.pa, e, raw);
    P = make_coef<DIAG>(raw);
  }
  int64_t seg = jd.step0 / jd.hold;
  int32_t left = jd.hold - (int32_t)(jd.step0 - seg * jd.hold);
  const LagEnv L = lag_env(P.itau, fv.dt);
  float lb[MT];
  auto load = [&](int64_t sg) {
    float c[MT];
    procedural_commands<MT>(jd.cmd_seed, (uint64_t)el, sg, c);
#pragma unroll
    for (int i = 0; i < MT; ++i) c[i] = (i < nt) ? c[i] * P.itau : 0.f;
    lag_segment<MT>(c, L, lb);
  };
  load(seg);
  for (int32_t it = 0; it < jd.steps; ++it) {
    if (left == 0) {
      ++seg;
      left = jd.hold;
      load(seg);
    }
    rk4_step_lag<MT, DIAG, true, NH, XH>(s, lb, L, P, sdir, sarm, nt, current_accel, fv.dt,
                                         XH ? sxh + threadIdx.x * MG_NXPARAM : nullptr);
    --left;
    if (jd.traj) {
      float *t = jd.traj + ((int64_t)(jd.step0 + it) * MG_NTRAJ) * jd.n + el;
      const int64_t n = jd.n;
      t[0 * n] = s.p[0]; t[1 * n] = s.p[1]; t[2 * n] = s.p[2];
      t[3 * n] = s.q[0]; t[4 * n] = s.q[1]; t[5 * n] = s.q[2]; t[6 * n] = s.q[3];
      t[7 * n] = s.v[0]; t[8 * n] = s.v[1]; t[9 * n] = s.v[2];
      t[10 * n] = s.w[0]; t[11 * n] = s.w[1]; t[12 * n] = s.w[2];
    }
  }
  store_state<MT>(fv.st, e, s);
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace

}  // namespace mg

using namespace mg;

namespace {

mg_status pfail(mg_status st, const std::string &msg) { return set_error(st, msg); }

mg_status pfail_cuda(cudaError_t e, const char *what) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return pfail(e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA, buf);
}

#define PK(call)                                          \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return pfail_cuda(_e, #call);  \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool dev_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Job {
  bool live = false;
  bool xh = false;  // admitted with the off-diagonal hydrodynamic extension
  int64_t env0 = 0;
  int32_t n = 0, type = 0, hold = 1, horizon = 0, done = 0;
  uint64_t cmd_seed = 0;
  float *traj = nullptr;
};

// One slot of the pinned staging ring: the tick's job table followed by its block list.
struct Stage {
  void *host = nullptr;
  size_t cap = 0;
  cudaEvent_t used = nullptr;
};

}  // namespace

struct mg_pool {
  int64_t cap = 0;
  int32_t n_types = 0;
  std::vector<mg_vehicle_params> vp;
  bool diag = true;
  bool structured = true;  // every vehicle type has the vectored thruster layout
  cudaStream_t stream = nullptr;
  void *arena = nullptr;
  StatePlanes st{};
  ParamPlanes pa{};
  float *raw = nullptr;
  int32_t *types = nullptr;
  Geo *geo = nullptr;
  float *nominal = nullptr;
  uint32_t *flags = nullptr, *episode = nullptr;
  unsigned long long *counters = nullptr;
  unsigned int *offdiag = nullptr;
  // off-diagonal hydrodynamics, [MG_NXPARAM][cap] planes (allocated at the first job that has
  // them; rows of other jobs are stale and never read)
  float *xh = nullptr;
  std::map<int64_t, int64_t> free_ranges;  // start -> length
  std::vector<Job> jobs;
  void *dev_table = nullptr;  // device copy of the tick's job table + block list
  size_t dev_table_cap = 0;
  Stage ring[3];
  int ring_at = 0;
  float dt = 0.01f;
  int n_sm = 1;
};

namespace {

FleetView pool_view(const mg_pool *p) {
  FleetView v{};
  v.st = p->st;
  v.pa = p->pa;
  v.geo = p->geo;
  v.n_types = p->n_types;
  v.n = p->cap;
  v.dt = p->dt;
  v.flags = p->flags;
  v.counters = p->counters;
  v.hold = 1;
  v.spin_limit = MG_WAIT_POLLS_DEFAULT;
  v.xh = p->xh;
  return v;
}

StatePlanes sub_state(const StatePlanes &s, int64_t e0) {
  StatePlanes r = s;
  r.s0 += e0; r.s1 += e0; r.s2 += e0; r.s3 += e0; r.s4 += e0; r.s5 += e0;
  return r;
}

ParamPlanes sub_params(const ParamPlanes &p, int64_t e0) {
  ParamPlanes r = p;
  r.d0 += e0; r.d1 += e0; r.d2 += e0; r.d3 += e0; r.d4 += e0; r.d5 += e0; r.d6 += e0;
  r.d7 += e0; r.d8 += e0; r.g0 += e0; r.g1 += e0; r.g2 += e0; r.g3 += e0; r.g4 += e0;
  r.g5 += e0;
  return r;
}

bool take_range(mg_pool *p, int64_t n, int64_t *start) {
  for (auto it = p->free_ranges.begin(); it != p->free_ranges.end(); ++it) {
    if (it->second >= n) {
      *start = it->first;
      const int64_t rest = it->second - n, at = it->first + n;
      p->free_ranges.erase(it);
      if (rest > 0) p->free_ranges[at] = rest;
      return true;
    }
  }
  return false;
}

void give_range(mg_pool *p, int64_t start, int64_t n) {
  auto it = p->free_ranges.emplace(start, n).first;
  auto nx = std::next(it);
  if (nx != p->free_ranges.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    p->free_ranges.erase(nx);
  }
  if (it != p->free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      p->free_ranges.erase(it);
    }
  }
}

}  // namespace

extern "C" {

mg_status mg_pool_create(int64_t capacity_envs, const mg_vehicle_params *params,
                         int32_t n_types, mg_pool **out) {
  if (!out || !params) return pfail(MG_EINVAL, "NULL argument");
  *out = nullptr;
  if (capacity_envs < 1 || capacity_envs > (int64_t)INT32_MAX - 1024)
    return pfail(MG_EINVAL, "capacity_envs out of range");
  if (n_types < 1 || n_types > MG_MAX_TYPES) return pfail(MG_EINVAL, "n_types out of range");
  for (int32_t t = 0; t < n_types; ++t)
    if (params[t].n_thr < 1 || params[t].n_thr > MG_MAX_THR)
      return pfail(MG_EINVAL, "n_thr out of range");
  mg_pool *p = new mg_pool();
  p->cap = capacity_envs;
  p->n_types = n_types;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    if (p->n_sm < 1) p->n_sm = 1;
  }
  p->vp.assign(params, params + n_types);
  for (int32_t t = 0; t < n_types; ++t)
    for (int i = 0; i < 3; ++i)
      if (params[t].rg[i] != 0.f) p->diag = false;
  const int64_t n = capacity_envs;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  size_t o_s[5], o_d[8], o_g[5];
  for (auto &x : o_s) x = take(16 * n);
  const size_t o_s5 = take(4 * n);
  for (auto &x : o_d) x = take(16 * n);
  const size_t o_d8 = take(8 * n);
  for (auto &x : o_g) x = take(16 * n);
  const size_t o_g5 = take(4 * n);
  const size_t o_raw = take(4 * n * MG_NPARAM), o_types = take(4 * n);
  const size_t o_geo = take(sizeof(Geo) * n_types), o_nom = take(4 * MG_NPARAM * n_types);
  const size_t o_flags = take(4 * n), o_ep = take(4 * n);
  const size_t o_cnt = take(3 * sizeof(unsigned long long)), o_off = take(sizeof(unsigned));
  cudaError_t e = cudaMalloc(&p->arena, off);
  if (e != cudaSuccess) {
    delete p;
    return pfail_cuda(e, "cudaMalloc(pool arena)");
  }
  char *a = static_cast<char *>(p->arena);
  float4 **sp[5] = {&p->st.s0, &p->st.s1, &p->st.s2, &p->st.s3, &p->st.s4};
  for (int i = 0; i < 5; ++i) *sp[i] = (float4 *)(a + o_s[i]);
  p->st.s5 = (float *)(a + o_s5);
  float4 **dp[8] = {&p->pa.d0, &p->pa.d1, &p->pa.d2, &p->pa.d3,
                    &p->pa.d4, &p->pa.d5, &p->pa.d6, &p->pa.d7};
  for (int i = 0; i < 8; ++i) *dp[i] = (float4 *)(a + o_d[i]);
  p->pa.d8 = (float2 *)(a + o_d8);
  float4 **gp[5] = {&p->pa.g0, &p->pa.g1, &p->pa.g2, &p->pa.g3, &p->pa.g4};
  for (int i = 0; i < 5; ++i) *gp[i] = (float4 *)(a + o_g[i]);
  p->pa.g5 = (float *)(a + o_g5);
  p->raw = (float *)(a + o_raw);
  p->types = (int32_t *)(a + o_types);
  p->geo = (Geo *)(a + o_geo);
  p->nominal = (float *)(a + o_nom);
  p->flags = (uint32_t *)(a + o_flags);
  p->episode = (uint32_t *)(a + o_ep);
  p->counters = (unsigned long long *)(a + o_cnt);
  p->offdiag = (unsigned *)(a + o_off);

  std::vector<Geo> geo(n_types);
  std::vector<float> nom((size_t)n_types * MG_NPARAM, 0.f);
  for (int32_t t = 0; t < n_types; ++t) {
    const mg_vehicle_params &v = params[t];
    Geo &g = geo[t];
    memset(&g, 0, sizeof g);
    g.n_thr = v.n_thr;
    for (int i = 0; i < v.n_thr; ++i) {
      const float *r = v.r[i], *d = v.d[i];
      g.dir[i] = make_float4(d[0], d[1], d[2], 0.f);
      g.arm[i] = make_float4(r[1] * d[2] - r[2] * d[1], r[2] * d[0] - r[0] * d[2],
                             r[0] * d[1] - r[1] * d[0], 0.f);
    }
    if (!vectored_layout(g)) p->structured = false;
    float *q = &nom[(size_t)t * MG_NPARAM];
    q[MG_P_M] = v.m;
    q[MG_P_IG] = v.Ixx;
    q[MG_P_IG + 1] = v.Iyy;
    q[MG_P_IG + 2] = v.Izz;
    for (int i = 0; i < 6; ++i) {
      q[MG_P_MA + i] = v.MA[i];
      q[MG_P_DL + i] = v.Dl[i];
      q[MG_P_DQ + i] = v.Dq[i];
    }
    q[MG_P_W] = v.W;
    q[MG_P_B] = v.B;
    for (int i = 0; i < 3; ++i) {
      q[MG_P_RG + i] = v.rg[i];
      q[MG_P_RB + i] = v.rb[i];
    }
    q[MG_P_KT] = v.kT;
    q[MG_P_TAU] = v.tau_m;
  }
  e = cudaMemset(p->arena, 0, off);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->geo, geo.data(), sizeof(Geo) * n_types, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->nominal, nom.data(), nom.size() * 4, cudaMemcpyHostToDevice);
  for (auto &r : p->ring)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.used, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    mg_pool_destroy(p);
    return pfail_cuda(e, "pool set-up");
  }
  p->free_ranges[0] = capacity_envs;
  *out = p;
  return MG_OK;
}

mg_status mg_pool_destroy(mg_pool *p) {
  if (!p) return MG_OK;
  cudaDeviceSynchronize();
  for (auto &r : p->ring) {
    if (r.host) cudaFreeHost(r.host);
    if (r.used) cudaEventDestroy(r.used);
  }
  cudaFree(p->dev_table);
  cudaFree(p->xh);
  cudaFree(p->arena);
  delete p;
  return MG_OK;
}

}  // extern "C"

cudaStream_t mg::pool_stream(const mg_pool *p) { return p->stream; }
int64_t mg::pool_capacity(const mg_pool *p) { return p->cap; }

extern "C" {

mg_status mg_pool_set_stream(mg_pool *p, void *stream) {
  if (!p) return pfail(MG_EINVAL, "NULL pool");
  p->stream = static_cast<cudaStream_t>(stream);
  return MG_OK;
}

}  // extern "C"

namespace {

// Device work of an admission: the job's type ids, its off-diagonal records (xh: host or device
// [n_envs][MG_NXPARAM], or null) into its columns of the pool's planes, randomised parameters
// and derived planes, episode counters and start states.
cudaError_t init_job(mg_pool *p, const mg_job_spec &s, int64_t env0, const float *xh) {
  const mg_ranges &r = s.ranges;
  const int64_t n = s.n_envs;
  const int grid = (int)((n + 255) / 256);
  k_fill_i32<<<grid, 256, 0, p->stream>>>(p->types + env0, n, s.vehicle_type);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SetupView v{};
  v.n = n;
  v.gid0 = 0;
  v.types = p->types + env0;
  v.raw = p->raw + env0 * MG_NPARAM;
  v.pa = sub_params(p->pa, env0);
  v.n_not_spd = p->counters + 1;
  v.any_offdiag = p->offdiag;
  if (xh) {
    // stride of the planes: the capacity
    const size_t bytes = (size_t)n * MG_NXPARAM * 4;
    if (dev_ptr(xh)) {
      e = launch_xh_transpose(xh, p->xh + env0, n, true, p->stream, p->cap);
    } else {
      float *tmp = nullptr;
      e = cudaMallocAsync(reinterpret_cast<void **>(&tmp), bytes, p->stream);
      if (e != cudaSuccess) return e;
      e = cudaMemcpyAsync(tmp, xh, bytes, cudaMemcpyHostToDevice, p->stream);
      if (e == cudaSuccess) e = launch_xh_transpose(tmp, p->xh + env0, n, true, p->stream, p->cap);
      cudaFreeAsync(tmp, p->stream);
    }
    if (e != cudaSuccess) return e;
    v.xh = p->xh + env0;
    v.xh_stride = p->cap;
  }
  e = launch_randomize(v, p->nominal, s.param_seed, (double)r.lo, (double)r.hi,
                       (double)r.current_sigma, (double)r.rg_halfwidth, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->episode + env0, 0, 4 * n, p->stream);
  if (e == cudaSuccess)
    e = launch_reset(sub_state(p->st, env0), n, 0, nullptr, s.param_seed, (double)r.nu0_sigma,
                     p->episode + env0, p->flags + env0, p->counters, p->stream);
  return e;
}

mg_status admit_job(mg_pool *p, const mg_job_spec *spec, float *traj, const float *xh,
                    int32_t *job_id) {
  if (!p || !spec || !job_id) return pfail(MG_EINVAL, "NULL argument");
  const mg_job_spec &s = *spec;
  const mg_ranges &r = s.ranges;
  if (s.n_envs < 1 || s.n_envs > p->cap || s.vehicle_type < 0 ||
      s.vehicle_type >= p->n_types || s.hold_steps < 1 || s.horizon < 1 || !(r.lo > 0.f) ||
      !(r.lo <= r.hi) || !(r.current_sigma >= 0.f) || !(r.nu0_sigma >= 0.f) || r.flags != 0 ||
      !(r.rg_halfwidth >= 0.f))
    return pfail(MG_EINVAL, "bad job spec");
  if (r.rg_halfwidth > 0.f && p->diag && !xh)
    return pfail(MG_EINVAL,
                 "randomised r_g needs a pool created with an off-centre-gravity vehicle type");
  if (traj && !dev_ptr(traj)) return pfail(MG_EINVAL, "traj must be device memory");
  if (xh && !p->xh) {
    const size_t bytes = (size_t)p->cap * MG_NXPARAM * 4;
    if (cudaMalloc(reinterpret_cast<void **>(&p->xh), bytes) != cudaSuccess) {
      cudaGetLastError();
      p->xh = nullptr;
      return pfail(MG_ENOMEM, "cudaMalloc(pool off-diagonal hydrodynamics)");
    }
    PK(cudaMemsetAsync(p->xh, 0, bytes, p->stream));
  }
  int64_t env0 = 0;
  if (!take_range(p, s.n_envs, &env0))
    return pfail(MG_ENOMEM, "no free range of the pool is large enough");
  int32_t id = 0;
  while (id < (int32_t)p->jobs.size() && p->jobs[id].live) ++id;
  if (id == (int32_t)p->jobs.size()) p->jobs.emplace_back();
  Job &j = p->jobs[id];
  j.live = true;
  j.xh = (xh != nullptr);
  j.env0 = env0;
  j.n = (int32_t)s.n_envs;
  j.type = s.vehicle_type;
  j.hold = s.hold_steps;
  j.horizon = s.horizon;
  j.done = 0;
  j.cmd_seed = s.cmd_seed;
  j.traj = traj;
  // Parameters and start state of the job's envs, keyed by its own seed and local env ids; on
  // a failure the range and the slot are given back.
  const cudaError_t e = init_job(p, s, env0, xh);
  if (e != cudaSuccess) {
    give_range(p, env0, s.n_envs);
    j.live = false;
    j.traj = nullptr;
    return pfail_cuda(e, "job admission");
  }
  *job_id = id;
  return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_pool_admit(mg_pool *p, const mg_job_spec *spec, float *traj, int32_t *job_id) {
  NvtxRange nvtx("mg_pool_admit");
  return admit_job(p, spec, traj, nullptr, job_id);
}

mg_status mg_pool_admit_offdiag(mg_pool *p, const mg_job_spec *spec, float *traj,
                                const float *xh, int32_t *job_id) {
  NvtxRange nvtx("mg_pool_admit_offdiag");
  return admit_job(p, spec, traj, xh, job_id);
}

mg_status mg_pool_tick(mg_pool *p, int32_t k, int32_t *n_running) {
  NvtxRange nvtx("mg_pool_tick");
  if (!p) return pfail(MG_EINVAL, "NULL pool");
  if (k < 1) return pfail(MG_EINVAL, "k must be >= 1");
  std::vector<JobDesc> table;
  std::vector<ServeBlock> blocks, xblocks;  // jobs without and with the off-diagonal extension
  for (size_t i = 0; i < p->jobs.size(); ++i) {
    Job &j = p->jobs[i];
    if (!j.live || j.done >= j.horizon) continue;
    JobDesc d{};
    d.env0 = j.env0;
    d.traj = j.traj;
    d.cmd_seed = j.cmd_seed;
    d.n = j.n;
    d.type = j.type;
    d.n_thr = p->vp[j.type].n_thr;
    d.hold = j.hold;
    d.step0 = j.done;
    d.steps = std::min(k, j.horizon - j.done);
    const int32_t idx = (int32_t)table.size();
    table.push_back(d);
    for (int32_t f = 0; f < j.n; f += kServeThreads)
      (j.xh ? xblocks : blocks).push_back(ServeBlock{idx, f, std::min(kServeThreads, j.n - f), 0});
    j.done += d.steps;
  }
  if (n_running) *n_running = (int32_t)table.size();
  if (table.empty()) return MG_OK;
  const size_t tb = align_up(table.size() * sizeof(JobDesc), 256);
  const size_t nb = blocks.size(), nx = xblocks.size();
  const size_t bytes = tb + (nb + nx) * sizeof(ServeBlock);
  Stage &sg = p->ring[p->ring_at];
  p->ring_at = (p->ring_at + 1) % 3;
  PK(cudaEventSynchronize(sg.used));  // the slot's previous copy has been consumed
  if (sg.cap < bytes) {
    if (sg.host) cudaFreeHost(sg.host);
    sg.host = nullptr;
    sg.cap = 0;
    PK(cudaMallocHost(&sg.host, bytes));
    sg.cap = bytes;
  }
  if (p->dev_table_cap < bytes) {
    PK(cudaStreamSynchronize(p->stream));
    cudaFree(p->dev_table);
    p->dev_table = nullptr;
    p->dev_table_cap = 0;
    PK(cudaMalloc(&p->dev_table, 2 * bytes));
    p->dev_table_cap = 2 * bytes;
  }
  char *h = static_cast<char *>(sg.host);
  memcpy(h, table.data(), table.size() * sizeof(JobDesc));
  memcpy(h + tb, blocks.data(), nb * sizeof(ServeBlock));
  memcpy(h + tb + nb * sizeof(ServeBlock), xblocks.data(), nx * sizeof(ServeBlock));
  PK(cudaMemcpyAsync(p->dev_table, h, bytes, cudaMemcpyHostToDevice, p->stream));
  PK(cudaEventRecord(sg.used, p->stream));
  const JobDesc *jt = static_cast<const JobDesc *>(p->dev_table);
  const ServeBlock *bl =
      reinterpret_cast<const ServeBlock *>(static_cast<char *>(p->dev_table) + tb);
  const FleetView v = pool_view(p);
  const int g = (int)nb;
  const bool wide = g <= 2 * p->n_sm;
  if (g == 0)
    ;
  else if (p->diag && p->structured && wide)
    k_serve<true, 4, true><<<g, kServeThreads, 0, p->stream>>>(v, jt, bl);
  else if (p->diag && p->structured)
    k_serve<true, 4><<<g, kServeThreads, 0, p->stream>>>(v, jt, bl);
  else if (p->diag && wide)
    k_serve<true, 0, true><<<g, kServeThreads, 0, p->stream>>>(v, jt, bl);
  else if (p->diag)
    k_serve<true, 0><<<g, kServeThreads, 0, p->stream>>>(v, jt, bl);
  else
    k_serve<false, 0><<<g, kServeThreads, 0, p->stream>>>(v, jt, bl);
  PK(cudaGetLastError());
  if (nx > 0) {
    constexpr size_t kXhBytes = sizeof(float) * kServeThreads * MG_NXPARAM;  // 23,040 B
    k_serve<false, 0, false, true>
        <<<(int)nx, kServeThreads, kXhBytes, p->stream>>>(v, jt, bl + nb);
    PK(cudaGetLastError());
  }
  return MG_OK;
}

mg_status mg_pool_job_progress(mg_pool *p, int32_t id, int32_t *done, int32_t *horizon) {
  if (!p || id < 0 || id >= (int32_t)p->jobs.size() || !p->jobs[id].live)
    return pfail(MG_EINVAL, "no such job");
  if (done) *done = p->jobs[id].done;
  if (horizon) *horizon = p->jobs[id].horizon;
  return MG_OK;
}

mg_status mg_pool_get_job_state(mg_pool *p, int32_t id, float *out) {
  if (!p || !out || id < 0 || id >= (int32_t)p->jobs.size() || !p->jobs[id].live)
    return pfail(MG_EINVAL, "no such job");
  const Job &j = p->jobs[id];
  const size_t bytes = (size_t)j.n * MG_NSTATE * 4;
  if (dev_ptr(out)) {
    PK(launch_export_state(sub_state(p->st, j.env0), j.n, out, p->stream));
    return MG_OK;
  }
  float *tmp = nullptr;
  PK(cudaMallocAsync(reinterpret_cast<void **>(&tmp), bytes, p->stream));
  cudaError_t e = launch_export_state(sub_state(p->st, j.env0), j.n, tmp, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, p->stream);
  cudaFreeAsync(tmp, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return pfail_cuda(e, "mg_pool_get_job_state");
  return MG_OK;
}

mg_status mg_pool_release(mg_pool *p, int32_t id) {
  if (!p || id < 0 || id >= (int32_t)p->jobs.size() || !p->jobs[id].live)
    return pfail(MG_EINVAL, "no such job");
  Job &j = p->jobs[id];
  give_range(p, j.env0, j.n);
  j.live = false;
  j.traj = nullptr;
  return MG_OK;
}

mg_status mg_pool_info(mg_pool *p, int64_t *free_envs, int64_t *largest_free, int32_t *n_jobs) {
  if (!p) return pfail(MG_EINVAL, "NULL pool");
  int64_t tot = 0, big = 0;
  for (auto &kv : p->free_ranges) {
    tot += kv.second;
    big = std::max(big, kv.second);
  }
  int32_t live = 0;
  for (auto &j : p->jobs) live += j.live ? 1 : 0;
  if (free_envs) *free_envs = tot;
  if (largest_free) *largest_free = big;
  if (n_jobs) *n_jobs = live;
  return MG_OK;
}

mg_status mg_pool_sync(mg_pool *p) {
  if (!p) return pfail(MG_EINVAL, "NULL pool");
  PK(cudaStreamSynchronize(p->stream));
  return MG_OK;
}

}  // extern "C"
