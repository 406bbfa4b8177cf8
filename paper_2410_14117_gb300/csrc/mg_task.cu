// Task layer (§EXPERIMENTS): after the sub-steps of a task step, each env's position error
// (Eq. 4), observation (Eq. 2), episode clock and accumulated error, with auto-reset of envs
// whose episode ended.  One thread per env; it reads the state once and builds the observation
// in shared memory, from which the block writes its envs' rows out together.
//
// Reference trajectories around the env's centre c (NED) with phase phi0, s = w t + phi0:
//   station keeping  p_r = c
//   circle           p_r = c + (R cos s, R sin s, 0)
//   helix            p_r = c + (R cos s, R sin s, vz t)
//   lemniscate       p_r = c + R (cos s, sin s cos s, 0) / (1 + sin^2 s)   (Bernoulli)
// Attitude reference: level, heading psi_r; attitude error = (phi, theta, wrap(psi - psi_r)) from
// the zyx Euler angles of q.  Observation: for i = 1..m (m = 1 for station keeping) the position
// error to p_r(t + i dt_look) followed by the attitude error, then nu.
#include "mg_advance.cuh"

namespace mg {

namespace {

__device__ __forceinline__ void reference(const TaskView &tv, const float4 c, float t,
                                          float &x, float &y, float &z) {
  x = c.x;
  y = c.y;
  z = c.z;
  if (tv.task == MG_TASK_STATION) return;
  float sn, cs;
  sincosf(tv.omega * t + c.w, &sn, &cs);
  if (tv.task == MG_TASK_LEMNISCATE) {
    const float d = 1.f + sn * sn;
    x += tv.radius * cs / d;
    y += tv.radius * sn * cs / d;
  } else {
    x += tv.radius * cs;
    y += tv.radius * sn;
    if (tv.task == MG_TASK_HELIX) z += tv.vz * t;
  }
}

__device__ __forceinline__ float wrap_pi(float a) {
  const float pi = 3.14159265358979f, two_pi = 6.28318530717959f;
  a = fmodf(a + pi, two_pi);
  if (a < 0.f) a += two_pi;
  return a - pi;
}

// Writes the observation at task time t of an env with reference centre cen, from its position
// p, attitude q and body velocity nu; returns |p - p_r(t)|.
__device__ __forceinline__ float observe(const TaskView &tv, const float4 cen, float t, float px,
                                         float py, float pz, float qw, float qx, float qy,
                                         float qz, const float (&nu)[6], float *__restrict__ obs) {
  const float sp = fminf(1.f, fmaxf(-1.f, 2.f * (qw * qy - qz * qx)));
  const float phi = atan2f(2.f * (qw * qx + qy * qz), 1.f - 2.f * (qx * qx + qy * qy));
  const float theta = asinf(sp);
  const float psi = wrap_pi(atan2f(2.f * (qw * qz + qx * qy), 1.f - 2.f * (qy * qy + qz * qz)) -
                            tv.psi_r);
  const int m = tv.task == MG_TASK_STATION ? 1 : tv.m;
  for (int i = 0; i < m; ++i) {
    float x, y, z;
    reference(tv, cen, tv.task == MG_TASK_STATION ? t : t + (float)(i + 1) * tv.dt_look, x, y,
              z);
    float *o = obs + 6 * i;
    o[0] = px - x;
    o[1] = py - y;
    o[2] = pz - z;
    o[3] = phi;
    o[4] = theta;
    o[5] = psi;
  }
  for (int k = 0; k < 6; ++k) obs[6 * m + k] = nu[k];
  float x, y, z;
  reference(tv, cen, t, x, y, z);
  return sqrtf((px - x) * (px - x) + (py - y) * (py - y) + (pz - z) * (pz - z));
}

__device__ __forceinline__ float observe_planes(const TaskView &tv, const StatePlanes &st,
                                                int64_t e, float t, float *__restrict__ obs) {
  const float4 a = st.s0[e], b = st.s1[e], c = st.s2[e], d = st.s3[e];
  const float nu[6] = {b.w, c.x, c.y, c.z, c.w, d.x};
  return observe(tv, tv.centre[e], t, a.x, a.y, a.z, a.w, b.x, b.y, b.z, nu, obs);
}

// Room kept for a fused task kernel's static shared memory (thruster geometry, counters: under
// 512 B) beside its dynamic staging of observation rows.
constexpr size_t kStaticSmemReserve = 1024;
// Dynamic shared memory a block may opt in to on GB300 (227 KB per block).
constexpr size_t kMaxDynSmem = 227 * 1024;

// Observation rows of `bytes` are staged in shared memory when they fit the opt-in limit.
inline bool stage_fits(size_t bytes) { return bytes + kStaticSmemReserve <= kMaxDynSmem; }

// Raise a kernel's dynamic shared-memory limit when a launch needs more than the default 48 KB.
inline cudaError_t allow_dynamic_smem(const void *kernel, size_t bytes) {
  if (bytes + kStaticSmemReserve <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Envs per block; the block's observations are staged in shared memory and written out as one
// contiguous, coalesced run (obs is env-major [n][obs_dim], so a thread's own row is strided
// across the warp).
constexpr int kTaskThreads = 64;
constexpr int kTaskMaxObs = 6 * 64 + 6;

__global__ void __launch_bounds__(kTaskThreads)
    k_task(const StatePlanes st, const TaskView tv, int64_t n, int64_t gid0, int32_t k, float dt,
           int32_t obs_dim, float *__restrict__ obs, float *__restrict__ err,
           uint8_t *__restrict__ done, float *__restrict__ ep_err, uint64_t seed, double sigma,
           uint32_t *__restrict__ episode, uint32_t *__restrict__ flags,
           unsigned long long *nonfinite_count) {
  extern __shared__ float sobs[];  // [kTaskThreads][obs_dim]
  const int64_t env0 = (int64_t)blockIdx.x * kTaskThreads;
  const int64_t e = env0 + threadIdx.x;
  if (e < n) {
    float *o = sobs + threadIdx.x * obs_dim;
    const int32_t clock = tv.clock[e] + k;
    const float e0 = observe_planes(tv, st, e, (float)clock * dt, o);
    if (k == 0) {  // observation only
      err[e] = e0;
      done[e] = 0;
      if (ep_err) ep_err[e] = 0.f;
    } else {
      const float sum = tv.err_sum[e] + e0;
      const bool bad = (flags[e] & 1u) || !(e0 == e0) || isinf(e0);
      const bool over = (tv.max_err > 0.f && e0 > tv.max_err) ||
                        (tv.episode_steps > 0 && clock >= tv.episode_steps);
      err[e] = e0;
      if (bad || over) {
        done[e] = 1;
        if (ep_err) ep_err[e] = sum;
        reset_env(st, e, (uint64_t)(gid0 + e), seed, sigma, episode, flags, nonfinite_count);
        tv.clock[e] = 0;
        tv.err_sum[e] = 0.f;
        observe_planes(tv, st, e, 0.f, o);
      } else {
        done[e] = 0;
        if (ep_err) ep_err[e] = 0.f;
        tv.clock[e] = clock;
        tv.err_sum[e] = sum;
      }
    }
  }
  __syncthreads();
  const int64_t cnt = n - env0 < kTaskThreads ? n - env0 : kTaskThreads;
  const int total = (int)cnt * obs_dim;
  float *dst = obs + env0 * obs_dim;
  int i0 = 0;
  if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {  // the run starts 16-byte aligned
    const int n4 = total >> 2;
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    const float4 *s4 = reinterpret_cast<const float4 *>(sobs);
    for (int i = threadIdx.x; i < n4; i += kTaskThreads) d4[i] = s4[i];
    i0 = n4 << 2;
  }
  for (int i = i0 + threadIdx.x; i < total; i += kTaskThreads) dst[i] = sobs[i];
}

// ---------------------------------------------------------------- fused task step
// Per-env inputs of the task epilogue, loaded before any of its stores.
struct TaskIn {
  float4 centre;
  int32_t clock;
  uint32_t flag, episode;
  float err_sum;
};

__device__ __forceinline__ TaskIn task_in(const FleetView &fv, const TaskView &tv,
                                          const TaskOut &to, int64_t e) {
  TaskIn in;
  in.centre = tv.centre[e];
  in.clock = tv.clock[e];
  in.flag = fv.flags[e];
  in.episode = to.episode[e];
  in.err_sum = tv.err_sum[e];
  return in;
}

// The task epilogue of env e from its state s after the task step's sub-steps (still in
// registers): the Eq. 4 error, the episode bookkeeping, the auto-reset (the new episode is built
// in s, so it is observed without a re-read), the state store and the Eq. 2 observation into row.
template <int MT>
__device__ __forceinline__ void task_epilogue(const FleetView &fv, const TaskView &tv,
                                              const TaskOut &to, int32_t k_task, int64_t e,
                                              const TaskIn &in, St<MT> &s, float *row) {
  const int32_t clock = in.clock + k_task;
  float t = (float)clock * fv.dt;
  float rx, ry, rz;
  reference(tv, in.centre, t, rx, ry, rz);
  const float e0 = sqrtf((s.p[0] - rx) * (s.p[0] - rx) + (s.p[1] - ry) * (s.p[1] - ry) +
                         (s.p[2] - rz) * (s.p[2] - rz));
  const uint32_t flag = in.flag;
  const bool bad = !all_finite<MT>(s) || (flag & 1u) || !(e0 == e0) || isinf(e0);
  const bool over = (tv.max_err > 0.f && e0 > tv.max_err) ||
                    (tv.episode_steps > 0 && clock >= tv.episode_steps);
  const float sum = in.err_sum + e0;
  if (to.err) to.err[e] = e0;
  if (to.reward) to.reward[e] = -e0;
  float nu[6] = {s.v[0], s.v[1], s.v[2], s.w[0], s.w[1], s.w[2]};
  if (bad || over) {
    // new episode (as reset_env)
    const uint32_t ep = in.episode;
    reset_nu(to.seed, (uint64_t)(fv.gid0 + e), ep, to.sigma, nu);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      s.p[i] = 0.f;
      s.v[i] = nu[i];
      s.w[i] = nu[3 + i];
    }
    s.q[0] = 1.f;
    s.q[1] = s.q[2] = s.q[3] = 0.f;
#pragma unroll
    for (int i = 0; i < MT; ++i) s.n[i] = 0.f;
    if (MT == 6) fv.st.s5[e] = 0.f;
    to.episode[e] = ep + 1u;
    if (flag & 1u) atomicAdd(fv.counters, ~0ull);  // decrement
    fv.flags[e] = 0u;
    to.done[e] = 1;
    if (to.ep_err) to.ep_err[e] = sum;
    tv.clock[e] = 0;
    tv.err_sum[e] = 0.f;
    t = 0.f;
  } else {
    to.done[e] = 0;
    if (to.ep_err) to.ep_err[e] = 0.f;
    tv.clock[e] = clock;
    tv.err_sum[e] = sum;
  }
  store_state<MT>(fv.st, e, s);
  observe(tv, in.centre, t, s.p[0], s.p[1], s.p[2], s.q[0], s.q[1], s.q[2], s.q[3], nu, row);
}

// Copy n_rows staged observation rows (src, in shared memory) to dst, by the warp's n_act live
// lanes (its low lanes); 16-byte stores when both ends allow.
__device__ __forceinline__ void copy_rows(const float *src, float *dst, int n_rows, int obs_dim,
                                          int lane, int n_act) {
  const int total = n_rows * obs_dim;
  int i0 = 0;
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
    const int n4 = total >> 2;
    for (int i = lane; i < n4; i += n_act)
      reinterpret_cast<float4 *>(dst)[i] = reinterpret_cast<const float4 *>(src)[i];
    i0 = n4 << 2;
  }
  for (int i = i0 + lane; i < total; i += n_act) dst[i] = src[i];
}

// The last launch of a task step: the env's final sub-steps as in k_fleet, then the task
// epilogue from the state still in registers, so the state is stored once and never re-read.
// Each warp stages its 32 rows of the observation in shared memory (when they fit) and writes
// them out as one contiguous run.
template <int NTV, bool DIAG, int NH, bool XH>
__global__ void __maxnreg__(XH ? kRegsXH : DIAG ? kRegsDiag : kRegsGeneral)
    k_fleet_task(const FleetView fv, const BlockDesc *__restrict__ blocks, const int32_t k_launch,
                 const int32_t k_task, const TaskView tv, const TaskOut to) {
  constexpr int MT = (NTV == NT_6) ? 6 : 8;
  constexpr bool MIXED = (NTV == NT_MIXED);
  __shared__ float4 sdir[MG_MAX_THR], sarm[MG_MAX_THR];
  __shared__ unsigned s_done;
  __shared__ int64_t s_cursor;
  // dynamic: [blockDim.x][MG_NXPARAM] off-diagonal hydrodynamics (XH), then
  // [blockDim.x][obs_dim] observation rows (to.stage)
  extern __shared__ float sdyn[];
  float *sxh = sdyn;
  float *sobs = sdyn + (XH ? blockDim.x * MG_NXPARAM : 0);

  const BlockDesc bd = blocks[blockIdx.x];
  if (threadIdx.x < MG_MAX_THR) {
    sdir[threadIdx.x] = fv.geo[bd.type].dir[threadIdx.x];
    sarm[threadIdx.x] = fv.geo[bd.type].arm[threadIdx.x];
  }
  // Programmatic dependent launch: the block descriptors and the geometry above are written
  // before any step; everything below waits for the previous kernel in the stream (the action
  // copy of mg_env_step, or the task step's leading launches) to complete.
  cudaGridDependencySynchronize();
  if (threadIdx.x == 0) {
    s_done = 0u;
    s_cursor = launch_cursor(fv);
  }
  if constexpr (XH) stage_xh(fv.xh, fv.n, bd.env0, bd.count, sxh);
  __syncthreads();
  if ((int)threadIdx.x >= bd.count) return;
  const int64_t e = (int64_t)bd.env0 + threadIdx.x;
  St<MT> s;
  // the classic lag update fits the 128-register variants' epilogue; the 255-register XH
  // variant takes the closed form, as k_fleet does
  advance_env<MT, DIAG, MIXED, false, false, NH, XH, XH>(
      fv, e, MIXED ? bd.n_thr : MT, sdir, sarm, s_cursor + fv.cursor_off, k_launch, nullptr, s,
      XH ? sxh + threadIdx.x * MG_NXPARAM : nullptr);

  const int obs_dim = to.obs_dim;
  task_epilogue<MT>(fv, tv, to, k_task, e, task_in(fv, tv, to, e), s,
                    to.stage ? sobs + threadIdx.x * obs_dim : to.obs + e * obs_dim);
  if (fv.cursor_adv) finish_envs(fv, &s_done, bd.count, fv.cursor_adv);
  if (!to.stage) return;
  // Warp copy-out: the warp's live lanes are its low lanes (threads below bd.count).
  const int lane = threadIdx.x & 31;
  const int wbase = threadIdx.x & ~31;
  const int n_act = min(32, bd.count - wbase);
  __syncwarp(n_act == 32 ? 0xffffffffu : ((1u << n_act) - 1u));
  copy_rows(sobs + wbase * obs_dim, to.obs + ((int64_t)bd.env0 + wbase) * obs_dim, n_act, obs_dim,
            lane, n_act);
}

template <int NTV, bool DIAG, int NH, bool XH = false>
cudaError_t fleet_task_t(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                         int32_t k_launch, int32_t k_task, const TaskView &tv, const TaskOut &to,
                         size_t smem, cudaStream_t stream) {
  const cudaError_t e = allow_dynamic_smem(
      reinterpret_cast<const void *>(&k_fleet_task<NTV, DIAG, NH, XH>), smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)n_blocks);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fleet_task<NTV, DIAG, NH, XH>, fv, blocks, k_launch, k_task,
                            tv, to);
}


template <int NTV>
cudaError_t fleet_task_d(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                         bool diag, bool structured, int32_t k_launch, int32_t k_task,
                         const TaskView &tv, const TaskOut &to, size_t smem,
                         cudaStream_t stream) {
  if (fv.xh)
    return fleet_task_t<NTV, false, 0, true>(fv, blocks, n_blocks, threads, k_launch, k_task, tv,
                                             to, smem, stream);
  if (diag && structured)
    return fleet_task_t<NTV, true, 4>(fv, blocks, n_blocks, threads, k_launch, k_task, tv, to,
                                      smem, stream);
  if (diag)
    return fleet_task_t<NTV, true, 0>(fv, blocks, n_blocks, threads, k_launch, k_task, tv, to,
                                      smem, stream);
  return fleet_task_t<NTV, false, 0>(fv, blocks, n_blocks, threads, k_launch, k_task, tv, to,
                                     smem, stream);
}

__global__ void k_clamp_actions(const float *__restrict__ in, float *__restrict__ out,
                                int64_t count) {
  // the task kernel that follows may launch now and wait for this copy at its dependency point
  cudaTriggerProgrammaticLaunchCompletion();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float x = in[i];
  out[i] = x < -1.f ? -1.f : (x > 1.f ? 1.f : x);
}

}  // namespace

cudaError_t launch_clamp_actions(const float *in, float *out, int64_t count, cudaStream_t stream) {
  if (count < 1) return cudaSuccess;
  const int64_t grid = (count + 255) / 256;
  k_clamp_actions<<<(unsigned)grid, 256, 0, stream>>>(in, out, count);
  return cudaGetLastError();
}

cudaError_t launch_task(const StatePlanes &st, const TaskView &tv, int64_t n, int64_t gid0,
                        int32_t k, float dt, float *obs, float *err, uint8_t *done,
                        float *ep_err, uint64_t seed, double sigma, uint32_t *episode,
                        uint32_t *flags, unsigned long long *nonfinite_count,
                        cudaStream_t stream) {
  const int obs_dim = 6 * (tv.task == MG_TASK_STATION ? 1 : tv.m) + 6;
  if (obs_dim > kTaskMaxObs) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * kTaskThreads * obs_dim;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_task, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(float) * kTaskThreads * kTaskMaxObs));
    if (e != cudaSuccess) return e;
  }
  const int64_t grid = (n + kTaskThreads - 1) / kTaskThreads;
  k_task<<<(unsigned)grid, kTaskThreads, smem, stream>>>(st, tv, n, gid0, k, dt, obs_dim, obs,
                                                         err, done, ep_err, seed, sigma, episode,
                                                         flags, nonfinite_count);
  return cudaGetLastError();
}

cudaError_t launch_fleet_task(const FleetView &fv, const BlockDesc *blocks, int n_blocks,
                              int threads, NtVariant ntv, bool diag, bool structured,
                              int32_t k_launch, int32_t k_task, const TaskView &tv, TaskOut to,
                              cudaStream_t stream) {
  if (threads < 32 || threads > 256 || threads % 32 || n_blocks < 1 || k_launch < 1 ||
      k_task < k_launch || (fv.xh && diag))
    return cudaErrorInvalidValue;
  // The off-diagonal hydrodynamics (if any) come first; the observation rows are staged in
  // shared memory when both fit beside the static shared memory (above 48 KB by opt-in).
  const size_t xh_bytes = fv.xh ? sizeof(float) * threads * MG_NXPARAM : 0;
  const size_t smem = sizeof(float) * threads * to.obs_dim;
  to.stage = stage_fits(xh_bytes + smem) ? 1 : 0;
  const size_t dyn = xh_bytes + (to.stage ? smem : 0);
  switch (ntv) {
    case NT_6:
      return fleet_task_d<NT_6>(fv, blocks, n_blocks, threads, diag, structured, k_launch,
                                k_task, tv, to, dyn, stream);
    case NT_8:
      return fleet_task_d<NT_8>(fv, blocks, n_blocks, threads, diag, structured, k_launch,
                                k_task, tv, to, dyn, stream);
    default:
      return fleet_task_d<NT_MIXED>(fv, blocks, n_blocks, threads, diag, structured, k_launch,
                                    k_task, tv, to, dyn, stream);
  }
}

}  // namespace mg
