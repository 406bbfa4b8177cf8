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
#include "mg_device.cuh"

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

// Writes the observation of env e at task time t; returns |p - p_r(t)|.
__device__ float observe(const TaskView &tv, const StatePlanes &st, int64_t e, float t,
                         float *__restrict__ obs) {
  const float4 a = st.s0[e], b = st.s1[e], c = st.s2[e], d = st.s3[e];
  const float px = a.x, py = a.y, pz = a.z, qw = a.w, qx = b.x, qy = b.y, qz = b.z;
  const float nu[6] = {b.w, c.x, c.y, c.z, c.w, d.x};
  const float sp = fminf(1.f, fmaxf(-1.f, 2.f * (qw * qy - qz * qx)));
  const float phi = atan2f(2.f * (qw * qx + qy * qz), 1.f - 2.f * (qx * qx + qy * qy));
  const float theta = asinf(sp);
  const float psi = wrap_pi(atan2f(2.f * (qw * qz + qx * qy), 1.f - 2.f * (qy * qy + qz * qz)) -
                            tv.psi_r);
  const float4 cen = tv.centre[e];
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
    const float e0 = observe(tv, st, e, (float)clock * dt, o);
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
        observe(tv, st, e, 0.f, o);
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

}  // namespace

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

}  // namespace mg
