// Per-env step loop shared by the step kernels (mg_step.cu) and the fused task step
// (mg_task.cu): commands from the action cursor, k RK4 sub-steps in registers, optional
// trajectory record, and the launch-completion count that advances the device-side cursor.
#pragma once

#include "mg_device.cuh"

namespace mg {

// Register caps: the narrow diagonal-mass step keeps 128 registers (16 resident warps per SM,
// for the per-step form and large per-step grids; about 100 bytes of the step coefficients
// spill to L1 at this cap); the general step keeps 168.
constexpr int kRegsDiag = 128;
constexpr int kRegsGeneral = 168;
// The wide diagonal-mass variants (mg_set_schedule's wide): the work-queue kernel runs at 8
// warps/SM, where 256 registers per thread would fit; a 200 cap measured best (ptxas uses 181;
// +1.7 % over 168, none at 255).  The static-grid kernel with the same cap runs small fleets
// (one warp per scheduler or fewer, latency-bound) 6-7 % faster than at 128: the extra
// registers let the compiler interleave more independent work.
constexpr int kRegsWide = 200;
// With the off-diagonal hydrodynamics the 45 extra coefficients stay in registers too (no
// spills up to 255; 8 resident warps per SM).
constexpr int kRegsXH = 255;

// Action cursor at the start of the launch's mg_step call (read through L2: the previous call's
// last block wrote it).
__device__ __forceinline__ int64_t launch_cursor(const FleetView &fv) {
  return (int64_t)__ldcg(reinterpret_cast<const unsigned long long *>(fv.cursor));
}

// Called by every thread of every block once it is done: the last block to finish advances the
// cursor by k and re-arms the counter.  Every block read the cursor before it counted itself
// finished, so all of them saw the launch's starting value.
__device__ __forceinline__ void finish_launch(const FleetView &fv, int32_t k) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(fv.done_blocks, 1u);
    if (prev == gridDim.x - 1) {
      atomicAdd(reinterpret_cast<unsigned long long *>(fv.cursor), (unsigned long long)k);
      atomicExch(fv.done_blocks, 0u);
      __threadfence();
    }
  }
}

// Static-grid form of finish_launch, for kernels whose idle threads have already returned (no
// block barrier possible): each warp adds its live lanes to the block's shared counter s_done
// (zeroed before the block's first barrier); the warp that completes the block's count of live
// envs adds one finished block to the grid's counter, and the block that completes the grid
// advances the cursor by k and re-arms the counter.  Every thread read the cursor before its
// warp counted itself, so every block saw the launch's starting value.
__device__ __forceinline__ void finish_envs(const FleetView &fv, unsigned *s_done, int count,
                                            int32_t k) {
  const unsigned mask = __activemask();
  __syncwarp(mask);
  if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
    const unsigned add = __popc(mask);
    if (atomicAdd(s_done, add) + add == (unsigned)count &&
        atomicAdd(fv.done_blocks, 1u) == gridDim.x - 1) {
      atomicAdd(reinterpret_cast<unsigned long long *>(fv.cursor), (unsigned long long)k);
      atomicExch(fv.done_blocks, 0u);
    }
  }
}

// Stage a block's off-diagonal hydrodynamic coefficients in shared memory: row t of sx (stride
// MG_NXPARAM, coprime with the 32 banks) receives env env0 + t's coefficients from the
// component-major planes xh [MG_NXPARAM][n] (each component read coalesced).
__device__ __forceinline__ void stage_xh(const float *__restrict__ xh, int64_t n, int64_t env0,
                                         int count, float *sx) {
  for (int c = 0; c < MG_NXPARAM; ++c)
    for (int t = threadIdx.x; t < count; t += blockDim.x)
      sx[t * MG_NXPARAM + c] = __ldg(xh + (int64_t)c * n + env0 + t);
}

template <int MT>
__device__ __forceinline__ void load_commands(const FleetView &fv, int64_t e, int64_t seg,
                                              int nt, float itau, float (&c)[MT]) {
  if (fv.proc) {
    procedural_commands<MT>(fv.cmd_seed, (uint64_t)(fv.gid0 + e), seg, c);
  } else if (fv.n_seg > 0) {
    const int64_t sg = seg < fv.n_seg - 1 ? seg : fv.n_seg - 1;
    if (MT == 6 && fv.act_w == 6) {
      // 24-byte rows (no padding): three 8-byte loads; a warp's rows are 768 contiguous bytes
      const float2 *a = reinterpret_cast<const float2 *>(fv.act + (sg * fv.n + e) * 6);
      const float2 x = __ldg(a), y = __ldg(a + 1), z = __ldg(a + 2);
      c[0] = x.x; c[1] = x.y; c[2] = y.x; c[3] = y.y; c[4] = z.x; c[5] = z.y;
    } else {
      const float4 *a = reinterpret_cast<const float4 *>(fv.act + (sg * fv.n + e) * MG_MAX_THR);
      const float4 lo = __ldg(a), hi = __ldg(a + 1);
      c[0] = lo.x; c[1] = lo.y; c[2] = lo.z; c[3] = lo.w; c[4] = hi.x; c[5] = hi.y;
      if constexpr (MT > 6) {
        c[6] = hi.z;
        c[7] = hi.w;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < MT; ++i) c[i] = 0.f;
  }
  // Entries past the vehicle's thruster count are ignored (the lag state there stays zero).
  // The step reads the command divided by the lag time constant.
#pragma unroll
  for (int i = 0; i < MT; ++i) c[i] = (i < nt) ? c[i] * itau : 0.f;
}

template <int MT>
__device__ __forceinline__ void record(float *__restrict__ traj, int64_t n, int64_t e,
                                       const St<MT> &s) {
  float *t = traj + e;
  t[0 * n] = s.p[0]; t[1 * n] = s.p[1]; t[2 * n] = s.p[2];
  t[3 * n] = s.q[0]; t[4 * n] = s.q[1]; t[5 * n] = s.q[2]; t[6 * n] = s.q[3];
  t[7 * n] = s.v[0]; t[8 * n] = s.v[1]; t[9 * n] = s.v[2];
  t[10 * n] = s.w[0]; t[11 * n] = s.w[1]; t[12 * n] = s.w[2];
}

template <int MT>
__device__ __forceinline__ bool all_finite(const St<MT> &s) {
  // x * 0 is 0 for finite x and NaN for +-Inf or NaN, so the sum is 0 exactly when all are
  // finite.
  float z = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) z += s.p[i] * 0.f + s.v[i] * 0.f + s.w[i] * 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) z += s.q[i] * 0.f;
#pragma unroll
  for (int i = 0; i < MT; ++i) z += s.n[i] * 0.f;
  return z == 0.f;
}

// Advance env e by k sub-steps starting at action-cursor position step0, leaving the result in
// s (the caller stores it: store_and_flag, or a fused epilogue).  L2: state loads bypass L1
// (work-queue schedule, where another SM may have written them).
// XH: xh is the env's row of staged off-diagonal hydrodynamic coefficients.  CF: the throttle
// lag in closed form (rk4_step_lag: fewer operations, one more live constant); the fused task
// kernel's 128-register variants keep the classic update (rk4_step), which fits their epilogue
// without spilling.  Both are RK4; they differ in the rounding of the lag state.
template <int MT, bool DIAG, bool MIXED, bool REC, bool L2, int NH, bool XH = false,
          bool CF = true>
__device__ __forceinline__ void advance_env(const FleetView &fv, int64_t e, int nt,
                                            const float4 *gdir, const float4 *garm,
                                            int64_t step0, int32_t k, float *traj, St<MT> &s,
                                            const float *xh = nullptr) {
  const bool current_accel = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);
  const float h = fv.dt;

  load_state<MT, L2>(fv.st, e, s);
  Coef<DIAG> P;
  {
    Par<DIAG> raw;
    load_par<DIAG>(fv.pa, e, raw);
    P = make_coef<DIAG>(raw);
  }

  // Action cursor: sub-step j uses segment j / hold (clamped to the last buffered segment).
  int64_t seg = step0 / fv.hold;
  int32_t left = fv.hold - (int32_t)(step0 - seg * fv.hold);
  const LagEnv L = lag_env(P.itau, h);
  float b[MT];  // CF: b_i = (h/2) c_i / tau_m; otherwise c_i / tau_m
  {
    float c[MT];
    load_commands<MT>(fv, e, seg, nt, P.itau, c);
    if constexpr (CF) lag_segment<MT>(c, L, b);
    else
#pragma unroll
      for (int i = 0; i < MT; ++i) b[i] = c[i];
  }

  for (int32_t it = 0; it < k; ++it) {
    if (left == 0) {
      ++seg;
      left = fv.hold;
      float c[MT];
      load_commands<MT>(fv, e, seg, nt, P.itau, c);
      if constexpr (CF) lag_segment<MT>(c, L, b);
      else
#pragma unroll
        for (int i = 0; i < MT; ++i) b[i] = c[i];
    }
    if constexpr (CF)
      rk4_step_lag<MT, DIAG, MIXED, NH, XH>(s, b, L, P, gdir, garm, nt, current_accel, h, xh);
    else
      rk4_step<MT, DIAG, MIXED, NH, XH>(s, b, P, gdir, garm, nt, current_accel, h, xh);
    --left;
    if constexpr (REC) record<MT>(traj + (int64_t)it * MG_NTRAJ * fv.n, fv.n, e, s);
  }
}

// Mark env e non-finite (flag bit 0, counted once) unless already marked.  L2: the flag is read
// through L2 (work-queue schedule).
template <bool L2>
__device__ __forceinline__ void flag_nonfinite(const FleetView &fv, int64_t e) {
  const uint32_t old = L2 ? __ldcg(fv.flags + e) : fv.flags[e];
  if (!(old & 1u)) {
    fv.flags[e] = old | 1u;
    atomicAdd(fv.counters, 1ull);
  }
}

template <int MT, bool L2>
__device__ __forceinline__ void store_and_flag(const FleetView &fv, int64_t e, const St<MT> &s) {
  store_state<MT>(fv.st, e, s);
  if (!all_finite<MT>(s)) flag_nonfinite<L2>(fv, e);
}

}  // namespace mg
