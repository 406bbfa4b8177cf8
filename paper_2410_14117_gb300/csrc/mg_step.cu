// Fleet step kernel: one thread per vehicle, k RK4 sub-steps of Eq. 1 (§METHOD) per launch with
// the state and parameters held in registers.  k = 1 is the plain per-step form (state and
// parameters read from and written to HBM every sub-step); k > 1 is the persistent form (read
// once, stepped k times, written once).
//
// Each block covers envs of a single vehicle type (its BlockDesc), so the thruster geometry is a
// block-wide broadcast from shared memory and no warp diverges on the type.
#include <type_traits>

#include "mg_device.cuh"

namespace mg {

namespace {

constexpr int kMaxThreads = 256;
// Register caps: the diagonal-mass step fits 128 registers (16 resident warps per SM, so a
// 65,536-env fleet runs in a single wave on 152 SMs); the general step keeps 168.
constexpr int kRegsDiag = 128;
constexpr int kRegsGeneral = 168;

template <int MT>
__device__ __forceinline__ void load_commands(const FleetView &fv, int64_t e, int64_t seg,
                                              int nt, float (&c)[MT]) {
  if (fv.proc) {
    const uint64_t gid = (uint64_t)(fv.gid0 + e);
    const uint4 a = draw4(fv.cmd_seed, gid, STREAM_CMD, (uint32_t)(2 * seg));
    c[0] = 2.f * u01f(a.x) - 1.f; c[1] = 2.f * u01f(a.y) - 1.f;
    c[2] = 2.f * u01f(a.z) - 1.f; c[3] = 2.f * u01f(a.w) - 1.f;
    const uint4 b = draw4(fv.cmd_seed, gid, STREAM_CMD, (uint32_t)(2 * seg + 1));
    c[4] = 2.f * u01f(b.x) - 1.f; c[5] = 2.f * u01f(b.y) - 1.f;
    if constexpr (MT > 6) {
      c[6] = 2.f * u01f(b.z) - 1.f;
      c[7] = 2.f * u01f(b.w) - 1.f;
    }
  } else if (fv.n_seg > 0) {
    const int64_t sg = seg < fv.n_seg - 1 ? seg : fv.n_seg - 1;
    const float4 *a = fv.act + (sg * fv.n + e) * 2;
    const float4 lo = __ldg(a), hi = __ldg(a + 1);
    c[0] = lo.x; c[1] = lo.y; c[2] = lo.z; c[3] = lo.w; c[4] = hi.x; c[5] = hi.y;
    if constexpr (MT > 6) {
      c[6] = hi.z;
      c[7] = hi.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < MT; ++i) c[i] = 0.f;
  }
  // Entries past the vehicle's thruster count are ignored (the lag state there stays zero).
#pragma unroll
  for (int i = 0; i < MT; ++i)
    if (i >= nt) c[i] = 0.f;
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

template <int NTV, bool DIAG, bool REC>
__global__ void __maxnreg__(DIAG ? kRegsDiag : kRegsGeneral)
    k_fleet(const FleetView fv, const BlockDesc *__restrict__ blocks, const int64_t step0,
            const int32_t k, float *__restrict__ traj) {
  constexpr int MT = (NTV == NT_6) ? 6 : 8;
  constexpr bool MIXED = (NTV == NT_MIXED);
  __shared__ float4 sdir[MG_MAX_THR], sarm[MG_MAX_THR];

  const BlockDesc bd = blocks[blockIdx.x];
  if (threadIdx.x < MG_MAX_THR) {
    sdir[threadIdx.x] = fv.geo[bd.type].dir[threadIdx.x];
    sarm[threadIdx.x] = fv.geo[bd.type].arm[threadIdx.x];
  }
  __syncthreads();
  if ((int)threadIdx.x >= bd.count) return;

  const int64_t e = (int64_t)bd.env0 + threadIdx.x;
  const int nt = MIXED ? bd.n_thr : MT;
  const bool current_accel = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);
  const float h = fv.dt;

  St<MT> s;
  load_state<MT>(fv.st, e, s);
  Par<DIAG> P;
  load_par<DIAG>(fv.pa, e, P);

  // Action cursor: sub-step j uses segment j / hold (clamped to the last buffered segment).
  int64_t seg = step0 / fv.hold;
  int32_t left = fv.hold - (int32_t)(step0 - seg * fv.hold);
  float c[MT];
  load_commands<MT>(fv, e, seg, nt, c);

  for (int32_t it = 0; it < k; ++it) {
    if (left == 0) {
      ++seg;
      left = fv.hold;
      load_commands<MT>(fv, e, seg, nt, c);
    }
    rk4_step<MT, DIAG, MIXED>(s, c, P, sdir, sarm, nt, current_accel, h);
    --left;
    if constexpr (REC) record<MT>(traj + (int64_t)it * MG_NTRAJ * fv.n, fv.n, e, s);
  }

  store_state<MT>(fv.st, e, s);
  if (!all_finite<MT>(s)) {
    const uint32_t old = fv.flags[e];
    if (!(old & 1u)) {
      fv.flags[e] = old | 1u;
      atomicAdd(fv.nonfinite_count, 1ull);
    }
  }
}

template <int NTV, bool DIAG, bool REC>
cudaError_t launch_t(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                     int64_t step0, int32_t k, float *traj, cudaStream_t stream) {
  k_fleet<NTV, DIAG, REC><<<n_blocks, threads, 0, stream>>>(fv, blocks, step0, k, traj);
  return cudaGetLastError();
}

template <int NTV, bool DIAG>
cudaError_t launch_r(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                     int64_t step0, int32_t k, float *traj, cudaStream_t stream) {
  return traj ? launch_t<NTV, DIAG, true>(fv, blocks, n_blocks, threads, step0, k, traj, stream)
              : launch_t<NTV, DIAG, false>(fv, blocks, n_blocks, threads, step0, k, traj, stream);
}

template <int NTV>
cudaError_t launch_d(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                     bool diag, int64_t step0, int32_t k, float *traj, cudaStream_t stream) {
  return diag ? launch_r<NTV, true>(fv, blocks, n_blocks, threads, step0, k, traj, stream)
              : launch_r<NTV, false>(fv, blocks, n_blocks, threads, step0, k, traj, stream);
}

template <int NTV, bool DIAG, bool REC>
const void *kernel_ptr() {
  return reinterpret_cast<const void *>(&k_fleet<NTV, DIAG, REC>);
}

}  // namespace

cudaError_t launch_fleet(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                         NtVariant ntv, bool diag, int64_t step0, int32_t k, float *traj,
                         cudaStream_t stream) {
  if (threads < 32 || threads > kMaxThreads || threads % 32 || n_blocks < 1) return cudaErrorInvalidValue;
  switch (ntv) {
    case NT_6: return launch_d<NT_6>(fv, blocks, n_blocks, threads, diag, step0, k, traj, stream);
    case NT_8: return launch_d<NT_8>(fv, blocks, n_blocks, threads, diag, step0, k, traj, stream);
    default:
      return launch_d<NT_MIXED>(fv, blocks, n_blocks, threads, diag, step0, k, traj, stream);
  }
}

cudaError_t fleet_kernel_attributes(NtVariant ntv, bool diag, bool rec,
                                    cudaFuncAttributes *attr) {
  const void *f = nullptr;
#define MG_PICK(N)                                                                  \
  f = diag ? (rec ? kernel_ptr<N, true, true>() : kernel_ptr<N, true, false>())     \
           : (rec ? kernel_ptr<N, false, true>() : kernel_ptr<N, false, false>());
  switch (ntv) {
    case NT_6: MG_PICK(NT_6) break;
    case NT_8: MG_PICK(NT_8) break;
    default: MG_PICK(NT_MIXED) break;
  }
#undef MG_PICK
  return cudaFuncGetAttributes(attr, f);
}

}  // namespace mg
