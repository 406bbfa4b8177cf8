// Fleet step kernels: one thread per vehicle advancing Eq. 1 (§METHOD) by RK4 sub-steps with
// the state and parameters held in registers.
//
// Two schedules share the per-vehicle loop (advance_env):
//   k_fleet        static grid, one block per BlockDesc, k sub-steps per launch.  k = 1 is the
//                  plain per-step form (state and parameters through HBM every sub-step); k > 1
//                  is the persistent form (read once, stepped k times, written once).
//   k_fleet_queue  one launch for all k sub-steps: each warp repeatedly claims a unit (one
//                  32-env slice, one chunk of sub-steps) from an atomic counter in chunk-major
//                  order, waits until that slice's previous chunk is done, and runs it.  Warps
//                  that run faster claim more units, so the work spreads evenly over the 608
//                  schedulers whatever the fleet size (a static grid of 65,536 envs gives 3 or 4
//                  warps to each scheduler and idles the 3-warp ones for a quarter of the time).
//
// Blocks / slices cover envs of a single vehicle type, so the thruster geometry is a broadcast
// from shared memory and no warp diverges on the type.  Fleets whose types have different
// thruster counts run the 8-thruster loop for every env ("padded"): absent thrusters have zero
// direction and arm and zero command, so they add exact zeros.
#include <algorithm>
#include <type_traits>

#include "mg_advance.cuh"

namespace mg {

namespace {

constexpr int kMaxThreads = 256;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// XH: off-diagonal hydrodynamics (general path), the block's coefficients staged in dynamic
// shared memory [blockDim.x][MG_NXPARAM].  WIDE (diagonal mass, no recording): 200 registers.
template <int NTV, bool DIAG, bool REC, int NH, bool XH = false, bool WIDE = false>
__global__ void __maxnreg__(XH ? kRegsXH : !DIAG ? kRegsGeneral : WIDE ? kRegsWide : kRegsDiag)
    k_fleet(const FleetView fv, const BlockDesc *__restrict__ blocks, const int32_t k,
            float *__restrict__ traj) {
  constexpr int MT = (NTV == NT_6) ? 6 : 8;
  constexpr bool MIXED = (NTV == NT_MIXED);
  __shared__ float4 sdir[MG_MAX_THR], sarm[MG_MAX_THR];
  __shared__ unsigned s_done;
  __shared__ int64_t s_cursor;
  extern __shared__ float sxh[];

  const BlockDesc bd = blocks[blockIdx.x];
  if (threadIdx.x < MG_MAX_THR) {
    sdir[threadIdx.x] = fv.geo[bd.type].dir[threadIdx.x];
    sarm[threadIdx.x] = fv.geo[bd.type].arm[threadIdx.x];
  }
  // Programmatic dependent launch: the next launch in the stream may start (and run up to its
  // own wait) now; everything above reads only buffers written before any step launch, and
  // everything below waits for the previous launch in the stream to complete.
  cudaTriggerProgrammaticLaunchCompletion();
  cudaGridDependencySynchronize();
  if (threadIdx.x == 0) {
    s_done = 0u;
    s_cursor = launch_cursor(fv);
  }
  if constexpr (XH) stage_xh(fv.xh, fv.n, bd.env0, bd.count, sxh);
  __syncthreads();
  if ((int)threadIdx.x >= bd.count) return;
  const int64_t e = (int64_t)bd.env0 + threadIdx.x;
  St<MT> st;
  advance_env<MT, DIAG, MIXED, REC, false, NH, XH>(fv, e, MIXED ? bd.n_thr : MT, sdir, sarm,
                                                   s_cursor + fv.cursor_off, k, traj, st,
                                                   XH ? sxh + threadIdx.x * MG_NXPARAM
                                                      : nullptr);
  store_and_flag<MT, false>(fv, e, st);
  if (fv.cursor_adv) finish_envs(fv, &s_done, bd.count, fv.cursor_adv);
}

// XH (general path): each warp stages the off-diagonal hydrodynamic coefficients of the slice it
// claimed into its own rows of dynamic shared memory [kQueueWarps * 32][MG_NXPARAM] (every lane
// writes and reads only its own row, so program order suffices).
template <int NTV, bool DIAG, bool WIDE, int NH, bool XH = false>
__global__ void __maxnreg__(XH ? kRegsXH : !DIAG ? kRegsGeneral : WIDE ? kRegsWide : kRegsDiag)
    k_fleet_queue(const FleetView fv, const BlockDesc *__restrict__ slices, const int32_t n_slices,
                  const int32_t k_total, const int32_t chunk, uint32_t *__restrict__ sched) {
  static_assert(!(XH && DIAG), "the off-diagonal hydrodynamics use the general path");
  extern __shared__ float sxh[];
  constexpr int MT = (NTV == NT_6) ? 6 : 8;
  constexpr bool MIXED = (NTV == NT_MIXED);
  // Thruster geometry of every vehicle type at fixed shared addresses (a per-warp copy at a
  // run-time address costs the sub-step loop dozens of registers).
  __shared__ float4 sgeo[MG_MAX_TYPES][2 * MG_MAX_THR];
  for (int i = threadIdx.x; i < fv.n_types * 2 * MG_MAX_THR; i += blockDim.x) {
    const int t = i / (2 * MG_MAX_THR), j = i % (2 * MG_MAX_THR);
    sgeo[t][j] = j < MG_MAX_THR ? fv.geo[t].dir[j] : fv.geo[t].arm[j - MG_MAX_THR];
  }
  const int64_t step0 = launch_cursor(fv) + fv.cursor_off;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t n_chunks = (uint32_t)((k_total + chunk - 1) / chunk);
  const uint32_t n_units = (uint32_t)n_slices * n_chunks;  // < 2^31, checked by the launcher

  for (;;) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(sched, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= n_units) break;
    const int32_t c = (int32_t)(u / (uint32_t)n_slices);
    const int32_t d = (int32_t)(u % (uint32_t)n_slices);
    if (c > 0 && lane == 0) {
      // The slice's previous chunk was claimed earlier by a running warp, so it completes.  The
      // wait is bounded (fv.spin_limit polls of ~128 ns, MG_WAIT_POLLS_DEFAULT unless set by
      // mg_set_wait_limit): on expiry it is counted as a time-out and the unit proceeds.
      uint32_t polls = 0;
      while (ld_acquire(sched + 4 + d) < (uint32_t)c) {
        if (++polls > fv.spin_limit) {
          atomicAdd(fv.counters + 2, 1ull);
          break;
        }
        __nanosleep(128);
      }
    }
    __syncwarp();
    const BlockDesc bd = slices[d];
    const float4 *gdir = sgeo[bd.type & (MG_MAX_TYPES - 1)], *garm = gdir + MG_MAX_THR;
    if (lane < bd.count) {
      const int64_t e = (int64_t)bd.env0 + lane;
      float *row = sxh + threadIdx.x * MG_NXPARAM;
      if constexpr (XH)
        for (int j = 0; j < MG_NXPARAM; ++j) row[j] = __ldg(fv.xh + (int64_t)j * fv.n + e);
      St<MT> st;
      advance_env<MT, DIAG, MIXED, false, true, NH, XH>(fv, e, MIXED ? bd.n_thr : MT, gdir, garm,
                                                        step0 + (int64_t)c * chunk,
                                                        min(chunk, k_total - c * chunk),
                                                        nullptr, st, XH ? row : nullptr);
      store_and_flag<MT, true>(fv, e, st);
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      st_release(sched + 4 + d, (uint32_t)(c + 1));
    }
  }
  if (fv.cursor_adv) finish_launch(fv, fv.cursor_adv);
}

// Launch a static-grid step kernel with programmatic stream serialisation: it may begin while
// the previous kernel in the stream finishes (see the wait in k_fleet).
template <typename Kernel>
cudaError_t launch_pdl(Kernel kernel, int n_blocks, int threads, size_t smem, cudaStream_t stream,
                       const FleetView &fv, const BlockDesc *blocks, int32_t k, float *traj) {
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
  return cudaLaunchKernelEx(&cfg, kernel, fv, blocks, k, traj);
}

// Structured allocation (NH = 4) is only instantiated for the diagonal-mass step, the
// off-diagonal hydrodynamics (XH) only for the general one, the wide register budget only for
// the diagonal-mass step without recording.
template <int NTV, bool DIAG, bool REC, bool WIDE>
cudaError_t launch_t(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                     bool structured, int32_t k, float *traj, cudaStream_t stream) {
  if constexpr (!DIAG) if (fv.xh)
    return launch_pdl(k_fleet<NTV, false, REC, 0, true>, n_blocks, threads,
                      sizeof(float) * MG_NXPARAM * threads, stream, fv, blocks, k, traj);
  if (DIAG && structured)
    return launch_pdl(k_fleet<NTV, DIAG, REC, (DIAG ? 4 : 0), false, WIDE>, n_blocks, threads,
                      0, stream, fv, blocks, k, traj);
  return launch_pdl(k_fleet<NTV, DIAG, REC, 0, false, WIDE>, n_blocks, threads, 0, stream, fv,
                    blocks, k, traj);
}

template <int NTV, bool DIAG>
cudaError_t launch_r(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                     bool structured, bool wide, int32_t k, float *traj, cudaStream_t stream) {
  if (traj)
    return launch_t<NTV, DIAG, true, false>(fv, blocks, n_blocks, threads, structured, k, traj,
                                            stream);
  if constexpr (DIAG)
    if (wide)
      return launch_t<NTV, true, false, true>(fv, blocks, n_blocks, threads, structured, k,
                                              traj, stream);
  return launch_t<NTV, DIAG, false, false>(fv, blocks, n_blocks, threads, structured, k, traj,
                                           stream);
}

template <int NTV>
cudaError_t launch_d(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                     bool diag, bool structured, bool wide, int32_t k, float *traj,
                     cudaStream_t stream) {
  return diag ? launch_r<NTV, true>(fv, blocks, n_blocks, threads, structured, wide, k, traj,
                                    stream)
              : launch_r<NTV, false>(fv, blocks, n_blocks, threads, structured, wide, k, traj,
                                     stream);
}

template <int NTV, bool DIAG, bool REC, bool WIDE = false>
const void *kernel_ptr(bool structured) {
  if (DIAG && structured)
    return reinterpret_cast<const void *>(&k_fleet<NTV, DIAG, REC, (DIAG ? 4 : 0), false, WIDE>);
  return reinterpret_cast<const void *>(&k_fleet<NTV, DIAG, REC, 0, false, WIDE>);
}

template <int NTV, bool DIAG>
const void *queue_ptr(bool wide, bool structured, bool xh) {
  constexpr int S = DIAG ? 4 : 0;
  if constexpr (!DIAG)
    if (xh) return reinterpret_cast<const void *>(&k_fleet_queue<NTV, false, false, 0, true>);
  if (DIAG && structured)
    return wide ? reinterpret_cast<const void *>(&k_fleet_queue<NTV, DIAG, true, S>)
                : reinterpret_cast<const void *>(&k_fleet_queue<NTV, DIAG, false, S>);
  return wide ? reinterpret_cast<const void *>(&k_fleet_queue<NTV, DIAG, true, 0>)
              : reinterpret_cast<const void *>(&k_fleet_queue<NTV, DIAG, false, 0>);
}

const void *queue_kernel(NtVariant ntv, bool diag, bool wide, bool structured, bool xh) {
  switch (ntv) {
    case NT_6:
      return diag ? queue_ptr<NT_6, true>(wide, structured, false)
                  : queue_ptr<NT_6, false>(wide, false, xh);
    case NT_8:
      return diag ? queue_ptr<NT_8, true>(wide, structured, false)
                  : queue_ptr<NT_8, false>(wide, false, xh);
    default:
      return diag ? queue_ptr<NT_MIXED, true>(wide, structured, false)
                  : queue_ptr<NT_MIXED, false>(wide, false, xh);
  }
}

// Dynamic shared memory of the XH work-queue kernel (one coefficient row per thread).
constexpr size_t kQueueXhBytes = sizeof(float) * kQueueWarps * 32 * MG_NXPARAM;

template <int NTV, bool DIAG, int NH>
void queue_launch_w(bool wide, int grid, const FleetView &fv, const BlockDesc *slices,
                    int32_t n_slices, int32_t k, int32_t chunk, uint32_t *sched,
                    cudaStream_t stream) {
  if constexpr (!DIAG)
    if (fv.xh) {
      k_fleet_queue<NTV, false, false, 0, true><<<grid, kQueueWarps * 32, kQueueXhBytes, stream>>>(
          fv, slices, n_slices, k, chunk, sched);
      return;
    }
  if (wide)
    k_fleet_queue<NTV, DIAG, true, NH><<<grid, kQueueWarps * 32, 0, stream>>>(
        fv, slices, n_slices, k, chunk, sched);
  else
    k_fleet_queue<NTV, DIAG, false, NH><<<grid, kQueueWarps * 32, 0, stream>>>(
        fv, slices, n_slices, k, chunk, sched);
}

template <int NTV>
void queue_launch(bool diag, bool wide, bool structured, int grid, const FleetView &fv,
                  const BlockDesc *slices, int32_t n_slices, int32_t k, int32_t chunk,
                  uint32_t *sched, cudaStream_t stream) {
  if (diag && structured)
    queue_launch_w<NTV, true, 4>(wide, grid, fv, slices, n_slices, k, chunk, sched, stream);
  else if (diag)
    queue_launch_w<NTV, true, 0>(wide, grid, fv, slices, n_slices, k, chunk, sched, stream);
  else
    queue_launch_w<NTV, false, 0>(wide, grid, fv, slices, n_slices, k, chunk, sched, stream);
}

}  // namespace

cudaError_t launch_fleet(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                         NtVariant ntv, bool diag, bool structured, bool wide, int32_t k,
                         float *traj, cudaStream_t stream) {
  if (threads < 32 || threads > kMaxThreads || threads % 32 || n_blocks < 1 || k < 1 ||
      (fv.xh && diag))
    return cudaErrorInvalidValue;
  switch (ntv) {
    case NT_6:
      return launch_d<NT_6>(fv, blocks, n_blocks, threads, diag, structured, wide, k, traj,
                            stream);
    case NT_8:
      return launch_d<NT_8>(fv, blocks, n_blocks, threads, diag, structured, wide, k, traj,
                            stream);
    default:
      return launch_d<NT_MIXED>(fv, blocks, n_blocks, threads, diag, structured, wide, k, traj,
                                stream);
  }
}

cudaError_t fleet_kernel_attributes(NtVariant ntv, bool diag, bool structured, bool rec,
                                    bool wide, cudaFuncAttributes *attr) {
  const void *f = nullptr;
#define MG_PICK(N)                                                                      \
  f = diag ? (rec ? kernel_ptr<N, true, true>(structured)                               \
                  : wide ? kernel_ptr<N, true, false, true>(structured)                 \
                         : kernel_ptr<N, true, false>(structured))                      \
           : (rec ? kernel_ptr<N, false, true>(false) : kernel_ptr<N, false, false>(false));
  switch (ntv) {
    case NT_6: MG_PICK(NT_6) break;
    case NT_8: MG_PICK(NT_8) break;
    default: MG_PICK(NT_MIXED) break;
  }
#undef MG_PICK
  return cudaFuncGetAttributes(attr, f);
}

size_t queue_sched_bytes(int n_slices) { return 16 + 4 * (size_t)n_slices; }

cudaError_t queue_kernel_attributes(NtVariant ntv, bool diag, bool wide, bool structured,
                                    bool xh, cudaFuncAttributes *attr, int *blocks_per_sm) {
  xh = xh && !diag;
  const void *f = queue_kernel(ntv, diag, wide, structured, xh);
  cudaError_t e = cudaFuncGetAttributes(attr, f);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, kQueueWarps * 32,
                                                       xh ? kQueueXhBytes : 0);
}

cudaError_t launch_fleet_queue(const FleetView &fv, const BlockDesc *slices, int n_slices,
                               NtVariant ntv, bool diag, bool structured, bool wide,
                               int warps_per_sm, int32_t k, int32_t chunk, uint32_t *sched,
                               int n_sm, cudaStream_t stream) {
  if (n_slices < 1 || k < 1 || chunk < 1 || n_sm < 1 || (fv.xh && diag))
    return cudaErrorInvalidValue;
  cudaFuncAttributes attr;
  int per_sm = 0;
  cudaError_t e = queue_kernel_attributes(ntv, diag, wide, structured, fv.xh != nullptr, &attr,
                                          &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  // Resident warps: at most what fits (and at most warps_per_sm per SM when that is > 0), and no
  // more than there are slices in a chunk.
  if (warps_per_sm > 0) per_sm = std::max(1, std::min(per_sm, warps_per_sm / kQueueWarps));
  int grid = per_sm * n_sm;
  const int need = (n_slices + kQueueWarps - 1) / kQueueWarps;
  if (grid > need) grid = need;
  // One launch per piece of the horizon whose unit count fits the 31-bit counter.
  const int64_t max_chunks = ((int64_t)1 << 31) / n_slices;
  if (max_chunks < 1) return cudaErrorInvalidValue;
  for (int64_t done = 0; done < k;) {
    const int64_t left = k - done;
    const int32_t kk = (int32_t)std::min<int64_t>(left, max_chunks * (int64_t)chunk);
    e = cudaMemsetAsync(sched, 0, queue_sched_bytes(n_slices), stream);
    if (e != cudaSuccess) return e;
    FleetView piece = fv;  // this piece's offset in the call; only the last piece advances
    piece.cursor_off = fv.cursor_off + (int32_t)done;
    piece.cursor_adv = (done + kk == k) ? fv.cursor_adv : 0;
    switch (ntv) {
      case NT_6:
        queue_launch<NT_6>(diag, wide, structured, grid, piece, slices, n_slices, kk, chunk,
                           sched, stream);
        break;
      case NT_8:
        queue_launch<NT_8>(diag, wide, structured, grid, piece, slices, n_slices, kk, chunk,
                           sched, stream);
        break;
      default:
        queue_launch<NT_MIXED>(diag, wide, structured, grid, piece, slices, n_slices, kk, chunk,
                               sched, stream);
        break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    done += kk;
  }
  return cudaSuccess;
}

}  // namespace mg
