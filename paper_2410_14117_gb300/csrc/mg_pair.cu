// Packed static-grid step kernel (k_fleet_pair): two vehicles per thread, every operation of the
// RK4 sub-step one FP32x2 instruction over the pair; the device code is in mg_pair.cuh.  A block
// of T threads covers 2T vehicles, thread t taking vehicles env0 + t and env0 + T + t.  (A
// work-queue form over 64-vehicle slices measured slower than this static grid at every fleet
// size and is not built.)
#include <algorithm>

#include "mg_pair.cuh"

namespace mg {

namespace {

template <int NTV, int NH>
__global__ void __maxnreg__(kRegsPair)
    k_fleet_pair(const FleetView fv, const BlockDesc *__restrict__ blocks, const int32_t k) {
  constexpr int MT = (NTV == NT_6) ? 6 : 8;
  constexpr bool MIXED = (NTV == NT_MIXED);
  __shared__ GeoPair sg;
  __shared__ unsigned s_done;
  __shared__ int64_t s_cursor;

  const BlockDesc bd = blocks[blockIdx.x];
  if (threadIdx.x < MG_MAX_THR) stage_geo_pair(fv.geo[bd.type], sg, threadIdx.x);
  // Programmatic dependent launch, as k_fleet: nothing above depends on the previous launch.
  cudaTriggerProgrammaticLaunchCompletion();
  cudaGridDependencySynchronize();
  if (threadIdx.x == 0) {
    s_done = 0u;
    s_cursor = launch_cursor(fv);
  }
  __syncthreads();
  const int T = (int)blockDim.x;
  const int live = min(bd.count, T);
  if ((int)threadIdx.x >= live) return;
  const int64_t ea = (int64_t)bd.env0 + threadIdx.x;
  const bool has_b = T + (int)threadIdx.x < bd.count;
  const int64_t eb = has_b ? ea + T : ea;
  St<MT> sa, sb;
  advance_pair<MT, false, NH>(fv, ea, eb, MIXED ? bd.n_thr : MT, sg, s_cursor + fv.cursor_off, k,
                              sa, sb);
  store_and_flag<MT, false>(fv, ea, sa);
  if (has_b) store_and_flag<MT, false>(fv, eb, sb);
  if (fv.cursor_adv) finish_envs(fv, &s_done, live, fv.cursor_adv);
}

template <typename Kernel>
cudaError_t launch_pdl_pair(Kernel kernel, int n_blocks, int threads, cudaStream_t stream,
                            const FleetView &fv, const BlockDesc *blocks, int32_t k) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)n_blocks);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, fv, blocks, k);
}

template <int NTV>
const void *pair_ptr(bool structured) {
  return structured ? reinterpret_cast<const void *>(&k_fleet_pair<NTV, 4>)
                    : reinterpret_cast<const void *>(&k_fleet_pair<NTV, 0>);
}

const void *pick_pair(NtVariant ntv, bool structured) {
  switch (ntv) {
    case NT_6: return pair_ptr<NT_6>(structured);
    case NT_8: return pair_ptr<NT_8>(structured);
    default: return pair_ptr<NT_MIXED>(structured);
  }
}

template <int NTV>
cudaError_t launch_pair_t(const FleetView &fv, const BlockDesc *blocks, int n_blocks,
                          int threads, bool structured, int32_t k, cudaStream_t stream) {
  return structured
             ? launch_pdl_pair(k_fleet_pair<NTV, 4>, n_blocks, threads, stream, fv, blocks, k)
             : launch_pdl_pair(k_fleet_pair<NTV, 0>, n_blocks, threads, stream, fv, blocks, k);
}

}  // namespace

cudaError_t launch_fleet_pair(const FleetView &fv, const BlockDesc *blocks, int n_blocks,
                              int threads, NtVariant ntv, bool structured, int32_t k,
                              cudaStream_t stream) {
  if (threads < 32 || threads > 256 || threads % 32 || n_blocks < 1 || k < 1 || fv.xh)
    return cudaErrorInvalidValue;
  switch (ntv) {
    case NT_6: return launch_pair_t<NT_6>(fv, blocks, n_blocks, threads, structured, k, stream);
    case NT_8: return launch_pair_t<NT_8>(fv, blocks, n_blocks, threads, structured, k, stream);
    default:
      return launch_pair_t<NT_MIXED>(fv, blocks, n_blocks, threads, structured, k, stream);
  }
}

cudaError_t pair_kernel_attributes(NtVariant ntv, bool structured, cudaFuncAttributes *attr) {
  return cudaFuncGetAttributes(attr, pick_pair(ntv, structured));
}

}  // namespace mg
