// Host side of the C ABI declared in include/mg.h.
//
// A sim owns one device arena holding the state planes, the raw parameter records, the derived
// parameter planes, per-env flags and episode counters, the per-type thruster geometry and the
// block list; the action buffer and a staging buffer for host I/O are separate allocations that
// grow on demand.  Every device operation is issued on the sim's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mg_internal.h"

using namespace mg;

namespace {

thread_local std::string g_err;

mg_status fail(mg_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

}  // namespace

mg_status mg::set_error(mg_status st, const std::string &msg) { return fail(st, msg); }

bool mg::vectored_layout(const Geo &g) {
  if (g.n_thr < 4) return false;
  for (int i = 0; i < g.n_thr; ++i) {
    if (i < 4 && g.dir[i].z != 0.f) return false;
    if (i >= 4 && (g.dir[i].x != 0.f || g.dir[i].y != 0.f || g.arm[i].z != 0.f)) return false;
  }
  return true;
}

namespace {

mg_status fail_cuda(cudaError_t e, const char *what) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return fail(e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA, buf);
}

#define MG_CK(call)                                      \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return fail_cuda(_e, #call); \
  } while (0)

#define MG_NONNULL(p) \
  do {                \
    if (!(p)) return fail(MG_EINVAL, #p " is NULL"); \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// True when p can be dereferenced by a kernel (device or managed memory).
bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A captured mg_step launch sequence.  Besides k it bakes in the action source the kernels read
// (buffer, segment count, hold, procedural seed), so those are part of the key: alternating
// between action buffers replays cached graphs instead of capturing new ones.  Every other
// setting a capture depends on drops the cache when it changes.
struct GraphEntry {
  int32_t k;
  const float *act_src;
  int32_t n_seg, hold, proc;
  uint64_t cmd_seed;
  cudaGraphExec_t exec;
  uint64_t last_use;
};

}  // namespace

struct mg_sim {
  int dev = 0;
  int64_t n = 0;
  int32_t n_types = 0;
  std::vector<int32_t> types_h;
  std::vector<mg_vehicle_params> vp;
  NtVariant ntv = NT_6;
  // mass_diag: every env's M_RB + M_A is diagonal (r_g = 0, no off-diagonal extension).  diag:
  // the step kernels take the diagonal-mass path, whose coefficients also fold in the
  // current-acceleration term, so a sim that switches that term off takes the general path.
  bool mass_diag = true;
  bool diag = true;
  bool structured = false;  // every type present has the vectored thruster layout
  bool nominal_diag = true;  // every type has r_g = 0 (randomised M_RB + M_A stays diagonal)
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;

  // arena
  void *arena = nullptr;
  StatePlanes st{};
  ParamPlanes pa{};
  float *raw = nullptr;
  int32_t *types_d = nullptr;
  Geo *geo_d = nullptr;
  float *nominal_d = nullptr;
  uint32_t *flags = nullptr;
  uint32_t *episode = nullptr;
  unsigned long long *counters = nullptr;  // [0] non-finite envs, [1] non-SPD envs,
                                           // [2] work-queue wait time-outs, [3] action
                                           // cursor, [4] finished-block count
  unsigned int *offdiag = nullptr;
  // off-diagonal hydrodynamics, [MG_NXPARAM][n] planes (mg_set_hydro_offdiag), and whether set
  float *xh = nullptr;
  bool has_xh = false;
  // backward kernel (mg_set_adjoint_mode) and the two-warp form's workspace
  int32_t adj_mode = 0;
  float *adj_ws = nullptr;
  size_t adj_ws_cap = 0;
  // the arena's parameter range (derived planes, then the raw records): one contiguous span
  size_t par_off = 0, par_bytes = 0;

  // background randomisation (mg_randomize_prefetch): a second parameter range of the same
  // layout, followed by its own non-SPD count and off-diagonal word, drawn on the library's own
  // stream; pf_done orders the install after the draw, pf_consumed the next draw after the
  // install's copy.  Keyed by everything the draw depends on.  Created on first use.
  cudaStream_t pf_stream = nullptr;
  char *pf_buf = nullptr;
  cudaEvent_t pf_done = nullptr, pf_consumed = nullptr;
  bool pf_valid = false;
  uint64_t pf_seed = 0;
  float pf_lo = 0.f, pf_hi = 0.f, pf_current_sigma = 0.f;
  int64_t pf_gid0 = 0;

  // static-schedule blocks
  BlockDesc *blocks_d = nullptr;
  int n_blocks = 0;
  int threads = 128;
  // work-queue schedule: 32-env slices and the scheduler words
  BlockDesc *slices_d = nullptr;
  int n_slices = 0;
  uint32_t *sched = nullptr;
  int n_sm = 1;
  bool queue = false;
  bool wide = true;
  int32_t queue_warps_per_sm = 0;
  uint32_t wait_limit = MG_WAIT_POLLS_DEFAULT;  // bound on a work-queue wait (mg_set_wait_limit)

  // actions (act_src: what the kernels read — the sim's copy, or a caller's borrowed buffer)
  float *act = nullptr;
  const float *act_src = nullptr;
  size_t act_cap = 0;  // floats
  int32_t act_w = MG_MAX_THR;  // floats per env and segment of every action buffer
  int32_t n_seg = 0, hold = 1;
  int32_t proc = 0;
  uint64_t cmd_seed = 0;
  int64_t cursor = 0;  // host copy of the device cursor (counters[3])

  // knobs
  int32_t epb = 128, spl = 50;
  bool use_graph = true;
  float dt = 0.01f;
  uint32_t model_flags = 0;
  int64_t gid0 = 0;
  uint64_t reset_seed = 0;
  double nu0_sigma = 0.0;

  // staging for host I/O
  void *stage = nullptr;
  size_t stage_cap = 0;

  // asynchronous transfers from / to page-locked host memory (mg_set_actions_async,
  // mg_get_state_async): two device buffers each way, used alternately, with their own copy
  // streams; events order each copy after the last reader of its buffer and the sim's work after
  // the copy it needs.  Created on first use.
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  float *abuf[2] = {nullptr, nullptr};
  size_t abuf_cap[2] = {0, 0};  // floats
  cudaEvent_t a_copied[2] = {nullptr, nullptr}, a_released[2] = {nullptr, nullptr};
  int a_next = 0, a_active = -1;  // a_active: the slot the kernels read, or -1
  float *obuf[2] = {nullptr, nullptr};
  cudaEvent_t o_exported[2] = {nullptr, nullptr}, o_read[2] = {nullptr, nullptr};
  int o_next = 0;

  // task layer
  bool has_task = false;
  const void *task_out_ok[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // last validated
  // environment step (mg_env_step): the library's one-segment schedule of clamped throttles
  // [n][act_w], and the last validated action input
  float *env_act = nullptr;
  size_t env_act_cap = 0;  // floats
  const void *env_in_ok = nullptr;
  mg_task_spec task{};
  void *task_buf = nullptr;  // centre [n] float4, clock [n] int32, err_sum [n] float
  TaskView task_view() const {
    TaskView v{};
    v.task = task.task;
    v.m = task.lookahead;
    v.radius = task.radius;
    v.omega = task.omega;
    v.vz = task.vz;
    v.psi_r = task.psi_r;
    v.dt_look = task.lookahead_dt;
    v.max_err = task.max_error;
    v.episode_steps = task.episode_steps > 0 ? task.episode_steps : 0;
    char *b = static_cast<char *>(task_buf);
    v.centre = reinterpret_cast<const float4 *>(b);
    v.clock = reinterpret_cast<int32_t *>(b + 16 * n);
    v.err_sum = reinterpret_cast<float *>(b + 20 * n);
    return v;
  }

  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;

  FleetView view() const {
    FleetView v{};
    v.st = st;
    v.pa = pa;
    v.geo = geo_d;
    v.n_types = n_types;
    v.n = n;
    v.gid0 = gid0;
    v.act = act_src;
    v.act_w = act_w;
    v.n_seg = proc ? 0 : n_seg;
    v.hold = hold;
    v.cmd_seed = cmd_seed;
    v.proc = proc;
    v.model_flags = model_flags;
    v.dt = dt;
    v.flags = flags;
    v.counters = counters;
    v.xh = has_xh ? xh : nullptr;
    v.spin_limit = wait_limit;
    v.cursor = reinterpret_cast<int64_t *>(counters + 3);
    v.done_blocks = reinterpret_cast<unsigned int *>(counters + 4);
    return v;
  }

  SetupView setup_view() const {
    SetupView v{};
    v.n = n;
    v.gid0 = gid0;
    v.types = types_d;
    v.raw = raw;
    v.pa = pa;
    v.n_not_spd = counters + 1;
    v.any_offdiag = offdiag;
    v.xh = has_xh ? xh : nullptr;
    return v;
  }

  // setup_view() with every parameter pointer moved into the background range
  SetupView staged_setup_view() const {
    SetupView v = setup_view();
    const char *base = static_cast<const char *>(arena) + par_off;
    auto move = [&](auto *ptr) {
      return reinterpret_cast<decltype(ptr)>(pf_buf + (reinterpret_cast<const char *>(ptr) - base));
    };
    v.raw = move(v.raw);
    v.pa.d0 = move(v.pa.d0); v.pa.d1 = move(v.pa.d1); v.pa.d2 = move(v.pa.d2);
    v.pa.d3 = move(v.pa.d3); v.pa.d4 = move(v.pa.d4); v.pa.d5 = move(v.pa.d5);
    v.pa.d6 = move(v.pa.d6); v.pa.d7 = move(v.pa.d7); v.pa.d8 = move(v.pa.d8);
    v.pa.g0 = move(v.pa.g0); v.pa.g1 = move(v.pa.g1); v.pa.g2 = move(v.pa.g2);
    v.pa.g3 = move(v.pa.g3); v.pa.g4 = move(v.pa.g4); v.pa.g5 = move(v.pa.g5);
    v.n_not_spd = reinterpret_cast<unsigned long long *>(pf_buf + par_bytes);
    v.any_offdiag = reinterpret_cast<unsigned int *>(pf_buf + par_bytes + 8);
    return v;
  }

  void drop_graphs() {
    for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
};

namespace {

mg_status ensure_stage(mg_sim *s, size_t bytes) {
  if (s->stage_cap >= bytes) return MG_OK;
  MG_CK(cudaStreamSynchronize(s->stream));
  if (s->stage) cudaFree(s->stage);
  s->stage = nullptr;
  s->stage_cap = 0;
  MG_CK(cudaMalloc(&s->stage, bytes));
  s->stage_cap = bytes;
  return MG_OK;
}

// Stage a host input into device memory (synchronous w.r.t. the host buffer), or pass a device
// pointer through.
mg_status input_ptr(mg_sim *s, const void *in, size_t bytes, const void **dev) {
  if (is_device_ptr(in)) {
    *dev = in;
    return MG_OK;
  }
  mg_status st = ensure_stage(s, bytes);
  if (st != MG_OK) return st;
  MG_CK(cudaMemcpyAsync(s->stage, in, bytes, cudaMemcpyHostToDevice, s->stream));
  *dev = s->stage;
  return MG_OK;
}

// Runs of equal vehicle type, cut into pieces of at most `width` envs.
std::vector<BlockDesc> cut_runs(const mg_sim *s, int width) {
  std::vector<BlockDesc> b;
  int64_t e = 0;
  while (e < s->n) {
    const int32_t t = s->types_h[e];
    int64_t end = e;
    while (end < s->n && s->types_h[end] == t) ++end;
    for (int64_t a = e; a < end; a += width) {
      BlockDesc d;
      d.env0 = (int32_t)a;
      d.count = (int32_t)std::min<int64_t>(width, end - a);
      d.type = t;
      d.n_thr = s->vp[t].n_thr;
      b.push_back(d);
    }
    e = end;
  }
  return b;
}

// Build the static-schedule block list: pieces of at most epb envs (one env per thread).
mg_status build_blocks(mg_sim *s) {
  s->threads = (int)align_up((size_t)s->epb, 32);
  const std::vector<BlockDesc> b = cut_runs(s, s->epb);
  if (s->blocks_d) {
    MG_CK(cudaStreamSynchronize(s->stream));
    cudaFree(s->blocks_d);
    s->blocks_d = nullptr;
  }
  MG_CK(cudaMalloc(&s->blocks_d, b.size() * sizeof(BlockDesc)));
  MG_CK(cudaMemcpy(s->blocks_d, b.data(), b.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice));
  s->n_blocks = (int)b.size();
  s->drop_graphs();
  return MG_OK;
}

// The launches of one call of k sub-steps: each reads the device cursor plus its offset in the
// call, and the last advances the cursor by k.
mg_status launch_chunks(mg_sim *s, int32_t k, float *traj, cudaStream_t stream) {
  FleetView v = s->view();
  if (s->queue && !traj) {
    v.cursor_adv = k;
    MG_CK(launch_fleet_queue(v, s->slices_d, s->n_slices, s->ntv, s->diag, s->structured,
                             s->wide, s->queue_warps_per_sm, k, s->spl, s->sched, s->n_sm,
                             stream));
    return MG_OK;
  }
  for (int32_t done = 0; done < k;) {
    const int32_t kk = std::min(s->spl, k - done);
    float *t = traj ? traj + (int64_t)done * MG_NTRAJ * s->n : nullptr;
    v.cursor_off = done;
    v.cursor_adv = (done + kk == k) ? k : 0;
    MG_CK(launch_fleet(v, s->blocks_d, s->n_blocks, s->threads, s->ntv, s->diag, s->structured,
                       s->wide, kk, t, stream));
    done += kk;
  }
  return MG_OK;
}

// Streams and events of the asynchronous host transfers.
mg_status ensure_async(mg_sim *s) {
  if (s->h2d_stream) return MG_OK;
  MG_CK(cudaStreamCreateWithFlags(&s->h2d_stream, cudaStreamNonBlocking));
  MG_CK(cudaStreamCreateWithFlags(&s->d2h_stream, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) {
    MG_CK(cudaEventCreateWithFlags(&s->a_copied[i], cudaEventDisableTiming));
    MG_CK(cudaEventCreateWithFlags(&s->a_released[i], cudaEventDisableTiming));
    MG_CK(cudaEventCreateWithFlags(&s->o_exported[i], cudaEventDisableTiming));
    MG_CK(cudaEventCreateWithFlags(&s->o_read[i], cudaEventDisableTiming));
  }
  return MG_OK;
}

// The asynchronous action buffer the kernels read (if any) stops being read: everything queued
// on the sim's stream so far is its last use.
mg_status release_async_actions(mg_sim *s) {
  if (s->a_active >= 0) MG_CK(cudaEventRecord(s->a_released[s->a_active], s->stream));
  s->a_active = -1;
  return MG_OK;
}

bool is_pinned_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

mg_status read_counter(mg_sim *s, int idx, unsigned long long *out) {
  MG_CK(cudaMemcpyAsync(out, s->counters + idx, sizeof(*out), cudaMemcpyDeviceToHost,
                        s->stream));
  MG_CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

// Record the fleet's mass structure and pick the kernel path (see mg_sim::diag).
void set_mass_diag(mg_sim *s, bool mass_diag) {
  s->mass_diag = mass_diag;
  const bool diag = mass_diag && !(s->model_flags & MG_MODEL_NO_CURRENT_ACCEL);
  if (diag != s->diag) s->drop_graphs();
  s->diag = diag;
}

// After a parameter change: count non-SPD envs and pick the diagonal or general kernel.
mg_status finish_params(mg_sim *s) {
  unsigned long long bad = 0;
  unsigned int off = 0;
  MG_CK(cudaMemcpyAsync(&off, s->offdiag, sizeof off, cudaMemcpyDeviceToHost, s->stream));
  mg_status st = read_counter(s, 1, &bad);
  if (st != MG_OK) return st;
  set_mass_diag(s, (off == 0) && !s->has_xh);  // the extension always takes the general path
  if (bad) {
    char buf[160];
    snprintf(buf, sizeof buf, "%llu envs have a mass matrix that is not positive definite", bad);
    return fail(MG_ENOTSPD, buf);
  }
  return MG_OK;
}

// Rewind the action cursor (host copy and the device word the step kernels read).
mg_status rewind_cursor(mg_sim *s) {
  s->cursor = 0;
  MG_CK(cudaMemsetAsync(s->counters + 3, 0, sizeof(unsigned long long), s->stream));
  return MG_OK;
}

mg_status begin_params(mg_sim *s) {
  MG_CK(cudaMemsetAsync(s->counters + 1, 0, sizeof(unsigned long long), s->stream));
  MG_CK(cudaMemsetAsync(s->offdiag, 0, sizeof(unsigned int), s->stream));
  return MG_OK;
}

}  // namespace

// ---------------------------------------------------------------- mg_step_noalloc scratch
// Scheduler words for mg_step_noalloc: the work-queue counter and one progress word per 32-env
// slice, in a fixed device array instead of the sim's arena, so that the call itself never
// allocates.  Every GPU that loads the library holds it (256 KB) until the process exits.
constexpr int kNoAllocMaxSlices = 65536;  // fleets up to 2,097,152 envs
static __device__ __align__(256) uint32_t g_noalloc_sched[4 + kNoAllocMaxSlices];

namespace {

constexpr int kMaxDevices = 64;
uint32_t *g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of g_noalloc_sched on device dev (the sim's), looked up once per device with
// that device current: the array has one copy per device, and in host code its name is only a
// host-side stand-in, so kernels must be given this address.  The caller's current device is
// restored before returning.
mg_status noalloc_scratch(int dev, uint32_t **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(MG_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    int cur = 0;
    MG_CK(cudaGetDevice(&cur));
    if (cur != dev) MG_CK(cudaSetDevice(dev));
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_sched);
    if (cur != dev) MG_CK(cudaSetDevice(cur));
    MG_CK(e);
    g_noalloc_ptr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return MG_OK;
}

}  // namespace

extern "C" {

const char *mg_last_error(void) { return g_err.c_str(); }

mg_status mg_step_noalloc(mg_sim *s, int32_t k) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_step_noalloc");
  if (k < 1) return fail(MG_EINVAL, "k must be >= 1");
  if (s->n_slices > kNoAllocMaxSlices) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "fleet has %d 32-env slices; mg_step_noalloc supports at most %d (%d envs of one "
             "vehicle type)", s->n_slices, kNoAllocMaxSlices, 32 * kNoAllocMaxSlices);
    return fail(MG_EINVAL, buf);
  }
  uint32_t *sched = nullptr;
  mg_status st = noalloc_scratch(s->dev, &sched);
  if (st != MG_OK) return st;
  FleetView v = s->view();
  v.cursor_adv = k;
  MG_CK(launch_fleet_queue(v, s->slices_d, s->n_slices, s->ntv, s->diag, s->structured,
                           s->wide, s->queue_warps_per_sm, k, s->spl, sched, s->n_sm,
                           s->stream));
  s->cursor += k;
  return MG_OK;
}

mg_status mg_create(int64_t n_envs, const int32_t *vehicle_types,
                    const mg_vehicle_params *params, int32_t n_types, mg_sim **out) {
  MG_NONNULL(out);
  *out = nullptr;
  MG_NONNULL(vehicle_types);
  MG_NONNULL(params);
  if (n_envs < 1 || n_envs > (int64_t)INT32_MAX - 1024)
    return fail(MG_EINVAL, "n_envs must be in [1, 2^31 - 1025]");
  if (n_types < 1 || n_types > MG_MAX_TYPES) return fail(MG_EINVAL, "n_types out of range");
  for (int32_t t = 0; t < n_types; ++t)
    if (params[t].n_thr < 1 || params[t].n_thr > MG_MAX_THR)
      return fail(MG_EINVAL, "n_thr out of [1, MG_MAX_THR]");
  std::vector<int32_t> types(vehicle_types, vehicle_types + n_envs);
  bool seen[MG_MAX_TYPES] = {};
  for (int64_t e = 0; e < n_envs; ++e) {
    if (types[e] < 0 || types[e] >= n_types) return fail(MG_EINVAL, "vehicle type out of range");
    seen[types[e]] = true;
  }

  mg_sim *s = new mg_sim();
  s->n = n_envs;
  s->n_types = n_types;
  s->types_h = std::move(types);
  s->vp.assign(params, params + n_types);
  cudaGetDevice(&s->dev);

  // Kernel variant from the thruster counts present.
  int nt_seen = -1;
  bool uniform = true;
  for (int32_t t = 0; t < n_types; ++t) {
    if (!seen[t]) continue;
    if (nt_seen < 0) nt_seen = params[t].n_thr;
    else if (nt_seen != params[t].n_thr) uniform = false;
  }
  s->ntv = (uniform && nt_seen == 6) ? NT_6 : (uniform && nt_seen == 8) ? NT_8 : NT_MIXED;

  // Arena layout.
  const int64_t n = n_envs;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_s4[5] = {take(16 * n), take(16 * n), take(16 * n), take(16 * n), take(16 * n)};
  const size_t o_s5 = take(4 * n);
  size_t o_d[8];
  for (auto &x : o_d) x = take(16 * n);
  const size_t o_d8 = take(8 * n);
  size_t o_g[5];
  for (auto &x : o_g) x = take(16 * n);
  const size_t o_g5 = take(4 * n);
  const size_t o_raw = take(4 * n * MG_NPARAM);
  const size_t o_types = take(4 * n);
  const size_t o_geo = take(sizeof(Geo) * n_types);
  const size_t o_nom = take(4 * MG_NPARAM * n_types);
  const size_t o_flags = take(4 * n);
  const size_t o_ep = take(4 * n);
  const std::vector<BlockDesc> slices = cut_runs(s, 32);
  s->n_slices = (int)slices.size();
  const size_t o_slices = take(sizeof(BlockDesc) * slices.size());
  const size_t o_sched = take(queue_sched_bytes(s->n_slices));
  const size_t o_cnt = take(5 * sizeof(unsigned long long));
  const size_t o_off = take(sizeof(unsigned int));
  cudaError_t e = cudaMalloc(&s->arena, off);
  if (e != cudaSuccess) {
    delete s;
    return fail_cuda(e, "cudaMalloc(arena)");
  }
  char *a = static_cast<char *>(s->arena);
  s->st.s0 = (float4 *)(a + o_s4[0]);
  s->st.s1 = (float4 *)(a + o_s4[1]);
  s->st.s2 = (float4 *)(a + o_s4[2]);
  s->st.s3 = (float4 *)(a + o_s4[3]);
  s->st.s4 = (float4 *)(a + o_s4[4]);
  s->st.s5 = (float *)(a + o_s5);
  float4 **dp[8] = {&s->pa.d0, &s->pa.d1, &s->pa.d2, &s->pa.d3,
                    &s->pa.d4, &s->pa.d5, &s->pa.d6, &s->pa.d7};
  for (int i = 0; i < 8; ++i) *dp[i] = (float4 *)(a + o_d[i]);
  s->pa.d8 = (float2 *)(a + o_d8);
  float4 **gp[5] = {&s->pa.g0, &s->pa.g1, &s->pa.g2, &s->pa.g3, &s->pa.g4};
  for (int i = 0; i < 5; ++i) *gp[i] = (float4 *)(a + o_g[i]);
  s->pa.g5 = (float *)(a + o_g5);
  s->raw = (float *)(a + o_raw);
  s->par_off = o_d[0];
  s->par_bytes = o_types - o_d[0];
  s->types_d = (int32_t *)(a + o_types);
  s->geo_d = (Geo *)(a + o_geo);
  s->nominal_d = (float *)(a + o_nom);
  s->flags = (uint32_t *)(a + o_flags);
  s->episode = (uint32_t *)(a + o_ep);
  s->counters = (unsigned long long *)(a + o_cnt);
  s->slices_d = (BlockDesc *)(a + o_slices);
  s->sched = (uint32_t *)(a + o_sched);
  {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, s->dev) == cudaSuccess) s->n_sm = prop.multiProcessorCount;
  }
  s->offdiag = (unsigned int *)(a + o_off);

  // Per-type geometry and nominal records.
  std::vector<Geo> geo(n_types);
  s->structured = true;
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
    if (seen[t] && !vectored_layout(g)) s->structured = false;
    if (v.rg[0] != 0.f || v.rg[1] != 0.f || v.rg[2] != 0.f) s->nominal_diag = false;
    float *p = &nom[(size_t)t * MG_NPARAM];
    p[MG_P_M] = v.m;
    p[MG_P_IG] = v.Ixx;
    p[MG_P_IG + 1] = v.Iyy;
    p[MG_P_IG + 2] = v.Izz;
    for (int i = 0; i < 6; ++i) {
      p[MG_P_MA + i] = v.MA[i];
      p[MG_P_DL + i] = v.Dl[i];
      p[MG_P_DQ + i] = v.Dq[i];
    }
    p[MG_P_W] = v.W;
    p[MG_P_B] = v.B;
    for (int i = 0; i < 3; ++i) {
      p[MG_P_RG + i] = v.rg[i];
      p[MG_P_RB + i] = v.rb[i];
    }
    p[MG_P_KT] = v.kT;
    p[MG_P_TAU] = v.tau_m;
  }
  auto bail = [&](mg_status st) {
    mg_destroy(s);
    return st;
  };
  mg_status st;
#define MG_CKB(call)                                              \
  do {                                                            \
    cudaError_t _e = (call);                                      \
    if (_e != cudaSuccess) return bail(fail_cuda(_e, #call));     \
  } while (0)
  MG_CKB(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
  MG_CKB(cudaMemcpy(s->geo_d, geo.data(), sizeof(Geo) * n_types, cudaMemcpyHostToDevice));
  MG_CKB(cudaMemcpy(s->nominal_d, nom.data(), nom.size() * 4, cudaMemcpyHostToDevice));
  MG_CKB(cudaMemcpy(s->types_d, s->types_h.data(), 4 * n, cudaMemcpyHostToDevice));
  MG_CKB(cudaMemset(s->flags, 0, 4 * n));
  MG_CKB(cudaMemset(s->episode, 0, 4 * n));
  MG_CKB(cudaMemset(s->counters, 0, 5 * sizeof(unsigned long long)));
  MG_CKB(cudaMemcpy(s->slices_d, slices.data(), sizeof(BlockDesc) * slices.size(),
                    cudaMemcpyHostToDevice));
  MG_CKB(cudaMemset(s->offdiag, 0, sizeof(unsigned int)));
  // Nominal parameters: a randomisation with zero width.
  MG_CKB(launch_randomize(s->setup_view(), s->nominal_d, 0, 1.0, 1.0, 0.0, 0.0, s->stream));
  if ((st = finish_params(s)) != MG_OK) return bail(st);
  // Zero state with identity attitude.
  MG_CKB(cudaMemset(s->arena, 0, o_s5 + 4 * n));
  MG_CKB(launch_reset(s->st, n, 0, nullptr, 0, 0.0, s->episode, s->flags, s->counters,
                      s->stream));
  MG_CKB(cudaMemset(s->episode, 0, 4 * n));
  if ((st = build_blocks(s)) != MG_OK) return bail(st);
  MG_CKB(cudaStreamSynchronize(s->stream));
#undef MG_CKB
  *out = s;
  return MG_OK;
}

mg_status mg_destroy(mg_sim *s) {
  if (!s) return MG_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  cudaDeviceSynchronize();
  s->drop_graphs();
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->pf_stream) {
    cudaStreamSynchronize(s->pf_stream);
    cudaStreamDestroy(s->pf_stream);
    cudaEventDestroy(s->pf_done);
    cudaEventDestroy(s->pf_consumed);
    cudaFree(s->pf_buf);
  }
  if (s->h2d_stream) {
    cudaStreamSynchronize(s->h2d_stream);
    cudaStreamSynchronize(s->d2h_stream);
    cudaStreamDestroy(s->h2d_stream);
    cudaStreamDestroy(s->d2h_stream);
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(s->a_copied[i]);
      cudaEventDestroy(s->a_released[i]);
      cudaEventDestroy(s->o_exported[i]);
      cudaEventDestroy(s->o_read[i]);
      cudaFree(s->abuf[i]);
      cudaFree(s->obuf[i]);
    }
  }
  cudaFree(s->blocks_d);
  cudaFree(s->task_buf);
  cudaFree(s->act);
  cudaFree(s->stage);
  cudaFree(s->xh);
  cudaFree(s->env_act);
  cudaFree(s->adj_ws);
  cudaFree(s->arena);
  delete s;
  return MG_OK;
}

mg_status mg_set_stream(mg_sim *s, void *stream) {
  MG_NONNULL(s);
  s->stream = static_cast<cudaStream_t>(stream);
  return MG_OK;
}

mg_status mg_set_env_id_offset(mg_sim *s, int64_t offset) {
  MG_NONNULL(s);
  if (offset < 0) return fail(MG_EINVAL, "offset must be >= 0");
  s->gid0 = offset;
  s->drop_graphs();
  return MG_OK;
}

mg_status mg_set_model_flags(mg_sim *s, uint32_t flags) {
  MG_NONNULL(s);
  if (flags & ~MG_MODEL_NO_CURRENT_ACCEL) return fail(MG_EINVAL, "unknown model flag");
  s->model_flags = flags;
  s->drop_graphs();
  set_mass_diag(s, s->mass_diag);
  return MG_OK;
}

mg_status mg_set_timestep(mg_sim *s, float dt) {
  MG_NONNULL(s);
  if (!(dt > 0.f && dt <= 1.f)) return fail(MG_EINVAL, "dt must be in (0, 1]");
  s->dt = dt;
  s->drop_graphs();
  return MG_OK;
}

mg_status mg_set_launch(mg_sim *s, int32_t envs_per_block, int32_t steps_per_launch,
                        int32_t use_graph) {
  MG_NONNULL(s);
  if (envs_per_block < 32 || envs_per_block > 256)
    return fail(MG_EINVAL, "envs_per_block must be in [32, 256]");
  if (steps_per_launch < 1) return fail(MG_EINVAL, "steps_per_launch must be >= 1");
  s->spl = steps_per_launch;
  s->use_graph = use_graph != 0;
  s->drop_graphs();
  if (envs_per_block != s->epb) {
    s->epb = envs_per_block;
    return build_blocks(s);
  }
  return MG_OK;
}

mg_status mg_set_schedule(mg_sim *s, int32_t work_queue, int32_t wide, int32_t warps_per_sm) {
  MG_NONNULL(s);
  if (warps_per_sm < 0 || warps_per_sm > 64) return fail(MG_EINVAL, "warps_per_sm in [0, 64]");
  s->queue = work_queue != 0;
  s->wide = wide != 0;
  s->queue_warps_per_sm = warps_per_sm;
  s->drop_graphs();
  return MG_OK;
}

mg_status mg_set_wait_limit(mg_sim *s, uint32_t polls) {
  MG_NONNULL(s);
  if (polls > (1u << 30)) return fail(MG_EINVAL, "polls must be <= 2^30");
  const uint32_t v = polls ? polls : (uint32_t)MG_WAIT_POLLS_DEFAULT;
  if (v != s->wait_limit) s->drop_graphs();
  s->wait_limit = v;
  return MG_OK;
}

namespace {

mg_status check_ranges(const mg_ranges *r) {
  if (!(r->lo > 0.f) || !(r->lo <= r->hi) || !(r->current_sigma >= 0.f) ||
      !(r->nu0_sigma >= 0.f) || (r->flags & ~MG_RANDOMIZE_ASYNC) != 0 ||
      !(r->rg_halfwidth >= 0.f))
    return fail(MG_EINVAL, "ranges: need 0 < lo <= hi, sigmas >= 0, rg_halfwidth >= 0, "
                           "flags 0 or MG_RANDOMIZE_ASYNC");
  return MG_OK;
}

// Mass matrices known to be diagonal before any draw (what MG_RANDOMIZE_ASYNC and
// mg_randomize_prefetch need).
bool diagonal_by_construction(const mg_sim *s, const mg_ranges *r) {
  return s->nominal_diag && r->rg_halfwidth == 0.f && !s->has_xh;
}

// Whether the background range holds exactly what mg_randomize(s, seed, r) would draw.
bool staged_matches(const mg_sim *s, uint64_t seed, const mg_ranges *r) {
  return s->pf_valid && diagonal_by_construction(s, r) && s->pf_seed == seed &&
         s->pf_lo == r->lo && s->pf_hi == r->hi && s->pf_current_sigma == r->current_sigma &&
         s->pf_gid0 == s->gid0;
}

}  // namespace

mg_status mg_randomize_prefetch(mg_sim *s, uint64_t seed, const mg_ranges *r) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_randomize_prefetch");
  MG_NONNULL(r);
  mg_status st = check_ranges(r);
  if (st != MG_OK) return st;
  if (!diagonal_by_construction(s, r))
    return fail(MG_EINVAL, "mg_randomize_prefetch needs mass matrices known to be diagonal "
                           "(r_g = 0 for every type, rg_halfwidth = 0, no extension)");
  if (!s->pf_stream) {
    MG_CK(cudaStreamCreateWithFlags(&s->pf_stream, cudaStreamNonBlocking));
    MG_CK(cudaEventCreateWithFlags(&s->pf_done, cudaEventDisableTiming));
    MG_CK(cudaEventCreateWithFlags(&s->pf_consumed, cudaEventDisableTiming));
    if (cudaMalloc(&s->pf_buf, s->par_bytes + 16) != cudaSuccess) {
      cudaGetLastError();
      s->pf_buf = nullptr;
      cudaEventDestroy(s->pf_done);
      cudaEventDestroy(s->pf_consumed);
      cudaStreamDestroy(s->pf_stream);
      s->pf_stream = nullptr;
      return fail(MG_ENOMEM, "cudaMalloc(background parameter range)");
    }
  }
  s->pf_valid = false;
  // the last install's copy must have read the range (a never-recorded event is no wait)
  MG_CK(cudaStreamWaitEvent(s->pf_stream, s->pf_consumed, 0));
  const SetupView v = s->staged_setup_view();
  MG_CK(cudaMemsetAsync(v.n_not_spd, 0, 16, s->pf_stream));
  MG_CK(launch_randomize(v, s->nominal_d, seed, (double)r->lo, (double)r->hi,
                         (double)r->current_sigma, 0.0, s->pf_stream, s->n_sm));
  MG_CK(cudaEventRecord(s->pf_done, s->pf_stream));
  s->pf_valid = true;
  s->pf_seed = seed;
  s->pf_lo = r->lo;
  s->pf_hi = r->hi;
  s->pf_current_sigma = r->current_sigma;
  s->pf_gid0 = s->gid0;
  return MG_OK;
}

mg_status mg_randomize(mg_sim *s, uint64_t seed, const mg_ranges *r) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_randomize");
  MG_NONNULL(r);
  mg_status st = check_ranges(r);
  if (st != MG_OK) return st;
  const bool async = (r->flags & MG_RANDOMIZE_ASYNC) != 0;
  if (async && !diagonal_by_construction(s, r))
    return fail(MG_EINVAL, "MG_RANDOMIZE_ASYNC needs mass matrices known to be diagonal "
                           "(r_g = 0 for every type, rg_halfwidth = 0, no extension)");
  if (staged_matches(s, seed, r)) {
    // install the background draw: one copy of the parameter range and its two check words
    char *live = static_cast<char *>(s->arena) + s->par_off;
    MG_CK(cudaStreamWaitEvent(s->stream, s->pf_done, 0));
    MG_CK(cudaMemcpyAsync(live, s->pf_buf, s->par_bytes, cudaMemcpyDeviceToDevice, s->stream));
    MG_CK(cudaMemcpyAsync(s->counters + 1, s->pf_buf + s->par_bytes, 8,
                          cudaMemcpyDeviceToDevice, s->stream));
    MG_CK(cudaMemcpyAsync(s->offdiag, s->pf_buf + s->par_bytes + 8, 4,
                          cudaMemcpyDeviceToDevice, s->stream));
    MG_CK(cudaEventRecord(s->pf_consumed, s->stream));
  } else {
    if ((st = begin_params(s)) != MG_OK) return st;
    MG_CK(launch_randomize(s->setup_view(), s->nominal_d, seed, (double)r->lo, (double)r->hi,
                           (double)r->current_sigma, (double)r->rg_halfwidth, s->stream));
  }
  MG_CK(cudaMemsetAsync(s->episode, 0, 4 * s->n, s->stream));
  s->reset_seed = seed;
  s->nu0_sigma = (double)r->nu0_sigma;
  if (async) {  // diagonal by construction; a pivot <= 0 is left to mg_sync
    set_mass_diag(s, true);
    return MG_OK;
  }
  return finish_params(s);
}

mg_status mg_set_params(mg_sim *s, const float *in) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_set_params");
  MG_NONNULL(in);
  const void *d = nullptr;
  mg_status st = input_ptr(s, in, (size_t)s->n * MG_NPARAM * 4, &d);
  if (st != MG_OK) return st;
  if ((st = begin_params(s)) != MG_OK) return st;
  MG_CK(launch_import_params(s->setup_view(), static_cast<const float *>(d), s->stream));
  return finish_params(s);
}

mg_status mg_get_params(mg_sim *s, float *out) {
  MG_NONNULL(s);
  MG_NONNULL(out);
  const size_t bytes = (size_t)s->n * MG_NPARAM * 4;
  if (is_device_ptr(out)) {
    MG_CK(launch_export_params(s->setup_view(), out, s->stream));
    return MG_OK;
  }
  mg_status st = ensure_stage(s, bytes);
  if (st != MG_OK) return st;
  MG_CK(launch_export_params(s->setup_view(), static_cast<float *>(s->stage), s->stream));
  MG_CK(cudaMemcpyAsync(out, s->stage, bytes, cudaMemcpyDeviceToHost, s->stream));
  MG_CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

mg_status mg_set_hydro_offdiag(mg_sim *s, const float *x) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_set_hydro_offdiag");
  mg_status st;
  if (x) {
    const size_t bytes = (size_t)s->n * MG_NXPARAM * 4;
    const void *d = nullptr;
    if ((st = input_ptr(s, x, bytes, &d)) != MG_OK) return st;
    if (!s->xh) {
      MG_CK(cudaStreamSynchronize(s->stream));
      if (cudaMalloc(&s->xh, bytes) != cudaSuccess) {
        cudaGetLastError();
        s->xh = nullptr;
        return fail(MG_ENOMEM, "cudaMalloc(off-diagonal hydrodynamics)");
      }
    }
    MG_CK(launch_xh_transpose(static_cast<const float *>(d), s->xh, s->n, true, s->stream));
  }
  s->has_xh = (x != nullptr);
  s->drop_graphs();
  // re-derive every env's planes (M^-1 with the off-diagonal added mass) from its own record
  if ((st = begin_params(s)) != MG_OK) return st;
  MG_CK(launch_import_params(s->setup_view(), s->raw, s->stream));
  return finish_params(s);
}

mg_status mg_get_hydro_offdiag(mg_sim *s, float *out) {
  MG_NONNULL(s);
  MG_NONNULL(out);
  const size_t bytes = (size_t)s->n * MG_NXPARAM * 4;
  const bool dev = is_device_ptr(out);
  float *dst = out;
  if (!dev) {
    mg_status st = ensure_stage(s, bytes);
    if (st != MG_OK) return st;
    dst = static_cast<float *>(s->stage);
  }
  if (s->has_xh)
    MG_CK(launch_xh_transpose(s->xh, dst, s->n, false, s->stream));
  else
    MG_CK(cudaMemsetAsync(dst, 0, bytes, s->stream));
  if (!dev) {
    MG_CK(cudaMemcpyAsync(out, s->stage, bytes, cudaMemcpyDeviceToHost, s->stream));
    MG_CK(cudaStreamSynchronize(s->stream));
  }
  return MG_OK;
}

mg_status mg_set_actions(mg_sim *s, const float *a, int32_t n_seg, int32_t hold_steps) {
  MG_NONNULL(s);
  if (n_seg < 0 || hold_steps < 1) return fail(MG_EINVAL, "need n_seg >= 0 and hold_steps >= 1");
  if (n_seg > 0 && !a) return fail(MG_EINVAL, "a is NULL with n_seg > 0");
  const size_t floats = (size_t)n_seg * s->n * s->act_w;
  if (floats > s->act_cap) {
    MG_CK(cudaStreamSynchronize(s->stream));
    cudaFree(s->act);
    s->act = nullptr;
    s->act_cap = 0;
    MG_CK(cudaMalloc(&s->act, floats * 4));
    s->act_cap = floats;
    s->drop_graphs();
  }
  mg_status rs = release_async_actions(s);
  if (rs != MG_OK) return rs;
  if (n_seg > 0) {
    const bool dev = is_device_ptr(a);
    MG_CK(cudaMemcpyAsync(s->act, a, floats * 4,
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
    if (!dev) MG_CK(cudaStreamSynchronize(s->stream));
  }
  s->act_src = s->act;
  s->proc = 0;
  s->n_seg = n_seg;
  s->hold = hold_steps;
  return rewind_cursor(s);
}

mg_status mg_set_actions_borrowed(mg_sim *s, const float *a, int32_t n_seg, int32_t hold_steps) {
  MG_NONNULL(s);
  MG_NONNULL(a);
  if (n_seg < 1 || hold_steps < 1) return fail(MG_EINVAL, "need n_seg >= 1 and hold_steps >= 1");
  if (!is_device_ptr(a)) return fail(MG_EINVAL, "borrowed actions must be device memory");
  if ((reinterpret_cast<uintptr_t>(a) & 15) != 0)
    return fail(MG_EINVAL, "borrowed actions must be 16-byte aligned");
  mg_status rs = release_async_actions(s);
  if (rs != MG_OK) return rs;
  s->act_src = a;
  s->proc = 0;
  s->n_seg = n_seg;
  s->hold = hold_steps;
  return rewind_cursor(s);
}

mg_status mg_set_actions_async(mg_sim *s, const float *a, int32_t n_seg, int32_t hold_steps) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_set_actions_async");
  MG_NONNULL(a);
  if (n_seg < 1 || hold_steps < 1) return fail(MG_EINVAL, "need n_seg >= 1 and hold_steps >= 1");
  if (!is_pinned_host(a))
    return fail(MG_EINVAL, "mg_set_actions_async needs page-locked host memory");
  mg_status st = ensure_async(s);
  if (st != MG_OK) return st;
  const int slot = s->a_next;
  // This slot's previous copy (two calls ago) read its host buffer; once it has finished, that
  // buffer is the caller's again.
  MG_CK(cudaEventSynchronize(s->a_copied[slot]));
  const size_t floats = (size_t)n_seg * s->n * s->act_w;
  if (floats > s->abuf_cap[slot]) {
    MG_CK(cudaStreamSynchronize(s->stream));
    MG_CK(cudaStreamSynchronize(s->h2d_stream));
    cudaFree(s->abuf[slot]);
    s->abuf[slot] = nullptr;
    s->abuf_cap[slot] = 0;
    MG_CK(cudaMalloc(&s->abuf[slot], floats * 4));
    s->abuf_cap[slot] = floats;
  }
  s->a_next ^= 1;
  // the copy waits for the last steps that read this buffer, the sim's later work for the copy
  MG_CK(cudaStreamWaitEvent(s->h2d_stream, s->a_released[slot], 0));
  MG_CK(cudaMemcpyAsync(s->abuf[slot], a, floats * 4, cudaMemcpyHostToDevice, s->h2d_stream));
  MG_CK(cudaEventRecord(s->a_copied[slot], s->h2d_stream));
  if ((st = release_async_actions(s)) != MG_OK) return st;
  MG_CK(cudaStreamWaitEvent(s->stream, s->a_copied[slot], 0));
  s->a_active = slot;
  s->act_src = s->abuf[slot];
  s->proc = 0;
  s->n_seg = n_seg;
  s->hold = hold_steps;
  return rewind_cursor(s);
}

mg_status mg_set_action_width(mg_sim *s, int32_t width) {
  MG_NONNULL(s);
  if (width != MG_MAX_THR && width != 6)
    return fail(MG_EINVAL, "the action width must be 6 or MG_MAX_THR");
  if (width < MG_MAX_THR && s->ntv != NT_6)
    return fail(MG_EINVAL, "a 6-float action width needs a fleet of 6-thruster vehicles only");
  if (width == s->act_w) return MG_OK;
  mg_status rs = release_async_actions(s);
  if (rs != MG_OK) return rs;
  // the buffered schedule was laid out for the old width: the commands become zero until the
  // next mg_set_actions* call
  s->act_w = width;
  s->act_src = nullptr;
  s->proc = 0;
  s->n_seg = 0;
  s->drop_graphs();
  return rewind_cursor(s);
}

mg_status mg_set_procedural_actions(mg_sim *s, uint64_t cmd_seed, int32_t hold_steps) {
  MG_NONNULL(s);
  if (hold_steps < 1) return fail(MG_EINVAL, "hold_steps must be >= 1");
  mg_status rs = release_async_actions(s);
  if (rs != MG_OK) return rs;
  s->proc = 1;
  s->cmd_seed = cmd_seed;
  s->hold = hold_steps;
  s->n_seg = 0;
  return rewind_cursor(s);
}

mg_status mg_step(mg_sim *s, int32_t k) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_step");
  if (k < 1) return fail(MG_EINVAL, "k must be >= 1");
  if (!s->use_graph) {
    mg_status st = launch_chunks(s, k, nullptr, s->stream);
    if (st != MG_OK) return st;
    s->cursor += k;
    return MG_OK;
  }
  GraphEntry *hit = nullptr;
  const float *src = s->proc ? nullptr : s->act_src;
  const uint64_t seed = s->proc ? s->cmd_seed : 0;
  for (auto &g : s->graphs)
    if (g.k == k && g.act_src == src && g.n_seg == s->n_seg && g.hold == s->hold &&
        g.proc == s->proc && g.cmd_seed == seed)
      hit = &g;
  if (!hit) {
    if (s->graphs.size() >= 16) {
      auto lru = std::min_element(s->graphs.begin(), s->graphs.end(),
                                  [](const GraphEntry &x, const GraphEntry &y) {
                                    return x.last_use < y.last_use;
                                  });
      cudaGraphExecDestroy(lru->exec);
      s->graphs.erase(lru);
    }
    cudaGraph_t graph = nullptr;
    MG_CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    mg_status st = launch_chunks(s, k, nullptr, s->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &graph);
    if (st != MG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    MG_CK(ce);
    GraphEntry g{k, src, s->n_seg, s->hold, s->proc, seed, nullptr, 0};
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    MG_CK(ce);
    s->graphs.push_back(g);
    hit = &s->graphs.back();
  }
  hit->last_use = ++s->graph_clock;
  MG_CK(cudaGraphLaunch(hit->exec, s->stream));
  s->cursor += k;
  return MG_OK;
}

mg_status mg_step_split(mg_sim *s, int32_t k, float *accel) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_step_split");
  MG_NONNULL(accel);
  if (k < 1) return fail(MG_EINVAL, "k must be >= 1");
  if (!is_device_ptr(accel)) return fail(MG_EINVAL, "accel must be device memory");
  FleetView v = s->view();
  for (int32_t done = 0; done < k;) {
    const int32_t kk = std::min(s->spl, k - done);
    v.cursor_off = done;
    v.cursor_adv = (done + kk == k) ? k : 0;
    MG_CK(launch_split(v, s->blocks_d, s->n_blocks, s->threads, s->ntv, !s->mass_diag, s->raw,
                       accel, kk, s->stream));
    done += kk;
  }
  s->cursor += k;
  return MG_OK;
}

mg_status mg_step_record(mg_sim *s, int32_t k, float *traj) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_step_record");
  MG_NONNULL(traj);
  if (k < 1) return fail(MG_EINVAL, "k must be >= 1");
  if (!is_device_ptr(traj)) return fail(MG_EINVAL, "traj must be device memory");
  mg_status st = launch_chunks(s, k, traj, s->stream);
  if (st != MG_OK) return st;
  s->cursor += k;
  return MG_OK;
}

mg_status mg_rollout_forward(mg_sim *s, int32_t T, int32_t C, float *traj, float *ckpt,
                             int64_t *step0_out) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_rollout_forward");
  MG_NONNULL(traj);
  MG_NONNULL(ckpt);
  if (T < 1 || C < 1 || C > adjoint_max_interval())
    return fail(MG_EINVAL, "need T >= 1 and 1 <= C <= 32");
  if (!is_device_ptr(traj) || !is_device_ptr(ckpt))
    return fail(MG_EINVAL, "traj and ckpt must be device memory");
  FleetView v = s->view();
  const int64_t step0 = s->cursor;
  v.cursor_off = 0;
  v.cursor_adv = T;
  MG_CK(launch_rollout_forward(v, s->blocks_d, s->n_blocks, s->threads, s->ntv, s->diag,
                               s->structured, T, C, traj, ckpt, s->stream));
  s->cursor += T;
  if (step0_out) *step0_out = step0;
  return MG_OK;
}

mg_status mg_rollout_backward(mg_sim *s, int32_t T, int32_t C, const float *ckpt,
                              const float *dtraj, int64_t step0, float *dcoef, float *dact,
                              float *dstate0) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_rollout_backward");
  MG_NONNULL(ckpt);
  MG_NONNULL(dtraj);
  MG_NONNULL(dcoef);
  if (T < 1 || C < 1 || C > adjoint_max_interval() || step0 < 0)
    return fail(MG_EINVAL, "need T >= 1, 1 <= C <= 32, step0 >= 0");
  if (s->proc) return fail(MG_EINVAL, "the adjoint needs buffered actions (mg_set_actions)");
  for (const void *p : {(const void *)ckpt, (const void *)dtraj, (const void *)dcoef})
    if (!is_device_ptr(p)) return fail(MG_EINVAL, "adjoint buffers must be device memory");
  if ((dact && !is_device_ptr(dact)) || (dstate0 && !is_device_ptr(dstate0)))
    return fail(MG_EINVAL, "adjoint buffers must be device memory");
  const bool eight = s->ntv != NT_6;
  bool split = false;
  MG_CK(adjoint_split(s->n, s->adj_mode, &split));
  if (split) {
    const size_t bytes = adjoint_workspace_bytes(eight, s->n, C);
    if (s->adj_ws_cap < bytes) {
      MG_CK(cudaStreamSynchronize(s->stream));
      cudaFree(s->adj_ws);
      s->adj_ws = nullptr;
      s->adj_ws_cap = 0;
      if (cudaMalloc(&s->adj_ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        s->adj_ws = nullptr;
        return fail(MG_ENOMEM, "cudaMalloc(adjoint workspace)");
      }
      s->adj_ws_cap = bytes;
    }
  }
  MG_CK(launch_adjoint(s->view(), s->types_d, eight, !s->diag || s->has_xh, ckpt, dtraj, T, C,
                       step0, dcoef, dact, dstate0, split, s->adj_ws, s->stream));
  return MG_OK;
}

mg_status mg_set_adjoint_mode(mg_sim *s, int32_t mode) {
  MG_NONNULL(s);
  if (mode < 0 || mode > 2) return fail(MG_EINVAL, "adjoint mode must be 0, 1 or 2");
  s->adj_mode = mode;
  return MG_OK;
}

mg_status mg_set_task(mg_sim *s, const mg_task_spec *spec, const float *centres) {
  MG_NONNULL(s);
  MG_NONNULL(spec);
  MG_NONNULL(centres);
  if (spec->task < MG_TASK_STATION || spec->task > MG_TASK_LEMNISCATE || spec->lookahead < 1 ||
      spec->lookahead > 64 || spec->flags != 0)
    return fail(MG_EINVAL, "task spec: unknown task, lookahead outside [1, 64] or flags != 0");
  if (!s->task_buf) MG_CK(cudaMalloc(&s->task_buf, 24 * (size_t)s->n));
  const void *d = nullptr;
  mg_status st = input_ptr(s, centres, 16 * (size_t)s->n, &d);
  if (st != MG_OK) return st;
  MG_CK(cudaMemcpyAsync(s->task_buf, d, 16 * (size_t)s->n, cudaMemcpyDeviceToDevice, s->stream));
  MG_CK(cudaMemsetAsync(static_cast<char *>(s->task_buf) + 16 * s->n, 0, 8 * (size_t)s->n,
                        s->stream));
  MG_CK(cudaStreamSynchronize(s->stream));
  s->task = *spec;
  s->has_task = true;
  return MG_OK;
}

mg_status mg_task_obs_dim(mg_sim *s, int32_t *obs_dim) {
  MG_NONNULL(s);
  MG_NONNULL(obs_dim);
  if (!s->has_task) return fail(MG_ESTATE, "no task set");
  *obs_dim = 6 * (s->task.task == MG_TASK_STATION ? 1 : s->task.lookahead) + 6;
  return MG_OK;
}

}  // extern "C"

namespace {

// A task step (mg_task_step) with its outputs; err and reward may each be null.
mg_status task_step_outputs(mg_sim *s, int32_t k, float *obs, float *err, float *reward,
                            uint8_t *done, float *episode_err) {
  if (!s->has_task) return fail(MG_ESTATE, "no task set");
  if (k < 0) return fail(MG_EINVAL, "k must be >= 0");
  // a policy loop passes the same output buffers every call: check them once (a pointer query
  // costs microseconds, more than the host budget of a task step)
  const void *outs[5] = {obs, err, done, episode_err, reward};
  if (!std::equal(outs, outs + 5, s->task_out_ok)) {
    for (const void *p : outs)
      if (p && !is_device_ptr(p)) return fail(MG_EINVAL, "task outputs must be device memory");
    std::copy(outs, outs + 5, s->task_out_ok);
  }
  if (k == 0) {  // observe only
    MG_CK(launch_task(s->st, s->task_view(), s->n, s->gid0, 0, s->dt, obs, err, done,
                      episode_err, s->reset_seed, s->nu0_sigma, s->episode, s->flags,
                      s->counters, s->stream));
    return MG_OK;
  }
  // Leading sub-steps as mg_step; the last static chunk carries the fused task epilogue.
  const int32_t k_last = (k - 1) % s->spl + 1;
  if (k > k_last) {
    mg_status st = mg_step(s, k - k_last);
    if (st != MG_OK) return st;
  }
  int32_t obs_dim = 0;
  mg_task_obs_dim(s, &obs_dim);
  TaskOut to{obs, err, done, episode_err, obs_dim, 0, s->reset_seed, s->nu0_sigma, s->episode,
             reward};
  FleetView v = s->view();
  v.cursor_adv = k_last;
  MG_CK(launch_fleet_task(v, s->blocks_d, s->n_blocks, s->threads, s->ntv, s->diag,
                          s->structured, k_last, k, s->task_view(), to, s->stream));
  s->cursor += k_last;
  return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_task_step(mg_sim *s, int32_t k, float *obs, float *err, uint8_t *done,
                       float *episode_err) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_task_step");
  MG_NONNULL(obs);
  MG_NONNULL(err);
  MG_NONNULL(done);
  return task_step_outputs(s, k, obs, err, nullptr, done, episode_err);
}

mg_status mg_env_step(mg_sim *s, int32_t k, const float *actions, float *obs, float *reward,
                      uint8_t *done, float *episode_err) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_env_step");
  MG_NONNULL(actions);
  MG_NONNULL(obs);
  MG_NONNULL(reward);
  MG_NONNULL(done);
  if (!s->has_task) return fail(MG_ESTATE, "no task set");
  if (k < 1) return fail(MG_EINVAL, "k must be >= 1");
  if (actions != s->env_in_ok) {
    if (!is_device_ptr(actions)) return fail(MG_EINVAL, "actions must be device memory");
    s->env_in_ok = actions;
  }
  const size_t floats = (size_t)s->n * s->act_w;
  if (s->env_act_cap < floats) {
    MG_CK(cudaStreamSynchronize(s->stream));
    cudaFree(s->env_act);
    s->env_act = nullptr;
    s->env_act_cap = 0;
    if (cudaMalloc(reinterpret_cast<void **>(&s->env_act), floats * sizeof(float)) !=
        cudaSuccess) {
      cudaGetLastError();
      s->env_act = nullptr;
      return fail(MG_ENOMEM, "cudaMalloc(environment actions)");
    }
    s->env_act_cap = floats;
  }
  // The schedule is one segment held for good (every sub-step past a schedule's end holds its
  // last segment), so it is set up once and then only rewritten.
  if (s->act_src != s->env_act || s->n_seg != 1 || s->proc) {
    mg_status st = release_async_actions(s);
    if (st != MG_OK) return st;
    s->act_src = s->env_act;
    s->proc = 0;
    s->n_seg = 1;
    s->hold = 1 << 30;
    if ((st = rewind_cursor(s)) != MG_OK) return st;
  }
  MG_CK(launch_clamp_actions(actions, s->env_act, (int64_t)floats, s->stream));
  return task_step_outputs(s, k, obs, nullptr, reward, done, episode_err);
}

mg_status mg_get_state(mg_sim *s, float *out) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_get_state");
  MG_NONNULL(out);
  const size_t bytes = (size_t)s->n * MG_NSTATE * 4;
  if (is_device_ptr(out)) {
    MG_CK(launch_export_state(s->st, s->n, out, s->stream));
    return MG_OK;
  }
  mg_status st = ensure_stage(s, bytes);
  if (st != MG_OK) return st;
  MG_CK(launch_export_state(s->st, s->n, static_cast<float *>(s->stage), s->stream));
  MG_CK(cudaMemcpyAsync(out, s->stage, bytes, cudaMemcpyDeviceToHost, s->stream));
  MG_CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

mg_status mg_get_state_async(mg_sim *s, float *out) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_get_state_async");
  MG_NONNULL(out);
  if (!is_pinned_host(out))
    return fail(MG_EINVAL, "mg_get_state_async needs page-locked host memory");
  mg_status st = ensure_async(s);
  if (st != MG_OK) return st;
  const int slot = s->o_next;
  const size_t bytes = (size_t)s->n * MG_NSTATE * 4;
  if (!s->obuf[slot]) MG_CK(cudaMalloc(&s->obuf[slot], bytes));
  s->o_next ^= 1;
  // the export waits for the previous read-back from this buffer, the read-back for the export
  MG_CK(cudaStreamWaitEvent(s->stream, s->o_read[slot], 0));
  MG_CK(launch_export_state(s->st, s->n, s->obuf[slot], s->stream));
  MG_CK(cudaEventRecord(s->o_exported[slot], s->stream));
  MG_CK(cudaStreamWaitEvent(s->d2h_stream, s->o_exported[slot], 0));
  MG_CK(cudaMemcpyAsync(out, s->obuf[slot], bytes, cudaMemcpyDeviceToHost, s->d2h_stream));
  MG_CK(cudaEventRecord(s->o_read[slot], s->d2h_stream));
  return MG_OK;
}

mg_status mg_set_state(mg_sim *s, const float *in) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_set_state");
  MG_NONNULL(in);
  const void *d = nullptr;
  mg_status st = input_ptr(s, in, (size_t)s->n * MG_NSTATE * 4, &d);
  if (st != MG_OK) return st;
  MG_CK(launch_import_state(s->st, s->n, static_cast<const float *>(d), s->stream));
  if (d == s->stage) MG_CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

mg_status mg_reset(mg_sim *s, const uint8_t *mask) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_reset");
  const void *d = nullptr;
  if (mask) {
    mg_status st = input_ptr(s, mask, (size_t)s->n, &d);
    if (st != MG_OK) return st;
  }
  MG_CK(launch_reset(s->st, s->n, s->gid0, static_cast<const uint8_t *>(d), s->reset_seed,
                     s->nu0_sigma, s->episode, s->flags, s->counters, s->stream));
  if (d && d == s->stage) MG_CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

mg_status mg_sync(mg_sim *s, int64_t *nonfinite_count) {
  MG_NONNULL(s);
  NvtxRange nvtx("mg_sync");
  if (s->pf_stream) MG_CK(cudaStreamSynchronize(s->pf_stream));
  if (s->h2d_stream) {
    MG_CK(cudaStreamSynchronize(s->h2d_stream));
    MG_CK(cudaStreamSynchronize(s->d2h_stream));
  }
  unsigned long long c = 0, to = 0;
  mg_status st = read_counter(s, 2, &to);
  if (st != MG_OK) return st;
  if ((st = read_counter(s, 0, &c)) != MG_OK) return st;
  if (nonfinite_count) *nonfinite_count = (int64_t)c;
  if (to) {
    // reported once: the count restarts from zero for the steps after this call
    MG_CK(cudaMemsetAsync(s->counters + 2, 0, sizeof(unsigned long long), s->stream));
    MG_CK(cudaStreamSynchronize(s->stream));
    char buf[128];
    snprintf(buf, sizeof buf, "%llu work-queue waits timed out", to);
    return fail(MG_ETIMEOUT, buf);
  }
  unsigned long long bad = 0;
  if ((st = read_counter(s, 1, &bad)) != MG_OK) return st;
  if (bad) {
    char buf[160];
    snprintf(buf, sizeof buf, "%llu envs have a mass matrix that is not positive definite", bad);
    return fail(MG_ENOTSPD, buf);
  }
  if (c) {
    char buf[128];
    snprintf(buf, sizeof buf, "%llu envs have a non-finite state", c);
    return fail(MG_ENONFINITE, buf);
  }
  return MG_OK;
}

mg_status mg_get_nonfinite(mg_sim *s, uint8_t *out) {
  MG_NONNULL(s);
  MG_NONNULL(out);
  if (is_device_ptr(out)) {
    MG_CK(launch_flags_to_bytes(s->flags, s->n, out, s->stream));
    return MG_OK;
  }
  mg_status st = ensure_stage(s, (size_t)s->n);
  if (st != MG_OK) return st;
  MG_CK(launch_flags_to_bytes(s->flags, s->n, static_cast<uint8_t *>(s->stage), s->stream));
  MG_CK(cudaMemcpyAsync(out, s->stage, (size_t)s->n, cudaMemcpyDeviceToHost, s->stream));
  MG_CK(cudaStreamSynchronize(s->stream));
  return MG_OK;
}

mg_status mg_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n) {
  MG_NONNULL(ctr);
  MG_NONNULL(key);
  MG_NONNULL(out);
  if (n < 1) return fail(MG_EINVAL, "n must be >= 1");
  uint32_t *d = nullptr;
  MG_CK(cudaMalloc(&d, (size_t)n * 40));
  cudaError_t e = cudaMemcpy(d, ctr, (size_t)n * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + 4 * n, key, (size_t)n * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_philox(d, d + 4 * n, d + 6 * n, n, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, d + 6 * n, (size_t)n * 16, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail_cuda(e, "mg_philox4x32_10");
  return MG_OK;
}

mg_status mg_kernel_info(mg_sim *s, int32_t *regs, int32_t *max_threads, int32_t *local_bytes) {
  MG_NONNULL(s);
  cudaFuncAttributes a;
  int per_sm = 0;
  if (s->queue)
    MG_CK(queue_kernel_attributes(s->ntv, s->diag, s->wide, s->structured, s->has_xh, &a,
                                  &per_sm));
  else
    MG_CK(fleet_kernel_attributes(s->ntv, s->diag, s->structured, false, s->wide, &a));
  if (regs) *regs = a.numRegs;
  if (max_threads) *max_threads = a.maxThreadsPerBlock;
  if (local_bytes) *local_bytes = (int32_t)a.localSizeBytes;
  return MG_OK;
}

}  // extern "C"
