// Internal data layout of a fleet in HBM and the launch-side structs shared by the host API
// and the kernels.  Everything is structure-of-arrays: plane j of a quantity is an array over
// envs, so that thread e's 16-byte load of plane j and thread e+1's are adjacent and a warp
// reads 512 contiguous bytes per plane.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "mg.h"

namespace mg {

// NVTX range around an entry point, for timeline tools (free when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Records msg as this thread's mg_last_error() and returns st (mg_api.cu).
mg_status set_error(mg_status st, const std::string &msg);

// ---------------------------------------------------------------- state planes
// 13 + n_thr floats per env packed into float4 planes (the 21-float record of mg.h minus
// padding):
//   S0 (px, py, pz, qw) | S1 (qx, qy, qz, u) | S2 (v, w, p, q) | S3 (r, n0, n1, n2)
//   S4 (n3, n4, n5, n6) | S5 n7 (a float plane, only touched by 8-thruster vehicles)
struct StatePlanes {
  float4 *s0, *s1, *s2, *s3, *s4;
  float *s5;
};

// ---------------------------------------------------------------- derived parameter planes
// What the step needs, derived once per parameter change (FP64 on the device, stored FP32).
// Diagonal-mass fleets (r_g = 0 everywhere, so M = M_RB + M_A is diagonal) read D0..D8 only:
//   D0 (m, Ma_u, Ma_v, Ma_w)       D1 (Jx, Jy, Jz, W - B)   J = diag(I_o) + Ma_rot
//   D2 (Dl_u, Dl_v, Dl_w, Dl_p)    D3 (Dl_q, Dl_r, Dq_u, Dq_v)   D4 (Dq_w, Dq_p, Dq_q, Dq_r)
//   D5 (Gx, Gy, Gz, kT)            G = W r_g - B r_b
//   D6 (vc_x, vc_y, vc_z, 1/tau_m) NED current
//   D7 (Mi00, Mi11, Mi22, Mi33)    D8 (Mi44, Mi55)            Mi = M^-1 (packed, symmetric)
// General fleets (some r_g != 0) also read:
//   G0 (m rg_x, m rg_y, m rg_z, Io_xy)   G1 (Io_xz, Io_yz, Mi01, Mi02)
//   G2 (Mi03, Mi04, Mi05, Mi12)          G3 (Mi13, Mi14, Mi15, Mi23)
//   G4 (Mi24, Mi25, Mi34, Mi35)          G5 Mi45
struct ParamPlanes {
  float4 *d0, *d1, *d2, *d3, *d4, *d5, *d6, *d7;
  float2 *d8;
  float4 *g0, *g1, *g2, *g3, *g4;
  float *g5;
};

// Per vehicle type: thruster count, unit directions d_i and moment arms r_i x d_i (w unused).
struct Geo {
  int32_t n_thr;
  int32_t pad[3];
  float4 dir[MG_MAX_THR];
  float4 arm[MG_MAX_THR];
};

// One thread block's slice of the fleet: envs [env0, env0 + count) all of vehicle type `type`.
struct BlockDesc {
  int32_t env0;
  int32_t count;
  int32_t type;
  int32_t n_thr;
};

// Everything a step kernel reads besides its block list; passed by value.
struct FleetView {
  StatePlanes st;
  ParamPlanes pa;
  const Geo *geo;            // device [n_types]
  int32_t n_types;
  int64_t n;                 // envs
  int64_t gid0;              // env id offset for counter-based draws
  const float *act;          // [n_seg][n][act_w] (16-byte aligned), or null
  int32_t act_w;             // floats per env and segment: MG_MAX_THR, or 6 (mg_set_action_width)
  int32_t n_seg;
  int32_t hold;
  uint64_t cmd_seed;         // procedural actions when proc != 0
  int32_t proc;
  uint32_t model_flags;
  float dt;
  uint32_t *flags;           // [n] bit 0 = non-finite
  unsigned long long *counters;  // [0] envs flagged non-finite, [2] work-queue wait time-outs
  // Action cursor (sub-steps since the actions were set) in device memory: every step launch
  // reads it at start and its last block to finish advances it, so a captured launch sequence
  // is valid whatever the cursor.  done_blocks counts finished blocks (reset by the last one).
  int64_t *cursor;
  unsigned int *done_blocks;
  // Per launch: the launch's sub-steps start at *cursor + cursor_off (the launch's offset within
  // its mg_step call), and a launch with cursor_adv != 0 (the call's last) advances *cursor by
  // cursor_adv once all its blocks are done.  Only that launch pays for the completion count.
  int32_t cursor_off;
  int32_t cursor_adv;
  // Work-queue schedule: polls of ~128 ns a unit's wait for its slice's previous chunk may take
  // before it gives up (counted in counters[2] and reported by mg_sync as MG_ETIMEOUT).
  uint32_t spin_limit;
  // Off-diagonal hydrodynamics, device [MG_NXPARAM][n] (component-major), or null: the static
  // and task kernels then run their XH variants (general path), staging each block's
  // coefficients in shared memory.
  const float *xh;
};

// Kernel variants: thruster count fixed at 6 or 8, or mixed (up to 8, read per block).
enum NtVariant { NT_6 = 0, NT_8 = 1, NT_MIXED = 2 };

// ---------------------------------------------------------------- launchers (mg_step.cu)
// Static schedule: one block per BlockDesc, k sub-steps per launch.
// structured: every vehicle type present has the vectored layout (thrusters 0..3 with d_z = 0,
// the rest with d_x = d_y = 0), so the allocation skips its exact zeros (diagonal mass only).
// wide: the diagonal-mass kernel without recording gets 200 registers instead of 128.
cudaError_t launch_fleet(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                         NtVariant ntv, bool diag, bool structured, bool wide, int32_t k,
                         float *traj, cudaStream_t stream);
cudaError_t fleet_kernel_attributes(NtVariant ntv, bool diag, bool structured, bool record,
                                    bool wide, cudaFuncAttributes *attr);

// Work-queue schedule: warps claim (32-env slice, chunk of sub-steps) units in chunk-major
// order.  sched: device words, zeroed by the launcher: [0] next unit, [1..3] unused,
// [4 + d] chunks completed by slice d.  One launch covers all k sub-steps (split into several
// if slices x chunks would not fit 31 bits).
constexpr int kQueueWarps = 4;
size_t queue_sched_bytes(int n_slices);
// wide: 200-register variant of the diagonal-mass step (fewer resident warps, more registers
// each); warps_per_sm > 0 caps the resident warps per SM.
cudaError_t launch_fleet_queue(const FleetView &fv, const BlockDesc *slices, int n_slices,
                               NtVariant ntv, bool diag, bool structured, bool wide,
                               int warps_per_sm, int32_t k, int32_t chunk, uint32_t *sched,
                               int n_sm, cudaStream_t stream);
// xh: the general path's off-diagonal-hydrodynamics variant.
cudaError_t queue_kernel_attributes(NtVariant ntv, bool diag, bool wide, bool structured,
                                    bool xh, cudaFuncAttributes *attr, int *blocks_per_sm);

// True when thrusters [0, 4) of the geometry have d_z = 0 and the rest d_x = d_y = 0.
bool vectored_layout(const Geo &g);

// ---------------------------------------------------------------- launchers (mg_setup.cu)
struct SetupView {
  int64_t n;
  int64_t gid0;
  const int32_t *types;      // device [n]
  float *raw;                // device [n][MG_NPARAM] (the record layout of mg.h)
  ParamPlanes pa;
  unsigned long long *n_not_spd;
  unsigned int *any_offdiag;
  const float *xh;           // device [MG_NXPARAM][xh_stride] off-diagonal hydrodynamics, or null
  int64_t xh_stride;         // floats between xh's component planes (0: n)
};

// background_blocks > 0: at most that many 64-thread blocks striding over the fleet (leaves room
// for a step kernel running concurrently on another stream); 0: one env per thread.
cudaError_t launch_randomize(const SetupView &v, const float *nominal /*dev [n_types][35]*/,
                             uint64_t seed, double lo, double hi, double current_sigma,
                             double rg_halfwidth, cudaStream_t stream, int background_blocks = 0);
cudaError_t launch_import_params(const SetupView &v, const float *in /*dev [n][35]*/,
                                 cudaStream_t stream);
// [n][MG_NXPARAM] records <-> [MG_NXPARAM][stride] planes (to_planes: records -> planes); the
// planes' first n floats of each component are read or written.  stride 0: n.
cudaError_t launch_xh_transpose(const float *in, float *out, int64_t n, bool to_planes,
                                cudaStream_t stream, int64_t stride = 0);
cudaError_t launch_export_params(const SetupView &v, float *out /*dev [n][35]*/,
                                 cudaStream_t stream);
cudaError_t launch_reset(const StatePlanes &st, int64_t n, int64_t gid0, const uint8_t *mask,
                         uint64_t seed, double nu0_sigma, uint32_t *episode, uint32_t *flags,
                         unsigned long long *nonfinite_count, cudaStream_t stream);
cudaError_t launch_export_state(const StatePlanes &st, int64_t n, float *out,
                                cudaStream_t stream);
cudaError_t launch_import_state(const StatePlanes &st, int64_t n, const float *in,
                                cudaStream_t stream);
cudaError_t launch_flags_to_bytes(const uint32_t *flags, int64_t n, uint8_t *out,
                                  cudaStream_t stream);
cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                          cudaStream_t stream);

// ---------------------------------------------------------------- job pool (mg_pool.cu)
// The pool's stream and arena capacity, for the native request loop (mg_serve.cu).
cudaStream_t pool_stream(const mg_pool *p);
int64_t pool_capacity(const mg_pool *p);

// ---------------------------------------------------------------- launchers (mg_adjoint.cu)
cudaError_t launch_checkpoint(const StatePlanes &st, int64_t n, float *ck, cudaStream_t stream);
// The rollout's forward in one launch on the static grid (mg_adjoint.cu): T sub-steps, ckpt
// [ceil(T / C)][MG_NSTATE][n] before sub-steps 0, C, ..., traj [T][MG_NTRAJ][n] after each.
cudaError_t launch_rollout_forward(const FleetView &fv, const BlockDesc *blocks, int n_blocks,
                                   int threads, NtVariant ntv, bool diag, bool structured,
                                   int32_t T, int32_t C, float *traj, float *ckpt,
                                   cudaStream_t stream);
// Backward kernel: mode 1 one warp per 32 envs, 2 the two-warp form (producer and consumer warps
// per 32 envs, through a workspace of adjoint_workspace_bytes), 0 chosen by fleet size.
cudaError_t adjoint_split(int64_t n, int mode, bool *split);
size_t adjoint_workspace_bytes(bool eight, int64_t n, int32_t C);
// general: the general-path kernels (off-centre gravity, off-diagonal extension, full M^-1).
cudaError_t launch_adjoint(const FleetView &fv, const int32_t *types, bool eight, bool general,
                           const float *ckpt, const float *dtraj, int32_t T, int32_t C,
                           int64_t step0, float *dcoef, float *dact, float *dstate0, bool split,
                           float *ws, cudaStream_t stream);
int adjoint_max_interval();

// ---------------------------------------------------------------- launchers (mg_task.cu)
struct TaskView {
  int32_t task, m;           // MG_TASK_*, look-ahead points
  float radius, omega, vz, psi_r, dt_look, max_err;
  int32_t episode_steps;     // auto-reset after this many sub-steps (0: never)
  const float4 *centre;      // [n] (cx, cy, cz, phi0)
  int32_t *clock;            // [n] sub-steps since the episode started
  float *err_sum;            // [n] Eq. 4 error summed over the episode's task steps
};

// Split-integration comparison step (mg_split.cu): k sub-steps of the engine-style scheme on the
// static grid; raw [n][MG_NPARAM] parameter records, accel [6][n] acceleration memory (in/out).
// general: the full M_RB (off-centre gravity) and fv.xh's off-diagonal M_A / D_l (or none).
cudaError_t launch_split(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                         NtVariant ntv, bool general, const float *raw, float *accel, int32_t k,
                         cudaStream_t stream);

// Outputs and reset inputs of the fused task step.
struct TaskOut {
  float *obs;        // [n][obs_dim]
  float *err;        // [n] or null
  uint8_t *done;     // [n]
  float *ep_err;     // [n] or null
  int32_t obs_dim;
  int32_t stage;     // set by the launcher: rows staged through shared memory
  uint64_t seed;     // episode-start draws (as mg_reset)
  double sigma;
  uint32_t *episode;
  float *reward;     // [n] or null: the negative error
};

// Final launch of a task step: k_launch sub-steps (static grid), then the task epilogue for a
// task step of k_task sub-steps in total.
cudaError_t launch_fleet_task(const FleetView &fv, const BlockDesc *blocks, int n_blocks,
                              int threads, NtVariant ntv, bool diag, bool structured,
                              int32_t k_launch, int32_t k_task, const TaskView &tv, TaskOut to,
                              cudaStream_t stream);

// Throttles clamped to [-1, 1] (NaN kept): out[i] = clamp(in[i]) for i < count.
cudaError_t launch_clamp_actions(const float *in, float *out, int64_t count, cudaStream_t stream);

cudaError_t launch_task(const StatePlanes &st, const TaskView &tv, int64_t n, int64_t gid0,
                        int32_t k, float dt, float *obs, float *err, uint8_t *done,
                        float *ep_err, uint64_t seed, double sigma, uint32_t *episode,
                        uint32_t *flags, unsigned long long *nonfinite_count,
                        cudaStream_t stream);

}  // namespace mg
