/*
 * mg.h — C ABI of the GB300 Fossen fleet stepper (libmg.so).
 *
 * The library advances many independent underwater vehicles ("envs") by the extended Fossen
 * equation of §METHOD (Eq. 1):
 *
 *   tau = M_RB nu' + C_RB(nu) nu + g_RB(eta) + M_A nu' + C_A(nu_r) nu_r + D(nu_r) nu_r + g_A(eta)
 *
 * with eta the pose in NED, nu = (u,v,w,p,q,r) the body-frame velocity, nu_r the velocity
 * relative to an ocean current constant in NED, tau the thruster wrench from per-thruster
 * throttle actions (Eq. 3) with a first-order motor lag.  Each sub-step (§METHOD, "multiple
 * sub-simulation steps within a single simulation step") is one classical RK4 step of size dt
 * with the command held over the step; the attitude quaternion is renormalised after it.
 *
 * Conventions shared by every call:
 *   - Body frame x forward, y starboard, z down; quaternion q = (w,x,y,z), Hamilton, body -> NED.
 *   - A pointer argument marked "host or device" may be either; the library asks the CUDA
 *     runtime which.  Device pointers are read or written asynchronously on the sim's stream
 *     (mg_set_stream); a host pointer makes the call synchronous (it returns once the data has
 *     been copied).  The caller owns every pointer it passes and may free it once the call has
 *     returned (device inputs: once the stream has passed the call).
 *   - The library owns every device buffer it allocates; mg_destroy frees them.
 *   - Every call returns an mg_status.  Nothing throws across the ABI.  On failure
 *     mg_last_error() gives a thread-local message.  Argument errors are found on the host and
 *     change nothing.
 *   - All floating-point state and parameters are FP32 on the device.  The 6x6 mass matrix is
 *     inverted in FP64 when parameters change (mg_randomize, mg_set_params).
 */
#ifndef MG_H
#define MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_NPARAM 35   /* per-env parameter record, layout below */
#define MG_NSTATE 21   /* per-env state record: p(3) q(4) nu(6) n(8) */
#define MG_NTRAJ 13    /* per-env trajectory record: p(3) q(4) nu(6) */
#define MG_MAX_THR 8   /* thrusters per vehicle type */
#define MG_MAX_TYPES 8 /* vehicle types per sim */

/* Parameter record (MG_NPARAM floats per env, "[n][MG_NPARAM]" below):
 *   0 m | 1..3 Ixx Iyy Izz about the centre of gravity | 4..9 added mass M_A (diagonal)
 *   10..15 linear damping (diagonal) | 16..21 quadratic damping (diagonal) | 22 W | 23 B
 *   24..26 r_g | 27..29 r_b | 30 k_T (thrust = k_T n|n| N) | 31 tau_m (motor lag, s)
 *   32..34 ocean current, NED, m/s */
#define MG_P_M 0
#define MG_P_IG 1
#define MG_P_MA 4
#define MG_P_DL 10
#define MG_P_DQ 16
#define MG_P_W 22
#define MG_P_B 23
#define MG_P_RG 24
#define MG_P_RB 27
#define MG_P_KT 30
#define MG_P_TAU 31
#define MG_P_VC 32

/* Off-diagonal hydrodynamic extension (MG_NXPARAM floats per env, optional; mg_set_hydro_offdiag):
 *   0..14  added mass M_A above its diagonal, row-major: (0,1) (0,2) (0,3) (0,4) (0,5) (1,2)
 *          (1,3) (1,4) (1,5) (2,3) (2,4) (2,5) (3,4) (3,5) (4,5); M_A is symmetric
 *   15..44 linear damping D_l off its diagonal, row-major with the diagonal skipped:
 *          (0,1)..(0,5) (1,0) (1,2)..(1,5) ... (5,0)..(5,4)
 * The diagonals stay in the parameter record; an all-zero extension is the diagonal model. */
#define MG_NXPARAM 45

typedef struct mg_sim mg_sim; /* opaque; owns all of a fleet's device buffers */

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,      /* bad argument; nothing changed */
  MG_ENOMEM = 2,      /* device allocation failed */
  MG_ECUDA = 3,       /* a CUDA runtime call failed; see mg_last_error() */
  MG_ENONFINITE = 4,  /* some env's state became NaN/Inf (mg_sync) */
  MG_ENOTSPD = 5,     /* some env's mass matrix M_RB + M_A is not positive definite */
  MG_ETIMEOUT = 6,    /* a bounded wait gave up */
  MG_ESTATE = 7       /* call not valid in the sim's current state */
} mg_status;

/* Nominal parameters and thruster geometry of one vehicle type (§METHOD: BlueROV2 and
 * BlueROV2 Heavy).  Vectors are in the body frame above.  d[i] is a unit direction. */
typedef struct {
  float m, Ixx, Iyy, Izz;
  float MA[6], Dl[6], Dq[6];
  float W, B;
  float rg[3], rb[3];
  float kT, tau_m;
  int32_t n_thr; /* 1..MG_MAX_THR */
  float r[MG_MAX_THR][3], d[MG_MAX_THR][3];
} mg_vehicle_params;

/* Domain-randomisation ranges (§METHOD "physical parameter domain randomization"): each of the
 * 27 scalars m, Ixx, Iyy, Izz, M_A(6), Dl(6), Dq(6), W, B, r_b.z, k_T, tau_m is scaled by
 * U[lo, hi]; the NED current is N(0, current_sigma) per axis; with rg_halfwidth > 0 the centre
 * of gravity is the nominal one plus U[-rg_halfwidth, rg_halfwidth] m per axis (off-centre
 * gravity: the fleet then takes the general mass-matrix path); mg_reset draws the initial body
 * velocity N(0, nu0_sigma) per component.  flags must be 0. */
typedef struct {
  float lo, hi;
  float current_sigma;
  float nu0_sigma;
  uint32_t flags;     /* 0 or MG_RANDOMIZE_ASYNC */
  float rg_halfwidth;
} mg_ranges;

/* mg_ranges.flags: return without waiting for the new parameters (the next calls queue behind
 * them on the stream).  Only for fleets whose mass matrices are known on the host to be diagonal
 * (every vehicle type with r_g = 0, rg_halfwidth = 0, no off-diagonal extension); a mass matrix
 * that is not positive definite is then reported by mg_sync (MG_ENOTSPD) instead of by
 * mg_randomize. */
#define MG_RANDOMIZE_ASYNC 1u

/* Model switch: drop the added-mass inertia of the current, M_A [omega x v_c^b; 0], which
 * follows from nu_r' = nu' + [omega x v_c^b; 0] for a current constant in NED. */
#define MG_MODEL_NO_CURRENT_ACCEL 1u

/* Create a fleet of n_envs vehicles (§METHOD: "parallel execution of multiple environment
 * instances").  vehicle_types: host [n_envs], values in [0, n_types).  params: host
 * [n_types].  Each env starts with its type's nominal parameters, no current, zero state with
 * identity attitude, zero actions.  Envs of one type that are adjacent in the index order are
 * processed together; interleaving types costs throughput, not correctness.  The device is the
 * caller's current CUDA device.  Errors: MG_EINVAL (n_envs < 1, n_types out of [1,
 * MG_MAX_TYPES], a type id out of range, n_thr out of [1, MG_MAX_THR]), MG_ENOMEM, MG_ECUDA. */
mg_status mg_create(int64_t n_envs, const int32_t *vehicle_types,
                    const mg_vehicle_params *params, int32_t n_types, mg_sim **out);

/* Free the sim and all its device buffers (synchronises its stream first). NULL is a no-op. */
mg_status mg_destroy(mg_sim *sim);

/* Stream every later call runs on (a cudaStream_t; NULL = the legacy default stream). */
mg_status mg_set_stream(mg_sim *sim, void *cuda_stream);

/* Offset added to env indices wherever they key a counter-based draw (randomisation, reset,
 * procedural commands), so that disjoint shards of one logical fleet draw what the whole fleet
 * would.  Default 0. */
mg_status mg_set_env_id_offset(mg_sim *sim, int64_t offset);

/* MG_MODEL_* bits.  Default 0 (full model).  The diagonal-mass kernels fold the current term
 * into their coefficients, so with MG_MODEL_NO_CURRENT_ACCEL every fleet steps on the general
 * path (same results within rounding, more arithmetic per sub-step). */
mg_status mg_set_model_flags(mg_sim *sim, uint32_t flags);

/* Sub-step size dt in seconds (default 0.01).  MG_EINVAL unless 0 < dt <= 1. */
mg_status mg_set_timestep(mg_sim *sim, float dt);

/* Launch shape: envs_per_block in [32, 256] (one thread per env), steps_per_launch >= 1 (RK4
 * steps a kernel keeps state in registers for; 1 gives the plain per-step form), use_graph
 * != 0 to replay mg_step's launch sequence from a cached CUDA graph.  Defaults 128, 50, 1. */
mg_status mg_set_launch(mg_sim *sim, int32_t envs_per_block, int32_t steps_per_launch,
                        int32_t use_graph);

/* Schedule of mg_step.  work_queue != 0 runs all k sub-steps in one launch in which
 * warps claim (32-env slice, steps_per_launch-chunk) units from a queue in chunk-major order,
 * each unit waiting (bounded, see MG_ETIMEOUT in mg_sync) for its slice's previous chunk; faster
 * warps take more units, which balances the SMs when the fleet has more 32-env slices than
 * resident warps.  wide != 0 (default) gives that kernel, and the static grid's kernel
 * outside mg_step_record, up to 200 registers per thread instead of 128 (diagonal-mass fleets;
 * the general kernels always have 168): the queue at 8 warps/SM runs best with it, and a static
 * grid of few envs (a warp per scheduler or fewer) gains 6-7 %, while a large static grid
 * keeps more warps resident at 128; warps_per_sm > 0 caps the queue kernel's resident warps
 * per SM (0 = as many as fit).  work_queue = 0 (default) launches a static grid of
 * envs_per_block-env blocks per steps_per_launch sub-steps (steps_per_launch = 1: the plain
 * per-step form).  All choices give bit-identical results.  mg_step_record always uses the
 * static grid.  MG_EINVAL unless 0 <= warps_per_sm <= 64. */
mg_status mg_set_schedule(mg_sim *sim, int32_t work_queue, int32_t wide, int32_t warps_per_sm);

/* Bound on each wait of the work-queue schedule (a unit waiting for its slice's previous chunk):
 * at most `polls` polls of about 128 ns each (0 restores the default MG_WAIT_POLLS_DEFAULT,
 * about half a second).  A wait that runs out is counted, the unit goes on without the chunk it
 * waited for (its results are then unreliable, but every access stays in bounds and the launch
 * ends), and the next mg_sync returns MG_ETIMEOUT.  A failure-detection knob: a limit far below
 * a chunk's run time makes waits give up on purpose.  MG_EINVAL if polls > 2^30. */
#define MG_WAIT_POLLS_DEFAULT 4194304u
mg_status mg_set_wait_limit(mg_sim *sim, uint32_t polls);

/* Domain randomisation (§METHOD; §EXPERIMENTS "supports domain randomization"): per env, draws
 * from Philox4x32-10 keyed by (seed, env id + offset), then builds M = M_RB + M_A in FP64 and
 * inverts it by Cholesky.  Also records (seed, nu0_sigma) for mg_reset and zeroes every env's
 * episode counter.  Synchronous unless ranges->flags has MG_RANDOMIZE_ASYNC.  Errors: MG_EINVAL
 * (ranges NULL, lo > hi, lo <= 0, negative sigma or half-width, unknown flags, MG_RANDOMIZE_ASYNC
 * for a fleet whose mass matrices may be full), MG_ENOTSPD (parameters are stored but some mass
 * matrix has a pivot <= 0), MG_ECUDA. */
mg_status mg_randomize(mg_sim *sim, uint64_t seed, const mg_ranges *ranges);

/* Background randomisation (§METHOD's per-episode domain randomisation, drawn ahead): draws the
 * parameters mg_randomize(sim, seed, ranges) would draw into a second parameter buffer of the
 * sim, on the library's own stream, so that the draw runs while the sim's stream is still
 * stepping the current episode (a few 64-thread blocks striding over the fleet, leaving room on
 * every SM for a step kernel).  The draw waits only for the previous install's copy, never for
 * the sim's stream.  A later mg_randomize with the same seed, lo, hi and current_sigma, the same
 * env-id offset and rg_halfwidth 0 installs the buffer with one device-to-device copy on the
 * sim's stream (ordered after the draw) instead of drawing: the parameters are bit-identical to
 * a direct draw, and the rest of mg_randomize (nu0_sigma and the seed recorded for mg_reset,
 * episode counters zeroed, MG_RANDOMIZE_ASYNC) applies as usual.  Any other mg_randomize draws
 * directly and leaves the buffer in place; a new prefetch replaces it.  ranges->nu0_sigma and
 * ranges->flags are not used here.  The buffer (the sim's parameter planes and records, 360 B
 * per env) is allocated on first use.  Errors: MG_EINVAL (ranges as mg_randomize, or mass matrices
 * that may be full: some type with r_g != 0, rg_halfwidth != 0, or the off-diagonal extension
 * set), MG_ENOMEM, MG_ECUDA. */
mg_status mg_randomize_prefetch(mg_sim *sim, uint64_t seed, const mg_ranges *ranges);

/* Set every env's parameters from a [n][MG_NPARAM] record (host or device); inverts the mass
 * matrices as mg_randomize does.  Synchronous.  Errors: MG_EINVAL, MG_ENOTSPD, MG_ECUDA. */
mg_status mg_set_params(mg_sim *sim, const float *in);

/* Copy every env's parameters into out [n][MG_NPARAM] (host or device). */
mg_status mg_get_params(mg_sim *sim, float *out);

/* Full (non-diagonal) added mass and linear damping: set every env's off-diagonal extension from
 * x [n][MG_NXPARAM] (host or device; layout above), or clear it (x = NULL: the diagonal model).
 * The mass matrices are re-inverted in FP64 with the off-diagonal added mass; a fleet with a
 * non-zero extension steps on the general path (static grid or work queue, each block or warp
 * staging its envs' coefficients in shared memory; mg_step_split runs its general form).
 * mg_randomize and mg_set_params keep the extension.  Synchronous.  Errors: MG_EINVAL, MG_ENOMEM, MG_ENOTSPD
 * (stored, but some M_RB + M_A is not positive definite), MG_ECUDA. */
mg_status mg_set_hydro_offdiag(mg_sim *sim, const float *x);

/* Copy every env's off-diagonal extension into out [n][MG_NXPARAM] (host or device; zeros when
 * none is set). */
mg_status mg_get_hydro_offdiag(mg_sim *sim, float *out);

/* Width w of every action buffer below: floats per env and segment.  w = MG_MAX_THR (default:
 * rows padded to 8, entries past a vehicle's thruster count ignored) or w = 6 (24-byte rows
 * without padding: fleets whose vehicle types all have 6 thrusters, where padding would be a
 * quarter of the schedule's bytes).  Changing the width clears the current action schedule
 * (commands are zero until the next mg_set_actions*, cursor rewound).  Errors: MG_EINVAL (w not 6
 * or MG_MAX_THR; w = 6 with a type of another thruster count). */
mg_status mg_set_action_width(mg_sim *sim, int32_t w);

/* Throttle actions (Eq. 3: one throttle setting per thruster).  a: host or device
 * [n_seg][n_envs][w] (w from mg_set_action_width), entries past a vehicle's thruster count
 * ignored.  The library
 * copies it.  Sub-step j counted from this call (across later mg_step calls) uses segment
 * min(j / hold_steps, n_seg - 1).  n_seg = 0 (a may be NULL) sets all commands to zero.
 * Errors: MG_EINVAL (n_seg < 0, hold_steps < 1), MG_ENOMEM, MG_ECUDA. */
mg_status mg_set_actions(mg_sim *sim, const float *a, int32_t n_seg, int32_t hold_steps);

/* As mg_set_actions, but without a copy: the kernels read a (device, 16-byte aligned,
 * [n_seg][n_envs][w]) in place.  The caller keeps the buffer alive and unchanged until
 * the stream has passed every mg_step that uses it (e.g. a policy's output tensor consumed by the
 * next step).  Errors: MG_EINVAL (NULL or host pointer, misaligned, n_seg < 1, hold_steps < 1). */
mg_status mg_set_actions_borrowed(mg_sim *sim, const float *a, int32_t n_seg, int32_t hold_steps);

/* Procedural actions: throttle c_i = 2u - 1 with u from Philox4x32-10 keyed by (cmd_seed, env
 * id + offset, segment j / hold_steps), no end.  Replaces any action buffer.  Resets the action
 * cursor like mg_set_actions. */
mg_status mg_set_procedural_actions(mg_sim *sim, uint64_t cmd_seed, int32_t hold_steps);

/* Advance every env k >= 1 sub-steps (Eq. 1 integrated by RK4, §METHOD).  Asynchronous on the
 * stream; non-finite states are reported by mg_sync.  The action cursor is a word in the sim's
 * device memory: each step launch reads it when it starts and its last block advances it, so the
 * CUDA graph cached for a given k replays correctly at any cursor (one graph per distinct k, at
 * most 16 kept).  Steps of one sim must therefore stay ordered on its stream. */
mg_status mg_step(mg_sim *sim, int32_t k);

/* Split-integration comparison step (§METHOD: the physics engine integrates the rigid-body term
 * of Eq. 1 and the hydrodynamic term is applied to the body as an external force), for
 * measuring the coupled (M_RB + M_A)^-1 step against the paper's own arrangement.  Per sub-step
 * of dt: tau_h = -(M_A (a + [w x v_c^b; 0]) + C_A(nu_r) nu_r + D(nu_r) nu_r + g_A), then
 * nu' = M_RB^-1 (tau + tau_h - C_RB(nu) nu - g_RB) and a semi-implicit Euler update (nu first,
 * then p with the new v, q with the new w, renormalised; explicit Euler on the throttle lag);
 * a <- nu'.  a stands in for the unknown nu' in the added-mass force (the previous sub-step's
 * acceleration), which makes the scheme unstable in any degree of freedom whose added mass
 * exceeds the rigid-body mass.  accel: device [6][n_envs] (component-major), in: the previous
 * sub-step's acceleration (zeros at an episode start), out: the last sub-step's.  Uses and
 * advances the action cursor like mg_step, the static grid with the sim's envs_per_block and
 * steps_per_launch, no graph; non-finite states are flagged as by mg_step.  A fleet with
 * off-centre gravity or the off-diagonal extension takes the general form: the full M_RB (its
 * inverse in closed form, w' = I_g^-1 (f_w - r_g x f_v), v' = f_v / m + r_g x w'), C_RB with the
 * m r_g terms, the weight's moment, and the full M_A and D_l in the hydrodynamic force.  Errors:
 * MG_EINVAL (k < 1, accel NULL or not device memory). */
mg_status mg_step_split(mg_sim *sim, int32_t k, float *accel);

/* As mg_step with the work-queue schedule, for callers that must not allocate device memory
 * while they step (for instance a real-time control loop whose memory is fixed up front, or code
 * that runs with its memory pool capped): the call launches the work-queue kernel directly (no
 * CUDA graph is instantiated, nothing is staged) and keeps the queue's scheduler words in a
 * fixed 256 KB device array compiled into the library instead of the sim's own buffers.  The
 * paper has no counterpart; it is an interface convenience around the same kernel.
 *   - The first call for a sim on a device looks up that array's address on the sim's device
 *     (once per device; the sim's device is made current for the look-up and the caller's
 *     current device restored); make that first call before any stream capture.
 *   - Fleets of at most 65,536 32-env slices (2,097,152 envs of one vehicle type) are accepted;
 *     larger ones get MG_EINVAL with a message saying so.
 *   - All calls, from every sim on the device, share the one array and it keeps the last call's
 *     contents: each call zeroes the words it uses on the sim's stream before its launch, and
 *     calls whose launches overlap on the GPU (two sims on different streams) race on it.
 * Uses the sim's steps_per_launch as the chunk size and the wide / warps_per_sm settings of
 * mg_set_schedule, whatever the schedule chosen there; results equal mg_step's bit for bit. */
mg_status mg_step_noalloc(mg_sim *sim, int32_t k);

/* As mg_step, also writing the state after every sub-step to traj: device
 * [k][MG_NTRAJ][n_envs] (component-major per step: p(3) q(4) nu(6)). Never graph-replayed. */
mg_status mg_step_record(mg_sim *sim, int32_t k, float *traj);

/* Forward rollout for differentiation: T sub-steps from the current state and action cursor
 * in one launch on the static grid (results equal mg_step_record's bit for bit; the
 * checkpoints are written from registers), writing the state after every sub-step to traj, device
 * [T][MG_NTRAJ][n], and the full state before sub-steps 0, C, 2C, ... to ckpt, device
 * [ceil(T / C)][MG_NSTATE][n] (component-major).  *step0_out (may be NULL) receives the action
 * cursor at the start; pass it to mg_rollout_backward.  Errors: MG_EINVAL (T < 1, C outside
 * [1, 32], host buffers). */
mg_status mg_rollout_forward(mg_sim *sim, int32_t T, int32_t C, float *traj, float *ckpt,
                             int64_t *step0_out);

/* Reverse pass of that rollout: the discrete adjoint of the FP32 RK4 sub-steps (renormalisation
 * included), re-running each C-step segment from its checkpoint.  dtraj: device
 * [T][MG_NTRAJ][n], the loss gradient with respect to traj.  Writes dcoef, device [n][18], the
 * gradient with respect to each env's added-mass, linear-damping and quadratic-damping diagonals
 * (record entries 4..21, §METHOD Eq. 1 hydrodynamic term); adds the gradient with respect to the
 * buffered actions (Eq. 3) into dact, device [n_seg][n][w] (w the action width; may be NULL);
 * writes the gradient with respect to the start state into dstate0, device [n][MG_NSTATE] (may
 * be NULL).  Every fleet the step covers: diagonal-mass fleets, and on the general path fleets
 * with off-centre gravity (r_g != 0) and / or the off-diagonal extension, where a diagonal
 * coefficient M_A,jj also enters the full M = M_RB + M_A (its share of the gradient is
 * -(M^-1 g)_j nu'_j for the loss adjoint g of nu').  Parameters, extension and actions must be
 * those of the forward; the sim's state is not read or changed.
 * Errors: MG_EINVAL (bad sizes, host buffers, procedural actions). */
mg_status mg_rollout_backward(mg_sim *sim, int32_t T, int32_t C, const float *ckpt,
                              const float *dtraj, int64_t step0, float *dcoef, float *dact,
                              float *dstate0);

/* Backward kernel of mg_rollout_backward.  mode 1: one thread per env, each re-running a
 * checkpoint segment and then walking it backwards.  mode 2: two warps per 32 envs, one
 * re-running the segments and recording every sub-step's RK4 stage states in a workspace
 * (2 x C x (4 (10 + N) + 4) floats per env, N = 6 or 8 thrusters; allocated by
 * mg_rollout_backward on first use), the other applying the transposes from those records one
 * segment behind, so that a small fleet keeps twice as many schedulers busy.  mode 0 (default):
 * mode 2 while 2 x ceil(n_envs / 32) warps fit one per scheduler of the GPU, else mode 1.  The
 * per-env arithmetic is the same in both.  MG_EINVAL unless 0 <= mode <= 2. */
mg_status mg_set_adjoint_mode(mg_sim *sim, int32_t mode);

/* State in the record layout [n][MG_NSTATE] = p(3) q(4: w,x,y,z) nu(6) n(8, zero past n_thr);
 * host or device. */
mg_status mg_get_state(mg_sim *sim, float *out);
mg_status mg_set_state(mg_sim *sim, const float *in);

/* Asynchronous transfers with page-locked host memory (cudaHostAlloc / cudaHostRegister), for
 * pipelines in which one episode's copies overlap the neighbouring episodes' steps.  Neither
 * call waits: each copy runs on a stream of the library's own, into or out of one of two device
 * buffers used alternately, ordered after the work that last used that buffer; mg_sync waits
 * for these copies too.  Results are those of the synchronous calls.
 *   mg_set_actions_async: as mg_set_actions (a: host [n_seg][n_envs][w], n_seg >= 1);
 *     the steps queued after the call read the copy once it has landed.  The caller keeps a
 *     unchanged until mg_sync returns, or until the second later call of mg_set_actions_async
 *     has returned (that call reuses this call's device buffer: it first waits on the host for
 *     this call's copy, and its own copy waits on the device for this call's steps).
 *   mg_get_state_async: as mg_get_state into out (host [n_envs][MG_NSTATE]) of the state the
 *     steps queued so far leave; out is complete once mg_sync returns.  A third call reuses the
 *     first call's device buffer only after its copy has finished.
 * Errors: MG_EINVAL (NULL, pageable or device memory, n_seg < 1, hold_steps < 1), MG_ENOMEM,
 * MG_ECUDA. */
mg_status mg_set_actions_async(mg_sim *sim, const float *a, int32_t n_seg, int32_t hold_steps);
mg_status mg_get_state_async(mg_sim *sim, float *out);

/* Start a new episode for every env whose mask byte is non-zero (mask: host or device
 * [n_envs]; NULL = all): p = 0, q = identity, n = 0, nu ~ N(0, nu0_sigma) drawn from Philox
 * keyed by (seed, env id + offset, the env's episode counter; Box-Muller evaluated in FP32),
 * then the counter is incremented and the env's non-finite flag cleared. */
mg_status mg_reset(mg_sim *sim, const uint8_t *mask);

/* Wait for the stream (and the asynchronous host copies and background randomisation, if any
 * have been issued); *nonfinite_count (may be NULL) receives how many envs are flagged
 * non-finite.  Returns MG_ETIMEOUT if a work-queue wait gave up since the last mg_sync (results
 * of those steps are unreliable: restore the state with mg_set_state or mg_reset; not expected
 * with the default limit of mg_set_wait_limit) and clears that count, else MG_ENOTSPD if the
 * current parameters hold a mass matrix that is not positive definite, else MG_ENONFINITE when
 * that count is non-zero. */
mg_status mg_sync(mg_sim *sim, int64_t *nonfinite_count);

/* Per-env non-finite flags into out [n_envs] (host or device), 1 = flagged. */
mg_status mg_get_nonfinite(mg_sim *sim, uint8_t *out);

/* ------------------------------------------------------------------------------------------
 * Task layer (§EXPERIMENTS): the four tasks of the paper's experiments on top of the step.  Each
 * env tracks a reference around its own centre c (NED) with phase phi0, s = omega t + phi0:
 *   MG_TASK_STATION     p_r = c                                   (station keeping)
 *   MG_TASK_CIRCLE      p_r = c + (R cos s, R sin s, 0)
 *   MG_TASK_HELIX       p_r = c + (R cos s, R sin s, vz t)
 *   MG_TASK_LEMNISCATE  p_r = c + R (cos s, sin s cos s, 0) / (1 + sin^2 s)
 * with a level attitude reference of heading psi_r.  Observation (Eq. 2), per env, obs_dim =
 * 6 m + 6 floats: for i = 1..m the position error p - p_r(t + i lookahead_dt) and the attitude
 * error (roll, pitch, heading - psi_r wrapped to [-pi, pi), zyx Euler angles of q), then nu; m =
 * 1 and p_r(t) for station keeping.  Position error (Eq. 4): |p - p_r(t)|, summed over an
 * episode's task steps.  t counts sub-steps since the env's episode started (times dt).
 * ------------------------------------------------------------------------------------------ */
#define MG_TASK_STATION 0
#define MG_TASK_CIRCLE 1
#define MG_TASK_HELIX 2
#define MG_TASK_LEMNISCATE 3

typedef struct {
  int32_t task;           /* MG_TASK_* */
  int32_t lookahead;      /* m >= 1 reference points observed (tracking tasks) */
  float radius, omega, vz, psi_r, lookahead_dt;
  float max_error;        /* an episode ends when |p - p_r| exceeds it (<= 0: never) */
  int32_t episode_steps;  /* an episode ends after this many sub-steps (<= 0: never) */
  uint32_t flags;         /* must be 0 */
} mg_task_spec;

/* Set the task; centres: host or device [n_envs][4] = (cx, cy, cz, phi0).  Every env's episode
 * clock and error sum restart at 0 (the state is not touched).  Errors: MG_EINVAL (NULL, unknown
 * task, lookahead < 1 or > 64, flags != 0), MG_ENOMEM. */
mg_status mg_set_task(mg_sim *sim, const mg_task_spec *spec, const float *centres);

/* Observation length 6 m + 6 of the current task (MG_ESTATE if no task is set). */
mg_status mg_task_obs_dim(mg_sim *sim, int32_t *obs_dim);

/* One task step: k >= 1 sub-steps (as mg_step), then for every env: err = |p - p_r(t)|, the
 * episode's clock and error sum advance, and an env whose episode ended (error above max_error,
 * episode_steps reached, or a non-finite state) gets done = 1, episode_err = its error sum
 * (including this step), and an automatic reset (as mg_reset); obs is then the new episode's
 * first observation.  The last min(k, steps_per_launch) sub-steps and all of the above run in
 * one fused launch on the static grid (earlier sub-steps as mg_step, with its schedule), so the
 * state is stored once.  k = 0 only observes (no step, no clock, no reset).  obs: device
 * [n][obs_dim]; err: device [n]; done: device [n]; episode_err: device [n] or NULL (0 for envs
 * that did not finish).  Asynchronous.  Errors: MG_ESTATE (no task), MG_EINVAL. */
mg_status mg_task_step(mg_sim *sim, int32_t k, float *obs, float *err, uint8_t *done,
                       float *episode_err);

/* One step of a Gym-style environment (§EXPERIMENTS: the tasks in a Gym-style format; the
 * action space of Eq. 3): the policy's throttles actions (device [n][w], w = the action width
 * of mg_set_action_width) are clamped to [-1, 1] (NaN kept) into the library's own
 * one-segment schedule, held over all k >= 1 sub-steps, and the task step of mg_task_step
 * follows, writing reward = -(Eq. 4 position error) instead of err.  The schedule replaces the
 * sim's actions on the first call (and after any other action call) and is rewritten in place
 * by the later ones, so a policy loop pays one small copy kernel per step.  actions may be
 * reused once the stream has passed the call.  obs, reward, done, episode_err: device, as
 * mg_task_step.  Asynchronous.  Errors: MG_ESTATE (no task), MG_EINVAL (k < 1, NULL, host
 * memory), MG_ENOMEM (the schedule's first allocation). */
mg_status mg_env_step(mg_sim *sim, int32_t k, const float *actions, float *obs, float *reward,
                      uint8_t *done, float *episode_err);

/* ------------------------------------------------------------------------------------------
 * Serving: a job pool with continuous batching.  A pool holds an arena of capacity_envs envs; a
 * job (one vehicle type, its own parameter and command seeds, hold and horizon) is admitted into
 * a contiguous free range, randomised and reset with draws keyed by its own seeds and job-local
 * env ids (its result does not depend on its placement or on the other jobs), and advanced by
 * mg_pool_tick together with every other running job in one launch.  Commands are procedural
 * (as mg_set_procedural_actions, keyed by cmd_seed and the job-local env id).
 * ------------------------------------------------------------------------------------------ */
typedef struct mg_pool mg_pool;

typedef struct {
  int64_t n_envs;
  int32_t vehicle_type;  /* index into the pool's vehicle table */
  int32_t hold_steps;    /* sub-steps each procedural command is held */
  int32_t horizon;       /* sub-steps to run */
  int32_t pad;
  uint64_t param_seed;   /* randomisation and reset draws */
  uint64_t cmd_seed;     /* procedural commands */
  mg_ranges ranges;      /* as mg_randomize */
} mg_job_spec;

/* Create a pool on the current device; params host [n_types].  Errors as mg_create. */
mg_status mg_pool_create(int64_t capacity_envs, const mg_vehicle_params *params, int32_t n_types,
                         mg_pool **out);
/* Wait for the device and free the pool's arena, planes and staging buffers (a job's traj
 * buffer stays the caller's).  NULL is a no-op. */
mg_status mg_pool_destroy(mg_pool *pool);
/* Stream every later pool call runs on (a cudaStream_t; NULL = the legacy default stream). */
mg_status mg_pool_set_stream(mg_pool *pool, void *cuda_stream);

/* Admit a job: takes a free range of spec->n_envs envs, randomises and resets them (asynchronous
 * on the pool's stream).  traj: device [horizon][MG_NTRAJ][n_envs] the ticks will record into,
 * owned by the caller and kept alive until the job is released, or NULL.  *job_id receives the
 * job's handle.  Errors: MG_EINVAL (bad spec, host traj), MG_ENOMEM (no free range large
 * enough; nothing changed). */
mg_status mg_pool_admit(mg_pool *pool, const mg_job_spec *spec, float *traj, int32_t *job_id);

/* mg_pool_admit for a job with the off-diagonal hydrodynamic extension (full M_A and D_l, the
 * layout of MG_NXPARAM above): xh [n_envs][MG_NXPARAM] (NULL: mg_pool_admit); host memory may
 * be reused once the call returns, device memory is read in order on the pool's stream (keep it
 * until that stream passes the call).  The job's M^-1 is derived with the off-diagonal added mass,
 * and the ticks advance it on the general path in a second launch beside the other jobs (whose
 * results do not change).  A job with the extension may randomise r_g in any pool.  The first
 * such job allocates the pool's [MG_NXPARAM][capacity_envs] planes (MG_ENOMEM if that fails;
 * nothing changed).  The native request loop takes such jobs through mg_server_submit_offdiag.
 * Errors as mg_pool_admit. */
mg_status mg_pool_admit_offdiag(mg_pool *pool, const mg_job_spec *spec, float *traj,
                                const float *xh, int32_t *job_id);

/* One launch: every admitted job with sub-steps left advances min(k, horizon - done) of them.
 * *n_running (may be NULL) receives how many jobs advanced.  Asynchronous. */
mg_status mg_pool_tick(mg_pool *pool, int32_t k, int32_t *n_running);

/* Sub-steps a job has been scheduled for (completed once the stream passes the last tick). */
mg_status mg_pool_job_progress(mg_pool *pool, int32_t job_id, int32_t *done, int32_t *horizon);

/* A job's state [n_envs][MG_NSTATE], host or device. */
mg_status mg_pool_get_job_state(mg_pool *pool, int32_t job_id, float *out);

/* Return a job's envs to the pool (its traj buffer is the caller's again). */
mg_status mg_pool_release(mg_pool *pool, int32_t job_id);

/* Free envs in total and in the largest contiguous range; admitted jobs. */
mg_status mg_pool_info(mg_pool *pool, int64_t *free_envs, int64_t *largest_free_range,
                       int32_t *n_jobs);

/* Wait for the pool's stream. */
mg_status mg_pool_sync(mg_pool *pool);

/* Native request loop over a pool (continuous batching; the paper has no serving layer).  Jobs
 * are submitted as specs and wait in a FIFO queue; each mg_server_poll admits queued jobs in
 * order while the trajectory budget and a free arena range allow, issues one mg_pool_tick
 * (every running job advances min(k, horizon - done) sub-steps in one launch), records an event
 * after it and hands back the jobs whose last tick has completed.  At most
 * max_inflight ticks stay queued beyond the oldest incomplete one; a poll that would exceed that,
 * or that has nothing left to advance, waits for the oldest by polling its event (spinning for
 * the first millisecond, never longer than wait_timeout_s: then MG_ETIMEOUT, and the server
 * stays usable).  Trajectory records ([horizon][MG_NTRAJ][n_envs] floats each, when record != 0)
 * are stream-ordered allocations of the server's own memory pool on the pool's stream, freed
 * when a job leaves.  A job's result is the one it gets alone or on any other pool (its draws
 * are keyed by its own seeds).  The server uses the pool's stream as set when it is created. */
typedef struct mg_server mg_server;

typedef struct {
  double budget_bytes;     /* device bytes the resident jobs' trajectory records may take */
  int32_t k;               /* sub-steps per tick, >= 1 */
  int32_t max_inflight;    /* ticks queued beyond the oldest incomplete one, >= 1 */
  int32_t record;          /* != 0: every job records its trajectory */
  int32_t serial;          /* != 0: one job at a time (admitted only into an empty server) */
  int32_t keep_done;       /* != 0: a finished job stays admitted until mg_server_release */
  int32_t pad;
  double wait_timeout_s;   /* longest a poll waits for a tick, > 0 */
} mg_server_config;

/* Create a server over pool (which it does not own; destroy the server first).  Errors:
 * MG_EINVAL (NULL, k < 1, max_inflight < 1, negative budget, wait_timeout_s <= 0), MG_ECUDA. */
mg_status mg_server_create(mg_pool *pool, const mg_server_config *cfg, mg_server **out);

/* Wait for the device, release every job still admitted and free all records. NULL: no-op. */
mg_status mg_server_destroy(mg_server *srv);

/* Queue a job; *ticket (0, 1, 2, ... in submission order) names it in the calls below.  Errors:
 * MG_EINVAL (n_envs outside [1, the pool's capacity], horizon or hold < 1, a record larger than
 * the whole budget). */
mg_status mg_server_submit(mg_server *srv, const mg_job_spec *spec, int64_t *ticket);

/* mg_server_submit for a job with the off-diagonal hydrodynamic extension: xh [n_envs]
 * [MG_NXPARAM] (host or device) is copied into host memory before the call returns and handed
 * to mg_pool_admit_offdiag at admission (the pool's extension planes are not part of the
 * trajectory budget).  Errors as mg_server_submit, and MG_ECUDA if xh cannot be read. */
mg_status mg_server_submit_offdiag(mg_server *srv, const mg_job_spec *spec, const float *xh,
                                   int64_t *ticket);

/* One round of the loop (above); the counts (any may be NULL) are those after it: jobs queued,
 * admitted and not yet handed back, ticks in flight.  Errors: MG_ETIMEOUT, MG_ECUDA, and those of
 * the pool calls. */
mg_status mg_server_poll(mg_server *srv, int32_t *n_queued, int32_t *n_running,
                         int32_t *n_inflight);

/* A job's submission, admission and completion times in seconds on the server's clock (from
 * mg_server_create; monotonic), -1 while not yet admitted / done. */
mg_status mg_server_job(mg_server *srv, int64_t ticket, double *submit_s, double *admit_s,
                        double *done_s);

/* A finished job kept by keep_done: its final state into state ([n_envs][MG_NSTATE], host or
 * device, may be NULL) and its record into traj ([horizon][MG_NTRAJ][n_envs], host or device,
 * may be NULL).  Synchronous.  Errors: MG_EINVAL, MG_ESTATE (not finished, not kept, released,
 * or no record). */
mg_status mg_server_job_result(mg_server *srv, int64_t ticket, float *state, float *traj);

/* Release a finished job kept by keep_done (its envs and record).  Errors: MG_EINVAL, MG_ESTATE. */
mg_status mg_server_release(mg_server *srv, int64_t ticket);

/* The server's clock now, and the bytes of records held now and at most so far (any may be
 * NULL). */
mg_status mg_server_info(mg_server *srv, double *now_s, double *used_bytes, double *peak_bytes);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *mg_last_error(void);

/* Evaluate Philox4x32-10 on the device for n (counter, key) pairs: ctr host [n][4], key host
 * [n][2], out host [n][4].  The same generator keys every draw above; exposed so it can be
 * checked bit for bit against the published known answers. */
mg_status mg_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n);

/* Kernel attributes of the step kernel the sim would launch now (registers per thread,
 * maximum threads per block, local-memory bytes per thread); any pointer may be NULL. */
mg_status mg_kernel_info(mg_sim *sim, int32_t *regs, int32_t *max_threads, int32_t *local_bytes);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
