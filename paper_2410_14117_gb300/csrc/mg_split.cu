// Split-integration comparison step (§METHOD): the paper's arrangement of Eq. 1, in which the
// physics engine integrates the rigid-body term and a separate module computes the
// hydrodynamic term and applies it to the body as an external force.  One sub-step of h:
//
//   tau_h = -( M_A (a + [w x v_c^b; 0]) + C_A(nu_r) nu_r + D(nu_r) nu_r + g_A )
//   nu'   = M_RB^-1 ( tau + tau_h - C_RB(nu) nu - g_RB )
//   nu+ = nu + h nu',  p+ = p + h R(q) v+,  q+ = normalise(q + h/2 q (x) (0, w+)),
//   n+  = n + h (c - n) / tau_m,  a+ = nu'
//
// a is the previous sub-step's acceleration (the added-mass force needs nu', unknown when the
// force is computed); g_RB is the weight's part of the restoring vector, g_A the buoyancy's.
// Diagonal-mass fleets (r_g = 0: M_RB = diag(m, m, m, Ixx, Iyy, Izz)) take the plain form; the
// general form (GEN) has the full M_RB of an off-centre gravity and the off-diagonal M_A and
// D_l of the extension.  The kernel is a comparison point for the coupled (M_RB + M_A)^-1 step,
// not a production path: it reads the raw parameter records once per launch and keeps no
// derived planes.
#include "mg_advance.cuh"

namespace mg {

namespace {

struct SplitPar {
  float m, I[3], ma[6], dl[6], dq[6];
  float W, B, rg[3], rb[3], kT, itau, vc[3];
};

__device__ __forceinline__ void load_split_par(const float *__restrict__ raw, int64_t e,
                                               SplitPar &P) {
  const float *r = raw + e * MG_NPARAM;
  P.m = r[MG_P_M];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    P.I[i] = r[MG_P_IG + i];
    P.rg[i] = r[MG_P_RG + i];
    P.rb[i] = r[MG_P_RB + i];
    P.vc[i] = r[MG_P_VC + i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    P.ma[i] = r[MG_P_MA + i];
    P.dl[i] = r[MG_P_DL + i];
    P.dq[i] = r[MG_P_DQ + i];
  }
  P.W = r[MG_P_W];
  P.B = r[MG_P_B];
  P.kT = r[MG_P_KT];
  P.itau = 1.f / r[MG_P_TAU];
}

__device__ __forceinline__ void cross(const float a[3], const float b[3], float c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// y = M x for the symmetric added-mass matrix: diagonal d, entries above it from the extension
// record x (row-major: 01 02 03 04 05 12 ... 45).
__device__ __forceinline__ void sym6_apply(const float d[6], const float *__restrict__ u,
                                           const float x[6], float y[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = d[i] * x[i];
  int t = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j, ++t) {
      y[i] = fmaf(u[t], x[j], y[i]);
      y[j] = fmaf(u[t], x[i], y[j]);
    }
}

// One split sub-step of env state s with acceleration memory a (updated in place).  cs: the
// held command divided by tau_m (as load_commands returns it).  GEN: xh is the env's extension
// record (MG_NXPARAM floats; zeros for an env without one).
template <int MT, bool GEN>
__device__ __forceinline__ void split_substep(St<MT> &s, float (&a)[6], const float (&cs)[MT],
                                              const SplitPar &P, const float4 *gdir,
                                              const float4 *garm, int nt, bool current_accel,
                                              float h, const float *__restrict__ xh) {
  const float qw = s.q[0], qx = s.q[1], qy = s.q[2], qz = s.q[3];
  // R(q) = I + 2 qw S(eps) + 2 S(eps)^2, body -> NED
  float R[3][3];
  R[0][0] = 1.f - 2.f * (qy * qy + qz * qz);
  R[0][1] = 2.f * (qx * qy - qw * qz);
  R[0][2] = 2.f * (qx * qz + qw * qy);
  R[1][0] = 2.f * (qx * qy + qw * qz);
  R[1][1] = 1.f - 2.f * (qx * qx + qz * qz);
  R[1][2] = 2.f * (qy * qz - qw * qx);
  R[2][0] = 2.f * (qx * qz - qw * qy);
  R[2][1] = 2.f * (qy * qz + qw * qx);
  R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
  const float k[3] = {R[2][0], R[2][1], R[2][2]};  // R^T e3: the body-frame "down"
  float vcb[3], vr[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    vcb[i] = R[0][i] * P.vc[0] + R[1][i] * P.vc[1] + R[2][i] * P.vc[2];
    vr[i] = s.v[i] - vcb[i];
  }
  const float *w = s.w;

  // hydrodynamic module: added mass (lagged acceleration + current term), added-mass
  // Coriolis, damping, buoyancy
  float acc[3] = {a[0], a[1], a[2]};
  if (current_accel) {
    float wx[3];
    cross(w, vcb, wx);
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] += wx[i];
  }
  float Q1[3], Q2[3], mf[6], dmp[6];  // M_A nu_r, M_A (a + [w x v_c^b; 0]), D(nu_r) nu_r
  if constexpr (GEN) {
    const float nr[6] = {vr[0], vr[1], vr[2], w[0], w[1], w[2]};
    const float ac[6] = {acc[0], acc[1], acc[2], a[3], a[4], a[5]};
    float Q[6];
    sym6_apply(P.ma, xh, nr, Q);
    sym6_apply(P.ma, xh, ac, mf);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Q1[i] = Q[i];
      Q2[i] = Q[3 + i];
    }
    const float *dl = xh + 15;  // D_l off its diagonal, row-major, the diagonal skipped
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float x = (P.dl[i] + P.dq[i] * fabsf(nr[i])) * nr[i];
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if (j != i) x = fmaf(dl[5 * i + (j < i ? j : j - 1)], nr[j], x);
      dmp[i] = x;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Q1[i] = P.ma[i] * vr[i];
      Q2[i] = P.ma[3 + i] * w[i];
      mf[i] = P.ma[i] * acc[i];
      mf[3 + i] = P.ma[3 + i] * a[3 + i];
      dmp[i] = (P.dl[i] + P.dq[i] * fabsf(vr[i])) * vr[i];
      dmp[3 + i] = (P.dl[3 + i] + P.dq[3 + i] * fabsf(w[i])) * w[i];
    }
  }
  float ca_f[3], ca_m[3], t1[3], t2[3];
  cross(w, Q1, ca_f);
  cross(vr, Q1, t1);
  cross(w, Q2, t2);
  float rbk[3];
  cross(P.rb, k, rbk);
  float th_f[3], th_m[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ca_m[i] = t1[i] + t2[i];
    th_f[i] = -(mf[i] + ca_f[i] + dmp[i] + P.B * k[i]);
    th_m[i] = -(mf[3 + i] + ca_m[i] + dmp[3 + i] + P.B * rbk[i]);
  }

  // thrusters (lag state at the start of the sub-step)
  float tf[3] = {0.f, 0.f, 0.f}, tm[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const float F = P.kT * s.n[i] * fabsf(s.n[i]);
    const float4 d = gdir[i], r = garm[i];
    tf[0] += F * d.x; tf[1] += F * d.y; tf[2] += F * d.z;
    tm[0] += F * r.x; tm[1] += F * r.y; tm[2] += F * r.z;
  }

  // rigid body: M_RB nu' = tau + tau_h - C_RB(nu) nu - g_RB
  float nd[6];
  if constexpr (GEN) {
    // Momenta [P1; P2] = M_RB nu: P1 = m (v + w x r_g), P2 = m r_g x v + I_o w with
    // I_o = I_g - m S(r_g)^2; C_RB(nu) nu = [w x P1; v x P1 + w x P2]; g_RB = -W [k; r_g x k].
    float wr[3], rv[3], rw[3], rrw[3], P1[3], P2[3];
    cross(w, P.rg, wr);
    cross(P.rg, s.v, rv);
    cross(P.rg, w, rw);
    cross(P.rg, rw, rrw);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      P1[i] = P.m * (s.v[i] + wr[i]);
      P2[i] = P.m * rv[i] + (P.I[i] * w[i] - P.m * rrw[i]);
    }
    float c1[3], c2[3], c3[3], rk[3];
    cross(w, P1, c1);
    cross(s.v, P1, c2);
    cross(w, P2, c3);
    cross(P.rg, k, rk);
    float f1[3], f2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      f1[i] = tf[i] + th_f[i] - c1[i] + P.W * k[i];
      f2[i] = tm[i] + th_m[i] - (c2[i] + c3[i]) + P.W * rk[i];
    }
    // M_RB^-1 in closed form (its Schur complement is I_g): w' = I_g^-1 (f2 - r_g x f1),
    // v' = f1 / m + r_g x w'
    float rf[3];
    cross(P.rg, f1, rf);
#pragma unroll
    for (int i = 0; i < 3; ++i) nd[3 + i] = (f2[i] - rf[i]) / P.I[i];
    float rwd[3];
    cross(P.rg, nd + 3, rwd);
#pragma unroll
    for (int i = 0; i < 3; ++i) nd[i] = f1[i] / P.m + rwd[i];
  } else {
    // r_g = 0: g_RB = -[W k; 0], C_RB(nu) nu = [w x m v; w x I_g w]
    float mv[3], Iw[3], crb_f[3], crb_m[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      mv[i] = P.m * s.v[i];
      Iw[i] = P.I[i] * w[i];
    }
    cross(w, mv, crb_f);
    cross(w, Iw, crb_m);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      nd[i] = (tf[i] + th_f[i] - crb_f[i] + P.W * k[i]) / P.m;
      nd[3 + i] = (tm[i] + th_m[i] - crb_m[i]) / P.I[i];
    }
  }

  // semi-implicit Euler
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.v[i] += h * nd[i];
    s.w[i] += h * nd[3 + i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    s.p[i] += h * (R[i][0] * s.v[0] + R[i][1] * s.v[1] + R[i][2] * s.v[2]);
  const float hh = 0.5f * h;
  float q0 = qw - hh * (qx * s.w[0] + qy * s.w[1] + qz * s.w[2]);
  float q1 = qx + hh * (qw * s.w[0] + qy * s.w[2] - qz * s.w[1]);
  float q2 = qy + hh * (qw * s.w[1] + qz * s.w[0] - qx * s.w[2]);
  float q3 = qz + hh * (qw * s.w[2] + qx * s.w[1] - qy * s.w[0]);
  const float inv = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  s.q[0] = q0 * inv;
  s.q[1] = q1 * inv;
  s.q[2] = q2 * inv;
  s.q[3] = q3 * inv;
#pragma unroll
  for (int i = 0; i < MT; ++i) s.n[i] = (i < nt) ? s.n[i] + h * (cs[i] - s.n[i] * P.itau) : 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) a[i] = nd[i];
}

// GEN: each block stages its envs' extension records in dynamic shared memory
// [blockDim.x][MG_NXPARAM] (zeros when the fleet has none).
template <int MT, bool GEN>
__global__ void __launch_bounds__(256)
    k_split(const FleetView fv, const BlockDesc *__restrict__ blocks,
            const float *__restrict__ raw, float *__restrict__ accel, const int32_t k) {
  __shared__ float4 sdir[MG_MAX_THR], sarm[MG_MAX_THR];
  __shared__ unsigned s_done;
  __shared__ int64_t s_cursor;
  extern __shared__ float sxh[];
  const BlockDesc bd = blocks[blockIdx.x];
  if (threadIdx.x < MG_MAX_THR) {
    sdir[threadIdx.x] = fv.geo[bd.type].dir[threadIdx.x];
    sarm[threadIdx.x] = fv.geo[bd.type].arm[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    s_done = 0u;
    s_cursor = launch_cursor(fv);
  }
  if constexpr (GEN) {
    if (fv.xh)
      stage_xh(fv.xh, fv.n, bd.env0, bd.count, sxh);
    else
      for (int t = threadIdx.x; t < bd.count * MG_NXPARAM; t += blockDim.x) sxh[t] = 0.f;
  }
  __syncthreads();
  if ((int)threadIdx.x >= bd.count) return;
  const int64_t e = (int64_t)bd.env0 + threadIdx.x;
  const int nt = bd.n_thr;
  const bool current_accel = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);

  St<MT> s;
  load_state<MT, false>(fv.st, e, s);
  SplitPar P;
  load_split_par(raw, e, P);
  float a[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) a[i] = accel[i * fv.n + e];

  const int64_t step0 = s_cursor + fv.cursor_off;
  int64_t seg = step0 / fv.hold;
  int32_t left = fv.hold - (int32_t)(step0 - seg * fv.hold);
  float c[MT];
  load_commands<MT>(fv, e, seg, nt, P.itau, c);
  for (int32_t it = 0; it < k; ++it) {
    if (left == 0) {
      ++seg;
      left = fv.hold;
      load_commands<MT>(fv, e, seg, nt, P.itau, c);
    }
    split_substep<MT, GEN>(s, a, c, P, sdir, sarm, nt, current_accel, fv.dt,
                           GEN ? sxh + threadIdx.x * MG_NXPARAM : nullptr);
    --left;
  }
  store_and_flag<MT, false>(fv, e, s);
#pragma unroll
  for (int i = 0; i < 6; ++i) accel[i * fv.n + e] = a[i];
  if (fv.cursor_adv) finish_envs(fv, &s_done, bd.count, fv.cursor_adv);
}

}  // namespace

cudaError_t launch_split(const FleetView &fv, const BlockDesc *blocks, int n_blocks, int threads,
                         NtVariant ntv, bool general, const float *raw, float *accel, int32_t k,
                         cudaStream_t stream) {
  if (threads < 32 || threads > 256 || threads % 32 || n_blocks < 1 || k < 1 ||
      (fv.xh && !general))
    return cudaErrorInvalidValue;
  const size_t xh_bytes = general ? sizeof(float) * threads * MG_NXPARAM : 0;  // <= 46,080 B
  if (ntv == NT_6 && general)
    k_split<6, true><<<n_blocks, threads, xh_bytes, stream>>>(fv, blocks, raw, accel, k);
  else if (ntv == NT_6)
    k_split<6, false><<<n_blocks, threads, 0, stream>>>(fv, blocks, raw, accel, k);
  else if (general)
    k_split<8, true><<<n_blocks, threads, xh_bytes, stream>>>(fv, blocks, raw, accel, k);
  else
    k_split<8, false><<<n_blocks, threads, 0, stream>>>(fv, blocks, raw, accel, k);
  return cudaGetLastError();
}

}  // namespace mg
