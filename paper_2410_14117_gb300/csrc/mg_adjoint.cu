// Discrete adjoint of the FP32 rollout: gradients of a loss on the recorded trajectory with
// respect to each env's hydrodynamic coefficients (added mass, linear and quadratic damping
// diagonals of Eq. 1) and to the buffered throttle actions (Eq. 3).
//
// The forward pass (k_fleet with recording) writes the state after every sub-step; the
// checkpoint kernel below saves the full state every C sub-steps.  The backward kernel runs one
// thread per env: for each checkpoint segment, last first, it re-runs the segment's sub-steps
// from the checkpoint (keeping the C step-start states in local memory), then walks them in
// reverse, applying the transpose Jacobian of one sub-step
//     s+ = N(s + h/6 (k1 + 2 k2 + 2 k3 + k4)),  N = quaternion renormalisation,
// through N, the RK4 combination and the four right-hand-side evaluations (reverse mode of
// rhs(), written out below).  It is the adjoint of the discrete map the forward computes, so it
// matches finite differences of the rollout itself, not of the continuous equations.
//
// Two parameter paths, as the forward has:
//   - diagonal mass (r_g = 0, no off-diagonal extension): M^-1 = diag(1 / M_jj);
//   - general (GEN): off-centre gravity (the m r_g coupling of M_RB and C_RB, off-diagonal
//     I_o) and the off-diagonal added mass and linear damping of the extension record (zeros
//     when the fleet has none), with the full M^-1.  A diagonal coefficient theta = M_A,jj enters
//     M = M_RB + M_A, so nu' = M^-1 f gets d nu'/d theta = -M^-1 e_j nu'_j, whose contribution to
//     the gradient is -(M^-1 g)_j nu'_j for the loss adjoint g of nu' (M^-1 is symmetric).
#include <type_traits>

#include "mg_advance.cuh"

namespace mg {

namespace {

constexpr int kAdjThreads = 128;

struct Grad {
  float ma[3], J[3], mv[6], dl[6], dq[6];  // mv: the M_A,jj gradient through M^-1
};

// What the adjoint reads for one env: the loaded parameters (transposes), the coefficients the
// forward step used (re-running it bit for bit) and, on the general path, the env's off-diagonal
// hydrodynamic coefficients (a row of MG_NXPARAM floats in shared memory).
template <bool GEN>
struct AdjEnv {
  Par<!GEN> P;
  Coef<!GEN> F;
  const float *xh;
};

// Off-diagonal entries of the extension record (layout of mg.h): M_A above its diagonal
// (01 02 03 04 05 12 13 14 15 23 24 25 34 35 45, mirrored below), then D_l's off-diagonal
// entries row by row (5 per row).
__device__ __forceinline__ float xa(const float *xh, int i, int j) {
  const int a = i < j ? i : j, b = i < j ? j : i;
  return xh[5 * a - a * (a - 1) / 2 + (b - a - 1)];
}
__device__ __forceinline__ float xd(const float *xh, int i, int j) {
  return xh[15 + 5 * i + (j < i ? j : j - 1)];
}

// Every multiply-add of the adjoint code below is written as an explicit fmaf, so the compiler
// forms no fused operation of its own: the results do not depend on the surrounding code the
// functions are inlined into (the one-warp and two-warp backward kernels agree bit for bit).

__device__ __forceinline__ void cross_vjp(const float a[3], const float b[3], const float gc[3],
                                          float ga[3], float gb[3]) {
  // c = a x b:  ga += b x gc,  gb += gc x a.
  ga[0] = fmaf(b[1], gc[2], fmaf(-b[2], gc[1], ga[0]));
  ga[1] = fmaf(b[2], gc[0], fmaf(-b[0], gc[2], ga[1]));
  ga[2] = fmaf(b[0], gc[1], fmaf(-b[1], gc[0], ga[2]));
  gb[0] = fmaf(gc[1], a[2], fmaf(-gc[2], a[1], gb[0]));
  gb[1] = fmaf(gc[2], a[0], fmaf(-gc[0], a[2], gb[1]));
  gb[2] = fmaf(gc[0], a[1], fmaf(-gc[1], a[0], gb[2]));
}

// Packed symmetric M^-1 (general path) times x.
__device__ __forceinline__ void minv_apply(const ParGen &P, const float x[6], float y[6]) {
  const float *o = P.mo;  // 01 02 03 04 05 12 13 14 15 23 24 25 34 35 45
  y[0] = fmaf(P.mi[0], x[0], fmaf(o[0], x[1], fmaf(o[1], x[2], fmaf(o[2], x[3],
         fmaf(o[3], x[4], o[4] * x[5])))));
  y[1] = fmaf(o[0], x[0], fmaf(P.mi[1], x[1], fmaf(o[5], x[2], fmaf(o[6], x[3],
         fmaf(o[7], x[4], o[8] * x[5])))));
  y[2] = fmaf(o[1], x[0], fmaf(o[5], x[1], fmaf(P.mi[2], x[2], fmaf(o[9], x[3],
         fmaf(o[10], x[4], o[11] * x[5])))));
  y[3] = fmaf(o[2], x[0], fmaf(o[6], x[1], fmaf(o[9], x[2], fmaf(P.mi[3], x[3],
         fmaf(o[12], x[4], o[13] * x[5])))));
  y[4] = fmaf(o[3], x[0], fmaf(o[7], x[1], fmaf(o[10], x[2], fmaf(o[12], x[3],
         fmaf(P.mi[4], x[4], o[14] * x[5])))));
  y[5] = fmaf(o[4], x[0], fmaf(o[8], x[1], fmaf(o[11], x[2], fmaf(o[13], x[3],
         fmaf(o[14], x[4], P.mi[5] * x[5])))));
}

// gs += (d rhs / d s)^T gd; parameter and command adjoints accumulated into G and gcs.  The
// forward quantities are recomputed from Eq. 1 in the general path's Kirchhoff form (the
// diagonal-mass path drops the terms that vanish with r_g = 0 and diagonal M_A, D_l); gd.q is
// the adjoint of d.q = q (x) (0, w) (the doubled quaternion rate rhs() stores).
template <int MT, bool GEN>
__device__ void rhs_vjp(const St<MT> &s, const float (&cs)[MT], const AdjEnv<GEN> &A,
                        const float4 *gdir, const float4 *garm, int nt, bool current_accel,
                        const St<MT> &gd, St<MT> &gs, Grad &G, float (&gcs)[MT]) {
  const auto &P = A.P;
  const float *xh = A.xh;
  // ---------------- forward recomputation
  float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    if (i >= nt) continue;  // compile-time indices keep the arrays in registers
    const float f = s.n[i] * fabsf(s.n[i]);
    const float4 dd = gdir[i], aa = garm[i];
    t[0] = fmaf(f, dd.x, t[0]); t[1] = fmaf(f, dd.y, t[1]); t[2] = fmaf(f, dd.z, t[2]);
    t[3] = fmaf(f, aa.x, t[3]); t[4] = fmaf(f, aa.y, t[4]); t[5] = fmaf(f, aa.z, t[5]);
  }
  const float qw = s.q[0], qx = s.q[1], qy = s.q[2], qz = s.q[3];
  float R[3][3];
  R[0][0] = fmaf(-2.f, fmaf(qy, qy, qz * qz), 1.f);
  R[0][1] = 2.f * fmaf(qx, qy, -qw * qz);
  R[0][2] = 2.f * fmaf(qx, qz, qw * qy);
  R[1][0] = 2.f * fmaf(qx, qy, qw * qz);
  R[1][1] = fmaf(-2.f, fmaf(qx, qx, qz * qz), 1.f);
  R[1][2] = 2.f * fmaf(qy, qz, -qw * qx);
  R[2][0] = 2.f * fmaf(qx, qz, -qw * qy);
  R[2][1] = 2.f * fmaf(qy, qz, qw * qx);
  R[2][2] = fmaf(-2.f, fmaf(qx, qx, qy * qy), 1.f);
  const float v[3] = {s.v[0], s.v[1], s.v[2]}, w[3] = {s.w[0], s.w[1], s.w[2]};
  const float vc[3] = {P.vc0, P.vc1, P.vc2}, ma[3] = {P.ma0, P.ma1, P.ma2};
  const float J[3] = {P.J0, P.J1, P.J2}, G3[3] = {P.G0, P.G1, P.G2};
  float cb[3], r[3], qm[3], h[3], k[3], c[3] = {0.f, 0.f, 0.f}, am[3] = {0.f, 0.f, 0.f};
  float mrg[3] = {0.f, 0.f, 0.f};
  if constexpr (GEN) {
    mrg[0] = P.mrg0; mrg[1] = P.mrg1; mrg[2] = P.mrg2;
  }
  for (int i = 0; i < 3; ++i)
    cb[i] = fmaf(R[2][i], vc[2], fmaf(R[1][i], vc[1], R[0][i] * vc[0]));
  for (int i = 0; i < 3; ++i) {
    r[i] = v[i] - cb[i];
    qm[i] = ma[i] * r[i];
    k[i] = J[i] * w[i];
  }
  const float nur[6] = {r[0], r[1], r[2], w[0], w[1], w[2]};
  if constexpr (GEN) {
    // off-diagonal added mass in the momenta; w x m r_g; off-diagonal I_o w + m r_g x v
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j != i) qm[i] = fmaf(xa(xh, i, j), nur[j], qm[i]);
        if (j != 3 + i) k[i] = fmaf(xa(xh, 3 + i, j), nur[j], k[i]);
      }
    am[0] = fmaf(w[1], mrg[2], -w[2] * mrg[1]);
    am[1] = fmaf(w[2], mrg[0], -w[0] * mrg[2]);
    am[2] = fmaf(w[0], mrg[1], -w[1] * mrg[0]);
    k[0] = fmaf(P.Ixy, w[1], fmaf(P.Ixz, w[2], fmaf(mrg[1], v[2], fmaf(-mrg[2], v[1], k[0]))));
    k[1] = fmaf(P.Ixy, w[0], fmaf(P.Iyz, w[2], fmaf(mrg[2], v[0], fmaf(-mrg[0], v[2], k[1]))));
    k[2] = fmaf(P.Ixz, w[0], fmaf(P.Iyz, w[1], fmaf(mrg[0], v[1], fmaf(-mrg[1], v[0], k[2]))));
  }
  for (int i = 0; i < 3; ++i) h[i] = fmaf(P.m, v[i], qm[i]) + am[i];
  if (current_accel) {
    c[0] = fmaf(w[1], cb[2], -w[2] * cb[1]);
    c[1] = fmaf(w[2], cb[0], -w[0] * cb[2]);
    c[2] = fmaf(w[0], cb[1], -w[1] * cb[0]);
  }
  const float e[3] = {R[2][0], R[2][1], R[2][2]};
  // translational: kT t + (W - B) e - w x h - (Dl + Dq |r|) r [- M_A [w x v_c^b; 0]]
  //                [- off-diagonal D_l nu_r]
  float f[6];
  for (int i = 0; i < 3; ++i) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
    float x = fmaf(P.kT, t[i], P.wb * e[i]);
    x = fmaf(-w[i1], h[i2], fmaf(w[i2], h[i1], x));
    x = fmaf(-fmaf(P.dq[i], fabsf(r[i]), P.dl[i]), r[i], x);
    f[i] = fmaf(-ma[i], c[i], x);
  }
  // rotational: kT t' - r x Q1 - w x k [- v x (w x m r_g)] - (Dl + Dq |w|) w + G x e
  //             [- M_A [w x v_c^b; 0]] [- off-diagonal D_l nu_r]
  for (int i = 0; i < 3; ++i) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
    float x = fmaf(P.kT, t[3 + i], fmaf(-r[i1], qm[i2], r[i2] * qm[i1]));
    x = fmaf(-w[i1], k[i2], fmaf(w[i2], k[i1], x));
    if constexpr (GEN) x = fmaf(-v[i1], am[i2], fmaf(v[i2], am[i1], x));
    x = fmaf(-fmaf(P.dq[3 + i], fabsf(w[i]), P.dl[3 + i]), w[i], x);
    f[3 + i] = fmaf(G3[i1], e[i2], fmaf(-G3[i2], e[i1], x));
  }
  if constexpr (GEN) {
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j < 3 && j != i) f[i] = fmaf(-xa(xh, i, j), c[j], f[i]);
        if (j != i) f[i] = fmaf(-xd(xh, i, j), nur[j], f[i]);
      }
  }
  float nud[6];  // nu' = M^-1 f
  if constexpr (GEN) minv_apply(P, f, nud);
  else
    for (int j = 0; j < 6; ++j) nud[j] = P.mi[j] * f[j];

  // ---------------- reverse
  // lag: d.n_i = cs_i - n_i / tau_m
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    if (i >= nt) continue;
    gcs[i] += gd.n[i];
    gs.n[i] = fmaf(-P.itau, gd.n[i], gs.n[i]);
  }
  // nu' = M^-1 f: gf = M^-1 g (symmetric), and M_jj's share -gf_j nu'_j
  const float gnu[6] = {gd.v[0], gd.v[1], gd.v[2], gd.w[0], gd.w[1], gd.w[2]};
  float gf[6], gt[6];
  if constexpr (GEN) minv_apply(P, gnu, gf);
  else
    for (int j = 0; j < 6; ++j) gf[j] = P.mi[j] * gnu[j];
  for (int j = 0; j < 6; ++j) {
    G.mv[j] = fmaf(-gf[j], nud[j], G.mv[j]);
    gt[j] = P.kT * gf[j];
  }
  float gw[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f}, gr[3] = {0.f, 0.f, 0.f};
  float gh[3] = {0.f, 0.f, 0.f}, gk[3] = {0.f, 0.f, 0.f}, gqm[3] = {0.f, 0.f, 0.f};
  float gcb[3] = {0.f, 0.f, 0.f}, ge[3] = {0.f, 0.f, 0.f}, gc[3] = {0.f, 0.f, 0.f};
  float gam[3] = {0.f, 0.f, 0.f}, gnur[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if constexpr (GEN) {
    // off-diagonal current term and linear damping
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j < 3 && j != i) gc[j] = fmaf(-xa(xh, i, j), gf[i], gc[j]);
        if (j != i) gnur[j] = fmaf(-xd(xh, i, j), gf[i], gnur[j]);
      }
  }
  // rotational force
  const float gfr[3] = {gf[3], gf[4], gf[5]};
  const float ngfr[3] = {-gf[3], -gf[4], -gf[5]};
  cross_vjp(r, qm, ngfr, gr, gqm);   // - r x Q1
  cross_vjp(w, k, ngfr, gw, gk);     // - w x k
  if constexpr (GEN) cross_vjp(v, am, ngfr, gv, gam);  // - v x (w x m r_g)
  for (int j = 0; j < 3; ++j) {
    const float aw = fabsf(w[j]);
    gw[j] = fmaf(-fmaf(2.f * P.dq[3 + j], aw, P.dl[3 + j]), gfr[j], gw[j]);
    G.dl[3 + j] = fmaf(-w[j], gfr[j], G.dl[3 + j]);
    G.dq[3 + j] = fmaf(-aw * w[j], gfr[j], G.dq[3 + j]);
  }
  {
    float gG[3] = {0.f, 0.f, 0.f};
    cross_vjp(G3, e, gfr, gG, ge);   // + G x e
  }
  // translational force
  const float gfl[3] = {gf[0], gf[1], gf[2]};
  const float ngfl[3] = {-gf[0], -gf[1], -gf[2]};
  for (int j = 0; j < 3; ++j) ge[j] = fmaf(P.wb, gfl[j], ge[j]);
  cross_vjp(w, h, ngfl, gw, gh);     // - w x h
  for (int j = 0; j < 3; ++j) {
    const float ar = fabsf(r[j]);
    gr[j] = fmaf(-fmaf(2.f * P.dq[j], ar, P.dl[j]), gfl[j], gr[j]);
    G.dl[j] = fmaf(-r[j], gfl[j], G.dl[j]);
    G.dq[j] = fmaf(-ar * r[j], gfl[j], G.dq[j]);
  }
  if (current_accel) {
    for (int j = 0; j < 3; ++j) {
      G.ma[j] = fmaf(-c[j], gfl[j], G.ma[j]);
      gc[j] = fmaf(-ma[j], gfl[j], gc[j]);
    }
    cross_vjp(w, cb, gc, gw, gcb);   // c = w x v_c^b
  }
  if constexpr (GEN) {
    // k += off-diagonal I_o w + m r_g x v;  h += w x m r_g
    gw[0] = fmaf(P.Ixy, gk[1], fmaf(P.Ixz, gk[2], gw[0]));
    gw[1] = fmaf(P.Ixy, gk[0], fmaf(P.Iyz, gk[2], gw[1]));
    gw[2] = fmaf(P.Ixz, gk[0], fmaf(P.Iyz, gk[1], gw[2]));
    gv[0] = fmaf(gk[1], mrg[2], fmaf(-gk[2], mrg[1], gv[0]));
    gv[1] = fmaf(gk[2], mrg[0], fmaf(-gk[0], mrg[2], gv[1]));
    gv[2] = fmaf(gk[0], mrg[1], fmaf(-gk[1], mrg[0], gv[2]));
    for (int j = 0; j < 3; ++j) gam[j] += gh[j];
    float gmrg[3] = {0.f, 0.f, 0.f};
    cross_vjp(w, mrg, gam, gw, gmrg);
    // off-diagonal added mass in the momenta (Q1 enters through h and through r x Q1)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j != i) gnur[j] = fmaf(xa(xh, i, j), gqm[i] + gh[i], gnur[j]);
        if (j != 3 + i) gnur[j] = fmaf(xa(xh, 3 + i, j), gk[i], gnur[j]);
      }
  }
  // k = J w, h = m v + Q1, Q1 = M_A r, r = v - v_c^b
  for (int j = 0; j < 3; ++j) {
    gw[j] = fmaf(J[j], gk[j], gw[j]);
    G.J[j] = fmaf(w[j], gk[j], G.J[j]);
    gv[j] = fmaf(P.m, gh[j], gv[j]);
    gqm[j] += gh[j];
    gr[j] = fmaf(ma[j], gqm[j], gr[j]);
    G.ma[j] = fmaf(r[j], gqm[j], G.ma[j]);
    gr[j] += gnur[j];
    gw[j] += gnur[3 + j];
    gv[j] += gr[j];
    gcb[j] -= gr[j];
  }
  // R entries: v_c^b = R^T v_c, e = third row of R, p' = R v
  float gR[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) gR[i][j] = fmaf(vc[i], gcb[j], gd.p[i] * v[j]);
  for (int j = 0; j < 3; ++j) {
    gR[2][j] += ge[j];
    gv[j] = fmaf(R[0][j], gd.p[0], fmaf(R[1][j], gd.p[1], fmaf(R[2][j], gd.p[2], gv[j])));
  }
  // d.q = q (x) (0, w)
  const float g0 = gd.q[0], g1 = gd.q[1], g2 = gd.q[2], g3 = gd.q[3];
  gw[0] = fmaf(-qx, g0, fmaf(qw, g1, fmaf(qz, g2, fmaf(-qy, g3, gw[0]))));
  gw[1] = fmaf(-qy, g0, fmaf(-qz, g1, fmaf(qw, g2, fmaf(qx, g3, gw[1]))));
  gw[2] = fmaf(-qz, g0, fmaf(qy, g1, fmaf(-qx, g2, fmaf(qw, g3, gw[2]))));
  float gq[4];
  gq[0] = fmaf(w[0], g1, fmaf(w[1], g2, w[2] * g3));
  gq[1] = fmaf(-w[0], g0, fmaf(-w[2], g2, w[1] * g3));
  gq[2] = fmaf(-w[1], g0, fmaf(w[2], g1, -w[0] * g3));
  gq[3] = fmaf(-w[2], g0, fmaf(-w[1], g1, w[0] * g2));
  // R(q) -> q
  {
    const float s0 = fmaf(-qz, gR[0][1], fmaf(qz, gR[1][0], fmaf(qy, gR[0][2],
                     fmaf(-qy, gR[2][0], fmaf(-qx, gR[1][2], qx * gR[2][1])))));
    const float s1 = fmaf(qy, gR[0][1], fmaf(qy, gR[1][0], fmaf(qz, gR[0][2],
                     fmaf(qz, gR[2][0], fmaf(-qw, gR[1][2], qw * gR[2][1])))));
    const float s2 = fmaf(qx, gR[0][1], fmaf(qx, gR[1][0], fmaf(qw, gR[0][2],
                     fmaf(-qw, gR[2][0], fmaf(qz, gR[1][2], qz * gR[2][1])))));
    const float s3 = fmaf(-qw, gR[0][1], fmaf(qw, gR[1][0], fmaf(qx, gR[0][2],
                     fmaf(qx, gR[2][0], fmaf(qy, gR[1][2], qy * gR[2][1])))));
    gq[0] = fmaf(2.f, s0, gq[0]);
    gq[1] = fmaf(2.f, s1, fmaf(-4.f * qx, gR[1][1] + gR[2][2], gq[1]));
    gq[2] = fmaf(2.f, s2, fmaf(-4.f * qy, gR[0][0] + gR[2][2], gq[2]));
    gq[3] = fmaf(2.f, s3, fmaf(-4.f * qz, gR[0][0] + gR[1][1], gq[3]));
  }
  // thrust: t = sum_i n_i|n_i| b_i
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    if (i >= nt) continue;
    const float4 dd = gdir[i], aa = garm[i];
    const float gfi = fmaf(dd.x, gt[0], fmaf(dd.y, gt[1], fmaf(dd.z, gt[2],
                      fmaf(aa.x, gt[3], fmaf(aa.y, gt[4], aa.z * gt[5])))));
    gs.n[i] = fmaf(2.f * fabsf(s.n[i]), gfi, gs.n[i]);
  }
  for (int i = 0; i < 4; ++i) gs.q[i] += gq[i];
  for (int i = 0; i < 3; ++i) {
    gs.v[i] += gv[i];
    gs.w[i] += gw[i];
  }
}

// y = x + a W k with W the rk4 weighting (the quaternion takes half of each weight because
// rhs() stores its rate doubled):  out = a W x  or  out += a W x.
template <int MT>
__device__ __forceinline__ void wscale(St<MT> &out, const St<MT> &x, float a, bool add) {
  const float aq = 0.5f * a;
  for (int i = 0; i < 3; ++i) out.p[i] = add ? fmaf(a, x.p[i], out.p[i]) : a * x.p[i];
  for (int i = 0; i < 4; ++i) out.q[i] = add ? fmaf(aq, x.q[i], out.q[i]) : aq * x.q[i];
  for (int i = 0; i < 3; ++i) out.v[i] = add ? fmaf(a, x.v[i], out.v[i]) : a * x.v[i];
  for (int i = 0; i < 3; ++i) out.w[i] = add ? fmaf(a, x.w[i], out.w[i]) : a * x.w[i];
  for (int i = 0; i < MT; ++i) out.n[i] = add ? fmaf(a, x.n[i], out.n[i]) : a * x.n[i];
}

template <int MT>
__device__ __forceinline__ void st_zero(St<MT> &x) {
  for (int i = 0; i < 3; ++i) x.p[i] = x.v[i] = x.w[i] = 0.f;
  for (int i = 0; i < 4; ++i) x.q[i] = 0.f;
  for (int i = 0; i < MT; ++i) x.n[i] = 0.f;
}

// The forward's right-hand side and closed-form-lag sub-step for this env (the step kernels'
// own code: the diagonal-mass coefficients, or the general path with the staged off-diagonal
// coefficients).
template <int MT, bool GEN>
__device__ __forceinline__ void fwd_rhs(const St<MT> &y, const float (&cs)[MT],
                                        const AdjEnv<GEN> &A, const float4 *gdir,
                                        const float4 *garm, int nt, bool ca, St<MT> &k) {
  rhs<MT, !GEN, true, 0, GEN>(y, cs, A.F, gdir, garm, nt, ca, k, A.xh);
}

template <int MT, bool GEN>
__device__ __forceinline__ void fwd_step(St<MT> &S, const float (&b)[MT], const LagEnv &L,
                                         const AdjEnv<GEN> &A, const float4 *gdir,
                                         const float4 *garm, int nt, bool ca, float h) {
  rk4_step_lag<MT, !GEN, true, 0, GEN>(S, b, L, A.F, gdir, garm, nt, ca, h, A.xh);
}

// The RK4 stage states of one sub-step from its start state s (y1 = s):
//   y2 = s + h/2 W k1,  y3 = s + h/2 W k2,  y4 = s + h W k3,  k_i = rhs(y_i),
//   z  = s + h/6 W k1 + h/3 W k2 + h/3 W k3 + h/6 W k4  (before renormalisation).
template <int MT, bool GEN>
__device__ __forceinline__ void stage_states(const St<MT> &s, const float (&cs)[MT],
                                             const AdjEnv<GEN> &A, const float4 *gdir,
                                             const float4 *garm, int nt, bool current_accel,
                                             float h, St<MT> &y2, St<MT> &y3, St<MT> &y4,
                                             St<MT> &z) {
  const float hh = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
  St<MT> k;
  fwd_rhs<MT, GEN>(s, cs, A, gdir, garm, nt, current_accel, k);
  axpy(z, s, h6, k);
  axpy(y2, s, hh, k);
  fwd_rhs<MT, GEN>(y2, cs, A, gdir, garm, nt, current_accel, k);
  axpy(z, z, h3, k);
  axpy(y3, s, hh, k);
  fwd_rhs<MT, GEN>(y3, cs, A, gdir, garm, nt, current_accel, k);
  axpy(z, z, h3, k);
  axpy(y4, s, h, k);
  fwd_rhs<MT, GEN>(y4, cs, A, gdir, garm, nt, current_accel, k);
  axpy(z, z, h6, k);
}

template <int MT>
__device__ __forceinline__ void st_add(St<MT> &y, const St<MT> &x) {
  for (int i = 0; i < 3; ++i) y.p[i] += x.p[i];
  for (int i = 0; i < 4; ++i) y.q[i] += x.q[i];
  for (int i = 0; i < 3; ++i) y.v[i] += x.v[i];
  for (int i = 0; i < 3; ++i) y.w[i] += x.w[i];
  for (int i = 0; i < MT; ++i) y.n[i] += x.n[i];
}

// lam: in, the adjoint of the sub-step's output s+; out, the adjoint of its input s.
// stage(i, y) gives stage i's state (0: s, 1: y2, 2: y3, 3: y4; stage_states) and zq is the
// quaternion before renormalisation.
//   s+ = N(z)
// reverse:  lk4 = h/6 W lz,            ly4 = J(y4)^T lk4
//           lk3 = h/3 W lz + h W ly4,   ly3 = J(y3)^T lk3
//           lk2 = h/3 W lz + h/2 W ly3, ly2 = J(y2)^T lk2
//           lk1 = h/6 W lz + h/2 W ly2, ly1 = J(s)^T lk1
//           ls  = lz + ly4 + ly3 + ly2 + ly1
// The four stages share one loop body, kept a loop (UNROLL false) with a single copy of rhs_vjp:
// a quarter of the code, which the instruction cache holds (unrolled, both backward kernels
// stalled mostly on instruction fetch: 1.41 / 1.29 ms against 1.11 / 1.04 ms rolled at 4,096
// envs).  The stage states are then selected or read by a runtime index.  Same operations
// either way.
template <int MT, bool GEN, bool UNROLL, typename Stage>
__device__ __forceinline__ void step_vjp_stages(Stage stage, const float (&zq)[4],
                                                const float (&cs)[MT], const AdjEnv<GEN> &A,
                                                const float4 *gdir, const float4 *garm, int nt,
                                                bool current_accel, float h, St<MT> &lam,
                                                Grad &G, float (&gcs)[MT]) {
  const float hh = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
  // renormalisation q+ = z_q / |z_q|:  lz_q = (lam_q - q+ (q+ . lam_q)) / |z_q|
  const float nq = sqrtf(fmaf(zq[0], zq[0], fmaf(zq[1], zq[1], fmaf(zq[2], zq[2], zq[3] * zq[3]))));
  float qn[4], dot = 0.f;
  for (int i = 0; i < 4; ++i) {
    qn[i] = zq[i] / nq;
    dot = fmaf(qn[i], lam.q[i], dot);
  }
  St<MT> lz = lam;
  for (int i = 0; i < 4; ++i) lz.q[i] = fmaf(-qn[i], dot, lam.q[i]) / nq;

  St<MT> lk, ly;
  St<MT> &ls = lam;
  ls = lz;
  st_zero(ly);
  auto body = [&](int i) {
    wscale(lk, lz, (i == 3 || i == 0) ? h6 : h3, false);
    if (i < 3) wscale(lk, ly, (i == 2) ? h : hh, true);
    St<MT> y;
    stage(i, y);
    st_zero(ly);
    rhs_vjp<MT, GEN>(y, cs, A, gdir, garm, nt, current_accel, lk, ly, G, gcs);
    st_add(ls, ly);
  };
  if constexpr (UNROLL) {
#pragma unroll
    for (int i = 3; i >= 0; --i) body(i);
  } else {
#pragma unroll 1
    for (int i = 3; i >= 0; --i) body(i);
  }
}

// The whole sub-step: stage states recomputed, then their transposes.
template <int MT, bool GEN>
__device__ void step_vjp(const St<MT> &s, const float (&cs)[MT], const AdjEnv<GEN> &A,
                         const float4 *gdir, const float4 *garm, int nt, bool current_accel,
                         float h, St<MT> &lam, Grad &G, float (&gcs)[MT]) {
  St<MT> y2, y3, y4, z;
  stage_states<MT, GEN>(s, cs, A, gdir, garm, nt, current_accel, h, y2, y3, y4, z);
  const float zq[4] = {z.q[0], z.q[1], z.q[2], z.q[3]};
  auto stage = [&](int i, St<MT> &y) { y = i == 0 ? s : i == 1 ? y2 : i == 2 ? y3 : y4; };
  step_vjp_stages<MT, GEN, false>(stage, zq, cs, A, gdir, garm, nt, current_accel, h, lam, G,
                                  gcs);
}

constexpr int kMaxSeg = 32;  // largest checkpoint interval

// The buffered command of sub-step j (cursor position), pre-divided by tau_m as the step reads it.
template <int MT>
__device__ __forceinline__ void commands_at(const FleetView &fv, int64_t e, int64_t j, int nt,
                                            float itau, float (&c)[MT]) {
  int64_t seg = j / fv.hold;
  if (seg > fv.n_seg - 1) seg = fv.n_seg - 1;
  for (int i = 0; i < MT; ++i) c[i] = 0.f;
  if (fv.n_seg > 0) {
    const float *a = fv.act + (seg * fv.n + e) * fv.act_w;
    #pragma unroll
    for (int i = 0; i < MT; ++i)
      if (i < nt) c[i] = a[i] * itau;
  }
}

__global__ void k_checkpoint(const StatePlanes st, int64_t n, float *__restrict__ ck) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float4 a = st.s0[e], b = st.s1[e], c = st.s2[e], d = st.s3[e], f = st.s4[e];
  const float r[MG_NSTATE] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z,
                              c.w, d.x, d.y, d.z, d.w, f.x, f.y, f.z, f.w, st.s5[e]};
  for (int j = 0; j < MG_NSTATE; ++j) ck[(int64_t)j * n + e] = r[j];
}

template <int MT>
__device__ __forceinline__ void load_checkpoint(const float *__restrict__ ckpt, int32_t sg,
                                                int64_t n, int64_t e, St<MT> &S) {
  const float *ck = ckpt + (int64_t)sg * MG_NSTATE * n + e;
  for (int i = 0; i < 3; ++i) S.p[i] = ck[(int64_t)(i)*n];
  for (int i = 0; i < 4; ++i) S.q[i] = ck[(int64_t)(3 + i) * n];
  for (int i = 0; i < 3; ++i) S.v[i] = ck[(int64_t)(7 + i) * n];
  for (int i = 0; i < 3; ++i) S.w[i] = ck[(int64_t)(10 + i) * n];
  for (int i = 0; i < MT; ++i) S.n[i] = ck[(int64_t)(13 + i) * n];
}

// lam += the loss adjoint of the state after sub-step t.
template <int MT>
__device__ __forceinline__ void add_traj_adjoint(const float *__restrict__ dtraj, int64_t t,
                                                 int64_t n, int64_t e, St<MT> &lam) {
  const float *g = dtraj + t * MG_NTRAJ * n + e;
  for (int i = 0; i < 3; ++i) lam.p[i] += g[(int64_t)i * n];
  for (int i = 0; i < 4; ++i) lam.q[i] += g[(int64_t)(3 + i) * n];
  for (int i = 0; i < 3; ++i) lam.v[i] += g[(int64_t)(7 + i) * n];
  for (int i = 0; i < 3; ++i) lam.w[i] += g[(int64_t)(10 + i) * n];
}

// Command adjoint of sub-step t into its action segment.
template <int MT>
__device__ __forceinline__ void add_action_adjoint(const FleetView &fv, int64_t t, int64_t e,
                                                   int nt, float itau, const float (&gcs)[MT],
                                                   float *__restrict__ dact) {
  if (!dact || fv.n_seg <= 0) return;
  int64_t seg = t / fv.hold;
  if (seg > fv.n_seg - 1) seg = fv.n_seg - 1;
  float *da = dact + (seg * fv.n + e) * fv.act_w;
  #pragma unroll
  for (int i = 0; i < MT; ++i)
    if (i < nt) da[i] = fmaf(itau, gcs[i], da[i]);
}

// Coefficients: M_A,jj enters the momenta (Q1 for j < 3, J = diag(I_o) + M_A,rot for j >= 3),
// the current term and M (G.mv); D_l and D_q their damping terms.
template <int MT>
__device__ __forceinline__ void write_gradients(const Grad &G, const St<MT> &lam, int64_t e,
                                                float *__restrict__ dcoef,
                                                float *__restrict__ dstate0) {
  float *dc = dcoef + e * 18;
  for (int j = 0; j < 3; ++j) {
    dc[j] = G.ma[j] + G.mv[j];
    dc[3 + j] = G.J[j] + G.mv[3 + j];
  }
  for (int j = 0; j < 6; ++j) {
    dc[6 + j] = G.dl[j];
    dc[12 + j] = G.dq[j];
  }
  if (dstate0) {
    float *o = dstate0 + e * MG_NSTATE;
    for (int i = 0; i < 3; ++i) o[i] = lam.p[i];
    for (int i = 0; i < 4; ++i) o[3 + i] = lam.q[i];
    for (int i = 0; i < 3; ++i) o[7 + i] = lam.v[i];
    for (int i = 0; i < 3; ++i) o[10 + i] = lam.w[i];
    for (int i = 0; i < MG_MAX_THR; ++i) o[13 + i] = i < MT ? lam.n[i] : 0.f;
  }
}

__device__ __forceinline__ void zero_grad(Grad &G) {
  for (int i = 0; i < 3; ++i) G.ma[i] = G.J[i] = 0.f;
  for (int i = 0; i < 6; ++i) G.mv[i] = G.dl[i] = G.dq[i] = 0.f;
}

__device__ __forceinline__ void stage_geometry(const FleetView &fv,
                                               float4 (*sgeo)[2 * MG_MAX_THR]) {
  for (int i = threadIdx.x; i < fv.n_types * 2 * MG_MAX_THR; i += blockDim.x) {
    const int t = i / (2 * MG_MAX_THR), j = i % (2 * MG_MAX_THR);
    sgeo[t][j] = j < MG_MAX_THR ? fv.geo[t].dir[j] : fv.geo[t].arm[j - MG_MAX_THR];
  }
}

// General path: rows [0, count) of sx receive the off-diagonal coefficients of envs env0, ...,
// or zeros when the fleet has no extension (off-centre gravity only).
__device__ __forceinline__ void stage_xh_or_zero(const FleetView &fv, int64_t env0, int count,
                                                 float *sx) {
  if (fv.xh) {
    stage_xh(fv.xh, fv.n, env0, count, sx);
  } else {
    for (int i = threadIdx.x; i < count * MG_NXPARAM; i += blockDim.x) sx[i] = 0.f;
  }
}

template <bool GEN>
__device__ __forceinline__ void load_env(const FleetView &fv, int64_t e, bool ca,
                                         const float *sxh_row, AdjEnv<GEN> &A) {
  load_par<!GEN>(fv.pa, e, A.P);
  A.F = make_coef<!GEN>(A.P);
  A.xh = GEN ? sxh_row : nullptr;
}

// One thread per env.  ckpt [n_ck][MG_NSTATE][n] (state at sub-steps 0, C, 2C, ...),
// dtraj [T][MG_NTRAJ][n] (loss adjoint of the state after each sub-step).  Outputs: dcoef
// [n][18] (M_A, Dl, Dq diagonals), dact [n_seg][n][w] accumulated, dstate0 [n][21] or null.
// GEN: dynamic shared memory [blockDim.x][MG_NXPARAM] for the block's off-diagonal coefficients.
template <int MT, bool GEN>
__global__ void __launch_bounds__(kAdjThreads)
    k_adjoint(const FleetView fv, const int32_t *__restrict__ types, const float *__restrict__ ckpt,
              const float *__restrict__ dtraj, int32_t T, int32_t C, int64_t step0,
              float *__restrict__ dcoef, float *__restrict__ dact, float *__restrict__ dstate0) {
  __shared__ float4 sgeo[MG_MAX_TYPES][2 * MG_MAX_THR];
  extern __shared__ float sxh[];
  stage_geometry(fv, sgeo);
  const int64_t env0 = (int64_t)blockIdx.x * blockDim.x;
  if constexpr (GEN)
    stage_xh_or_zero(fv, env0, (int)min((int64_t)blockDim.x, fv.n - env0), sxh);
  __syncthreads();
  const int64_t e = env0 + threadIdx.x;
  if (e >= fv.n) return;
  const int type = types[e];
  const float4 *gdir = sgeo[type], *garm = sgeo[type] + MG_MAX_THR;
  const int nt = fv.geo[type].n_thr;
  const bool ca = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);
  const float h = fv.dt;
  const int64_t n = fv.n;
  AdjEnv<GEN> A;
  load_env<GEN>(fv, e, ca, sxh + threadIdx.x * MG_NXPARAM, A);
  const LagEnv L = lag_env(A.P.itau, h);  // the forward's throttle-lag update (replay)

  Grad G;
  zero_grad(G);
  St<MT> lam;
  st_zero(lam);
  St<MT> S[kMaxSeg];
  float c[MT], gcs[MT];

  const int32_t n_ck = (T + C - 1) / C;
  for (int32_t sg = n_ck - 1; sg >= 0; --sg) {
    const int32_t t0 = sg * C, len = min(C, T - t0);
    // re-run the segment from its checkpoint
    load_checkpoint<MT>(ckpt, sg, n, e, S[0]);
    for (int32_t j = 1; j < len; ++j) {
      S[j] = S[j - 1];
      commands_at<MT>(fv, e, step0 + t0 + j - 1, nt, A.P.itau, c);
      float b[MT];
      lag_segment<MT>(c, L, b);
      fwd_step<MT, GEN>(S[j], b, L, A, gdir, garm, nt, ca, h);
    }
    // walk it backwards
    for (int32_t j = len - 1; j >= 0; --j) {
      const int64_t t = t0 + j;
      add_traj_adjoint<MT>(dtraj, t, n, e, lam);
      commands_at<MT>(fv, e, step0 + t, nt, A.P.itau, c);
      for (int i = 0; i < MT; ++i) gcs[i] = 0.f;
      step_vjp<MT, GEN>(S[j], c, A, gdir, garm, nt, ca, h, lam, G, gcs);
      add_action_adjoint<MT>(fv, step0 + t, e, nt, A.P.itau, gcs, dact);
    }
  }
  write_gradients<MT>(G, lam, e, dcoef, dstate0);
}

// ---------------------------------------------------------------- two-warp form
// For fleets with fewer 32-env warps than the GPU has schedulers, where the one-warp kernel
// above leaves most of them idle and runs on instruction latency: blocks of two warps over the
// same 32 envs.  Warp 0 re-runs each checkpoint segment and writes, for every sub-step, the
// stage states the transposes need (q, nu and n of y1..y4, and the quaternion before
// renormalisation) to a workspace; warp 1 applies step_vjp_stages from those records, one
// segment behind.  The workspace holds two segments, used alternately; a block barrier at each
// segment boundary hands one over.  The per-env arithmetic is k_adjoint's: stage_states and
// step_vjp_stages are the two halves of step_vjp.
constexpr int kWsThreads = 64;

template <int MT>
__host__ __device__ constexpr int rec_words() { return 4 * (10 + MT) + 4; }

template <int MT>
__device__ __forceinline__ void put_stage(float *__restrict__ r, int64_t n, int f,
                                          const St<MT> &y) {
  for (int i = 0; i < 4; ++i) r[(int64_t)(f + i) * n] = y.q[i];
  for (int i = 0; i < 3; ++i) r[(int64_t)(f + 4 + i) * n] = y.v[i];
  for (int i = 0; i < 3; ++i) r[(int64_t)(f + 7 + i) * n] = y.w[i];
  for (int i = 0; i < MT; ++i) r[(int64_t)(f + 10 + i) * n] = y.n[i];
}

// Warp 0: segment sg re-run from its checkpoint; record j of `rec` gets sub-step t0 + j.
template <int MT, bool GEN>
__device__ __forceinline__ void produce_segment(const FleetView &fv, int64_t e,
                                                const AdjEnv<GEN> &A, const LagEnv &L,
                                                const float4 *gdir, const float4 *garm, int nt,
                                                bool ca, float h, const float *__restrict__ ckpt,
                                                int32_t sg, int32_t C, int32_t T, int64_t step0,
                                                float *__restrict__ rec) {
  constexpr int W = rec_words<MT>(), Y = 10 + MT;
  const int64_t n = fv.n;
  const int32_t t0 = sg * C, len = min(C, T - t0);
  St<MT> S;
  load_checkpoint<MT>(ckpt, sg, n, e, S);
  float c[MT];
  for (int32_t j = 0; j < len; ++j) {
    commands_at<MT>(fv, e, step0 + t0 + j, nt, A.P.itau, c);
    St<MT> y2, y3, y4, z;
    stage_states<MT, GEN>(S, c, A, gdir, garm, nt, ca, h, y2, y3, y4, z);
    float *r = rec + (int64_t)j * W * n;
    put_stage<MT>(r, n, 0, S);
    put_stage<MT>(r, n, Y, y2);
    put_stage<MT>(r, n, 2 * Y, y3);
    put_stage<MT>(r, n, 3 * Y, y4);
    for (int i = 0; i < 4; ++i) r[(int64_t)(4 * Y + i) * n] = z.q[i];
    if (j + 1 < len) {  // the next start state, as the forward computed it
      float b[MT];
      lag_segment<MT>(c, L, b);
      fwd_step<MT, GEN>(S, b, L, A, gdir, garm, nt, ca, h);
    }
  }
}

// Per-lane asynchronous 4-byte copies global -> shared (sm_80+ cp.async), so that the consumer
// warp's next record is in flight while it works on the current one.
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all_but_one() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// What the consumer reads per sub-step: the stage record, the loss adjoint of the sub-step's
// output and the sub-step's buffered command.
template <int MT>
__host__ __device__ constexpr int fetch_words() { return rec_words<MT>() + MG_NTRAJ + MT; }

// Queue the copies of sub-step t0 + j's inputs into buf [fetch_words][32] (this lane's column).
template <int MT>
__device__ __forceinline__ void fetch_substep(const FleetView &fv, int64_t e,
                                              const float *__restrict__ rec,
                                              const float *__restrict__ dtraj, int64_t t0,
                                              int32_t j, int64_t step0, float *buf) {
  constexpr int W = rec_words<MT>();
  const int64_t n = fv.n;
  const float *r = rec + (int64_t)j * W * n;
  for (int f = 0; f < W; ++f) cp_async4(buf + f * 32, r + (int64_t)f * n);
  const float *g = dtraj + (t0 + j) * MG_NTRAJ * n + e;
  for (int f = 0; f < MG_NTRAJ; ++f) cp_async4(buf + (W + f) * 32, g + (int64_t)f * n);
  if (fv.n_seg > 0) {
    int64_t seg = (step0 + t0 + j) / fv.hold;
    if (seg > fv.n_seg - 1) seg = fv.n_seg - 1;
    const float *a = fv.act + (seg * n + e) * fv.act_w;
    for (int i = 0; i < MT; ++i) cp_async4(buf + (W + MG_NTRAJ + i) * 32, a + i);
  }
  cp_async_commit();
}

template <int MT>
__device__ __forceinline__ void read_stage(const float *buf, int f, St<MT> &y) {
  for (int i = 0; i < 3; ++i) y.p[i] = 0.f;  // p does not enter the right-hand side
  for (int i = 0; i < 4; ++i) y.q[i] = buf[(f + i) * 32];
  for (int i = 0; i < 3; ++i) y.v[i] = buf[(f + 4 + i) * 32];
  for (int i = 0; i < 3; ++i) y.w[i] = buf[(f + 7 + i) * 32];
  for (int i = 0; i < MT; ++i) y.n[i] = buf[(f + 10 + i) * 32];
}

// Warp 1: segment sg walked backwards from its records, each sub-step's inputs copied into
// shared memory (double buffer sbuf [2][fetch_words][32]) while the previous one is processed.
template <int MT, bool GEN>
__device__ __forceinline__ void consume_segment(const FleetView &fv, int64_t e, int lane,
                                                const AdjEnv<GEN> &A, const float4 *gdir,
                                                const float4 *garm, int nt, bool ca, float h,
                                                const float *__restrict__ dtraj, int32_t sg,
                                                int32_t C, int32_t T, int64_t step0,
                                                const float *__restrict__ rec, float *sbuf,
                                                float *__restrict__ dact, St<MT> &lam, Grad &G) {
  constexpr int W = rec_words<MT>(), Y = 10 + MT, F = fetch_words<MT>();
  const int32_t t0 = sg * C, len = min(C, T - t0);
  float c[MT], gcs[MT];
  fetch_substep<MT>(fv, e, rec, dtraj, t0, len - 1, step0, sbuf + ((len - 1) & 1) * F * 32 + lane);
  for (int32_t j = len - 1; j >= 0; --j) {
    if (j > 0)
      fetch_substep<MT>(fv, e, rec, dtraj, t0, j - 1, step0, sbuf + ((j - 1) & 1) * F * 32 + lane);
    else
      cp_async_commit();  // an empty group keeps "all but the newest" meaning sub-step j
    cp_async_wait_all_but_one();
    const float *b = sbuf + (j & 1) * F * 32 + lane;
    const int64_t t = t0 + j;
    for (int i = 0; i < 3; ++i) lam.p[i] += b[(W + i) * 32];
    for (int i = 0; i < 4; ++i) lam.q[i] += b[(W + 3 + i) * 32];
    for (int i = 0; i < 3; ++i) lam.v[i] += b[(W + 7 + i) * 32];
    for (int i = 0; i < 3; ++i) lam.w[i] += b[(W + 10 + i) * 32];
    for (int i = 0; i < MT; ++i)
      c[i] = (fv.n_seg > 0 && i < nt) ? b[(W + MG_NTRAJ + i) * 32] * A.P.itau : 0.f;
    for (int i = 0; i < MT; ++i) gcs[i] = 0.f;
    float zq[4];
    for (int i = 0; i < 4; ++i) zq[i] = b[(4 * Y + i) * 32];
    auto stage = [&](int i, St<MT> &y) { read_stage<MT>(b, i * Y, y); };
    step_vjp_stages<MT, GEN, false>(stage, zq, c, A, gdir, garm, nt, ca, h, lam, G, gcs);
    add_action_adjoint<MT>(fv, step0 + t, e, nt, A.P.itau, gcs, dact);
  }
}

// ws: [2][C][rec_words<MT>()][n] floats.  Grid: one block per 32 envs.  GEN: dynamic shared
// memory [32][MG_NXPARAM] for the block's off-diagonal coefficients (both warps read a lane's
// row).
template <int MT, bool GEN>
__global__ void __launch_bounds__(kWsThreads)
    k_adjoint_ws(const FleetView fv, const int32_t *__restrict__ types,
                 const float *__restrict__ ckpt, const float *__restrict__ dtraj, int32_t T,
                 int32_t C, int64_t step0, float *__restrict__ dcoef, float *__restrict__ dact,
                 float *__restrict__ dstate0, float *__restrict__ ws) {
  __shared__ float4 sgeo[MG_MAX_TYPES][2 * MG_MAX_THR];
  __shared__ float sbuf[2 * fetch_words<MT>() * 32];
  extern __shared__ float sxh[];
  stage_geometry(fv, sgeo);
  const int64_t env0 = (int64_t)blockIdx.x * 32;
  if constexpr (GEN) stage_xh_or_zero(fv, env0, (int)min((int64_t)32, fv.n - env0), sxh);
  __syncthreads();
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  const int64_t e = env0 + lane;
  const bool live = e < fv.n;  // lanes past the fleet only take part in the barriers
  const int64_t el = live ? e : 0;
  const int type = types[el];
  const float4 *gdir = sgeo[type], *garm = sgeo[type] + MG_MAX_THR;
  const int nt = fv.geo[type].n_thr;
  const bool ca = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);
  const float h = fv.dt;
  AdjEnv<GEN> A;
  load_env<GEN>(fv, el, ca, sxh + lane * MG_NXPARAM, A);
  const int64_t slot = (int64_t)C * rec_words<MT>() * fv.n;

  const int32_t n_ck = (T + C - 1) / C;
  if (warp == 0 && live)
    produce_segment<MT, GEN>(fv, e, A, lag_env(A.P.itau, h), gdir, garm, nt, ca, h, ckpt,
                             n_ck - 1, C, T, step0, ws + ((n_ck - 1) & 1) * slot + e);
  __syncthreads();
  Grad G;
  zero_grad(G);
  St<MT> lam;
  st_zero(lam);
  for (int32_t sg = n_ck - 1; sg >= 0; --sg) {
    if (warp == 0) {
      if (live && sg > 0)
        produce_segment<MT, GEN>(fv, e, A, lag_env(A.P.itau, h), gdir, garm, nt, ca, h, ckpt,
                                 sg - 1, C, T, step0, ws + ((sg - 1) & 1) * slot + e);
    } else if (live) {
      consume_segment<MT, GEN>(fv, e, lane, A, gdir, garm, nt, ca, h, dtraj, sg, C, T, step0,
                               ws + (sg & 1) * slot + e, sbuf, dact, lam, G);
    }
    __syncthreads();
  }
  if (warp == 1 && live) write_gradients<MT>(G, lam, e, dcoef, dstate0);
}

template <int MT, bool GEN>
cudaError_t launch_adjoint_t(const FleetView &fv, const int32_t *types, const float *ckpt,
                             const float *dtraj, int32_t T, int32_t C, int64_t step0,
                             float *dcoef, float *dact, float *dstate0, bool split, float *ws,
                             int n_sm, cudaStream_t stream) {
  if (split) {
    const int grid = (int)((fv.n + 31) / 32);
    const size_t smem = GEN ? sizeof(float) * 32 * MG_NXPARAM : 0;
    k_adjoint_ws<MT, GEN><<<grid, kWsThreads, smem, stream>>>(fv, types, ckpt, dtraj, T, C,
                                                               step0, dcoef, dact, dstate0, ws);
    return cudaGetLastError();
  }
  // One warp per block while the fleet has fewer warps than the GPU has SMs x 4 (the backward
  // pass is latency-bound, so its warps should be spread over all SMs, each with its own L1 for
  // the threads' recompute buffers), larger blocks beyond.
  const int64_t warps = (fv.n + 31) / 32;
  const int threads = warps <= 4 * (int64_t)n_sm ? 32 : kAdjThreads;
  const int grid = (int)((fv.n + threads - 1) / threads);
  const size_t smem = GEN ? sizeof(float) * threads * MG_NXPARAM : 0;
  k_adjoint<MT, GEN><<<grid, threads, smem, stream>>>(fv, types, ckpt, dtraj, T, C, step0, dcoef,
                                                      dact, dstate0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- forward pass
// The forward of the differentiable rollout in one launch: T sub-steps from the sim's state on
// the static grid, the state written to ckpt [n_ck][MG_NSTATE][n] (record order, lag entries
// past the vehicle's thrusters zero) before sub-steps 0, C, 2C, ... and the trajectory recorded
// after every sub-step into traj [T][MG_NTRAJ][n].  Per env the arithmetic is advance_env's
// (the same step code, commands and lag segments), so the result equals a chain of recording
// launches of C sub-steps each, bit for bit, without the launches or the state's round trips.
template <int MT>
__device__ __forceinline__ void write_checkpoint(float *__restrict__ ck, int64_t n, int64_t e,
                                                 const St<MT> &s) {
  float *c = ck + e;
  for (int i = 0; i < 3; ++i) c[(int64_t)i * n] = s.p[i];
  for (int i = 0; i < 4; ++i) c[(int64_t)(3 + i) * n] = s.q[i];
  for (int i = 0; i < 3; ++i) c[(int64_t)(7 + i) * n] = s.v[i];
  for (int i = 0; i < 3; ++i) c[(int64_t)(10 + i) * n] = s.w[i];
#pragma unroll
  for (int i = 0; i < MG_MAX_THR; ++i) c[(int64_t)(13 + i) * n] = i < MT ? s.n[i] : 0.f;
}

template <int NTV, bool DIAG, int NH, bool XH>
__global__ void __maxnreg__(XH ? kRegsXH : DIAG ? kRegsWide : kRegsGeneral)
    k_rollout_fwd(const FleetView fv, const BlockDesc *__restrict__ blocks, const int32_t T,
                  const int32_t C, float *__restrict__ traj, float *__restrict__ ckpt) {
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
  if (threadIdx.x == 0) {
    s_done = 0u;
    s_cursor = launch_cursor(fv);
  }
  if constexpr (XH) stage_xh(fv.xh, fv.n, bd.env0, bd.count, sxh);
  __syncthreads();
  if ((int)threadIdx.x >= bd.count) return;
  const int64_t e = (int64_t)bd.env0 + threadIdx.x;
  const int64_t n = fv.n;
  const int nt = MIXED ? bd.n_thr : MT;
  const bool current_accel = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);
  const float h = fv.dt;
  const float *xh = XH ? sxh + threadIdx.x * MG_NXPARAM : nullptr;

  St<MT> s;
  load_state<MT>(fv.st, e, s);
  Coef<DIAG> P;
  {
    Par<DIAG> raw;
    load_par<DIAG>(fv.pa, e, raw);
    P = make_coef<DIAG>(raw);
  }
  const int64_t step0 = s_cursor + fv.cursor_off;
  int64_t seg = step0 / fv.hold;
  int32_t left = fv.hold - (int32_t)(step0 - seg * fv.hold);
  const LagEnv L = lag_env(P.itau, h);
  float b[MT];
  {
    float c[MT];
    load_commands<MT>(fv, e, seg, nt, P.itau, c);
    lag_segment<MT>(c, L, b);
  }
  for (int32_t it = 0; it < T; ++it) {
    if (it % C == 0) write_checkpoint<MT>(ckpt + (int64_t)(it / C) * MG_NSTATE * n, n, e, s);
    if (left == 0) {
      ++seg;
      left = fv.hold;
      float c[MT];
      load_commands<MT>(fv, e, seg, nt, P.itau, c);
      lag_segment<MT>(c, L, b);
    }
    rk4_step_lag<MT, DIAG, MIXED, NH, XH>(s, b, L, P, sdir, sarm, nt, current_accel, h, xh);
    --left;
    record<MT>(traj + (int64_t)it * MG_NTRAJ * n, n, e, s);
  }
  store_and_flag<MT, false>(fv, e, s);
  if (fv.cursor_adv) finish_envs(fv, &s_done, bd.count, fv.cursor_adv);
}

template <int NTV, bool DIAG, int NH, bool XH>
cudaError_t rollout_fwd_t(const FleetView &fv, const BlockDesc *blocks, int n_blocks,
                          int threads, int32_t T, int32_t C, float *traj, float *ckpt,
                          cudaStream_t stream) {
  const size_t smem = XH ? sizeof(float) * threads * MG_NXPARAM : 0;  // <= 46,080 B
  k_rollout_fwd<NTV, DIAG, NH, XH><<<n_blocks, threads, smem, stream>>>(fv, blocks, T, C, traj,
                                                                         ckpt);
  return cudaGetLastError();
}

template <int NTV>
cudaError_t rollout_fwd_d(const FleetView &fv, const BlockDesc *blocks, int n_blocks,
                          int threads, bool diag, bool structured, int32_t T, int32_t C,
                          float *traj, float *ckpt, cudaStream_t stream) {
  if (fv.xh)
    return rollout_fwd_t<NTV, false, 0, true>(fv, blocks, n_blocks, threads, T, C, traj, ckpt,
                                              stream);
  if (diag && structured)
    return rollout_fwd_t<NTV, true, 4, false>(fv, blocks, n_blocks, threads, T, C, traj, ckpt,
                                              stream);
  if (diag)
    return rollout_fwd_t<NTV, true, 0, false>(fv, blocks, n_blocks, threads, T, C, traj, ckpt,
                                              stream);
  return rollout_fwd_t<NTV, false, 0, false>(fv, blocks, n_blocks, threads, T, C, traj, ckpt,
                                             stream);
}

}  // namespace

cudaError_t launch_checkpoint(const StatePlanes &st, int64_t n, float *ck, cudaStream_t stream) {
  k_checkpoint<<<(int)((n + 255) / 256), 256, 0, stream>>>(st, n, ck);
  return cudaGetLastError();
}

cudaError_t launch_rollout_forward(const FleetView &fv, const BlockDesc *blocks, int n_blocks,
                                   int threads, NtVariant ntv, bool diag, bool structured,
                                   int32_t T, int32_t C, float *traj, float *ckpt,
                                   cudaStream_t stream) {
  if (threads < 32 || threads > 256 || threads % 32 || n_blocks < 1 || T < 1 || C < 1 ||
      (fv.xh && diag))
    return cudaErrorInvalidValue;
  switch (ntv) {
    case NT_6:
      return rollout_fwd_d<NT_6>(fv, blocks, n_blocks, threads, diag, structured, T, C, traj,
                                 ckpt, stream);
    case NT_8:
      return rollout_fwd_d<NT_8>(fv, blocks, n_blocks, threads, diag, structured, T, C, traj,
                                 ckpt, stream);
    default:
      return rollout_fwd_d<NT_MIXED>(fv, blocks, n_blocks, threads, diag, structured, T, C,
                                     traj, ckpt, stream);
  }
}

namespace {

cudaError_t sm_count(int *n_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(n_sm, cudaDevAttrMultiProcessorCount, dev);
  return e;
}

}  // namespace

cudaError_t adjoint_split(int64_t n, int mode, bool *split) {
  if (mode == 1 || mode == 2) {
    *split = mode == 2;
    return cudaSuccess;
  }
  // by fleet size: the two-warp form while its 2 x ceil(n / 32) warps fit one per scheduler
  int n_sm = 0;
  cudaError_t e = sm_count(&n_sm);
  if (e != cudaSuccess) return e;
  *split = (n + 31) / 32 <= 2 * (int64_t)n_sm;
  return cudaSuccess;
}

size_t adjoint_workspace_bytes(bool eight, int64_t n, int32_t C) {
  return 2 * (size_t)C * (size_t)(eight ? rec_words<8>() : rec_words<6>()) * (size_t)n *
         sizeof(float);
}

cudaError_t launch_adjoint(const FleetView &fv, const int32_t *types, bool eight, bool general,
                           const float *ckpt, const float *dtraj, int32_t T, int32_t C,
                           int64_t step0, float *dcoef, float *dact, float *dstate0, bool split,
                           float *ws, cudaStream_t stream) {
  if (C < 1 || C > kMaxSeg || T < 1 || (split && !ws)) return cudaErrorInvalidValue;
  int n_sm = 0;
  cudaError_t e = sm_count(&n_sm);
  if (e != cudaSuccess) return e;
  if (eight)
    return general ? launch_adjoint_t<8, true>(fv, types, ckpt, dtraj, T, C, step0, dcoef, dact,
                                               dstate0, split, ws, n_sm, stream)
                   : launch_adjoint_t<8, false>(fv, types, ckpt, dtraj, T, C, step0, dcoef,
                                                dact, dstate0, split, ws, n_sm, stream);
  return general ? launch_adjoint_t<6, true>(fv, types, ckpt, dtraj, T, C, step0, dcoef, dact,
                                             dstate0, split, ws, n_sm, stream)
                 : launch_adjoint_t<6, false>(fv, types, ckpt, dtraj, T, C, step0, dcoef, dact,
                                              dstate0, split, ws, n_sm, stream);
}

int adjoint_max_interval() { return kMaxSeg; }

}  // namespace mg
