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
// Diagonal-mass fleets only (r_g = 0): the coefficient chain rule uses M^-1 = diag(1 / M_jj).
#include <type_traits>

#include "mg_device.cuh"

namespace mg {

namespace {

constexpr int kAdjThreads = 128;

struct Grad {
  float ma[3], J[3], mi[6], dl[6], dq[6];
};

__device__ __forceinline__ void cross_vjp(const float a[3], const float b[3], const float gc[3],
                                          float ga[3], float gb[3]) {
  // c = a x b:  ga += b x gc,  gb += gc x a.
  ga[0] += b[1] * gc[2] - b[2] * gc[1];
  ga[1] += b[2] * gc[0] - b[0] * gc[2];
  ga[2] += b[0] * gc[1] - b[1] * gc[0];
  gb[0] += gc[1] * a[2] - gc[2] * a[1];
  gb[1] += gc[2] * a[0] - gc[0] * a[2];
  gb[2] += gc[0] * a[1] - gc[1] * a[0];
}

// gs += (d rhs / d s)^T gd; parameter and command adjoints accumulated into G and gcs.  The
// forward quantities are recomputed with the formulas of rhs() (diagonal mass); gd.q is the
// adjoint of d.q = q (x) (0, w) (the doubled quaternion rate rhs() stores).
template <int MT>
__device__ void rhs_vjp(const St<MT> &s, const float (&cs)[MT], const ParDiag &P,
                        const float4 *gdir, const float4 *garm, int nt, bool current_accel,
                        const St<MT> &gd, St<MT> &gs, Grad &G, float (&gcs)[MT]) {
  // ---------------- forward recomputation
  float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int i = 0; i < nt; ++i) {
    const float f = s.n[i] * fabsf(s.n[i]);
    const float4 dd = gdir[i], aa = garm[i];
    t[0] += f * dd.x; t[1] += f * dd.y; t[2] += f * dd.z;
    t[3] += f * aa.x; t[4] += f * aa.y; t[5] += f * aa.z;
  }
  const float qw = s.q[0], qx = s.q[1], qy = s.q[2], qz = s.q[3];
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
  const float v[3] = {s.v[0], s.v[1], s.v[2]}, w[3] = {s.w[0], s.w[1], s.w[2]};
  const float vc[3] = {P.vc0, P.vc1, P.vc2}, ma[3] = {P.ma0, P.ma1, P.ma2};
  const float J[3] = {P.J0, P.J1, P.J2}, G3[3] = {P.G0, P.G1, P.G2};
  float cb[3], r[3], qm[3], h[3], k[3], a[3];
  for (int i = 0; i < 3; ++i) cb[i] = R[0][i] * vc[0] + R[1][i] * vc[1] + R[2][i] * vc[2];
  for (int i = 0; i < 3; ++i) {
    r[i] = v[i] - cb[i];
    qm[i] = ma[i] * r[i];
    h[i] = P.m * v[i] + qm[i];
    k[i] = J[i] * w[i];
  }
  a[0] = w[1] * cb[2] - w[2] * cb[1];
  a[1] = w[2] * cb[0] - w[0] * cb[2];
  a[2] = w[0] * cb[1] - w[1] * cb[0];
  const float e[3] = {R[2][0], R[2][1], R[2][2]};
  float f[6];
  f[0] = P.kT * t[0] + P.wb * e[0] - (w[1] * h[2] - w[2] * h[1]) -
         (P.dl[0] + P.dq[0] * fabsf(r[0])) * r[0];
  f[1] = P.kT * t[1] + P.wb * e[1] - (w[2] * h[0] - w[0] * h[2]) -
         (P.dl[1] + P.dq[1] * fabsf(r[1])) * r[1];
  f[2] = P.kT * t[2] + P.wb * e[2] - (w[0] * h[1] - w[1] * h[0]) -
         (P.dl[2] + P.dq[2] * fabsf(r[2])) * r[2];
  if (current_accel)
    for (int i = 0; i < 3; ++i) f[i] -= ma[i] * a[i];
  f[3] = P.kT * t[3] - (r[1] * qm[2] - r[2] * qm[1]) - (w[1] * k[2] - w[2] * k[1]) -
         (P.dl[3] + P.dq[3] * fabsf(w[0])) * w[0] + (G3[1] * e[2] - G3[2] * e[1]);
  f[4] = P.kT * t[4] - (r[2] * qm[0] - r[0] * qm[2]) - (w[2] * k[0] - w[0] * k[2]) -
         (P.dl[4] + P.dq[4] * fabsf(w[1])) * w[1] + (G3[2] * e[0] - G3[0] * e[2]);
  f[5] = P.kT * t[5] - (r[0] * qm[1] - r[1] * qm[0]) - (w[0] * k[1] - w[1] * k[0]) -
         (P.dl[5] + P.dq[5] * fabsf(w[2])) * w[2] + (G3[0] * e[1] - G3[1] * e[0]);

  // ---------------- reverse
  // lag: d.n_i = cs_i - n_i / tau_m
  for (int i = 0; i < nt; ++i) {
    gcs[i] += gd.n[i];
    gs.n[i] -= P.itau * gd.n[i];
  }
  // nu' = M^-1 f
  const float gnu[6] = {gd.v[0], gd.v[1], gd.v[2], gd.w[0], gd.w[1], gd.w[2]};
  float gf[6], gt[6];
  for (int j = 0; j < 6; ++j) {
    gf[j] = P.mi[j] * gnu[j];
    G.mi[j] += f[j] * gnu[j];
    gt[j] = P.kT * gf[j];
  }
  float gw[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f}, gr[3] = {0.f, 0.f, 0.f};
  float gh[3] = {0.f, 0.f, 0.f}, gk[3] = {0.f, 0.f, 0.f}, gqm[3] = {0.f, 0.f, 0.f};
  float gcb[3] = {0.f, 0.f, 0.f}, ge[3] = {0.f, 0.f, 0.f};
  // rotational force
  const float gfr[3] = {gf[3], gf[4], gf[5]};
  const float ngfr[3] = {-gf[3], -gf[4], -gf[5]};
  cross_vjp(r, qm, ngfr, gr, gqm);   // - r x Q1
  cross_vjp(w, k, ngfr, gw, gk);     // - w x k
  for (int j = 0; j < 3; ++j) {
    const float aw = fabsf(w[j]);
    gw[j] -= (P.dl[3 + j] + 2.f * P.dq[3 + j] * aw) * gfr[j];
    G.dl[3 + j] -= w[j] * gfr[j];
    G.dq[3 + j] -= aw * w[j] * gfr[j];
  }
  {
    float gG[3] = {0.f, 0.f, 0.f};
    cross_vjp(G3, e, gfr, gG, ge);   // + G x e
  }
  // translational force
  const float gfl[3] = {gf[0], gf[1], gf[2]};
  const float ngfl[3] = {-gf[0], -gf[1], -gf[2]};
  for (int j = 0; j < 3; ++j) ge[j] += P.wb * gfl[j];
  cross_vjp(w, h, ngfl, gw, gh);     // - w x h
  for (int j = 0; j < 3; ++j) {
    const float ar = fabsf(r[j]);
    gr[j] -= (P.dl[j] + 2.f * P.dq[j] * ar) * gfl[j];
    G.dl[j] -= r[j] * gfl[j];
    G.dq[j] -= ar * r[j] * gfl[j];
  }
  if (current_accel) {
    float ga[3];
    for (int j = 0; j < 3; ++j) {
      G.ma[j] -= a[j] * gfl[j];
      ga[j] = -ma[j] * gfl[j];
    }
    cross_vjp(w, cb, ga, gw, gcb);   // - M_A (w x v_c^b)
  }
  // k = J w, h = m v + Q1, Q1 = M_A r, r = v - v_c^b
  for (int j = 0; j < 3; ++j) {
    gw[j] += J[j] * gk[j];
    G.J[j] += w[j] * gk[j];
    gv[j] += P.m * gh[j];
    gqm[j] += gh[j];
    gr[j] += ma[j] * gqm[j];
    G.ma[j] += r[j] * gqm[j];
    gv[j] += gr[j];
    gcb[j] -= gr[j];
  }
  // R entries: v_c^b = R^T v_c, e = third row of R, p' = R v
  float gR[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) gR[i][j] = vc[i] * gcb[j] + gd.p[i] * v[j];
  for (int j = 0; j < 3; ++j) {
    gR[2][j] += ge[j];
    gv[j] += R[0][j] * gd.p[0] + R[1][j] * gd.p[1] + R[2][j] * gd.p[2];
  }
  // d.q = q (x) (0, w)
  const float g0 = gd.q[0], g1 = gd.q[1], g2 = gd.q[2], g3 = gd.q[3];
  gw[0] += -qx * g0 + qw * g1 + qz * g2 - qy * g3;
  gw[1] += -qy * g0 - qz * g1 + qw * g2 + qx * g3;
  gw[2] += -qz * g0 + qy * g1 - qx * g2 + qw * g3;
  float gq[4];
  gq[0] = w[0] * g1 + w[1] * g2 + w[2] * g3;
  gq[1] = -w[0] * g0 - w[2] * g2 + w[1] * g3;
  gq[2] = -w[1] * g0 + w[2] * g1 - w[0] * g3;
  gq[3] = -w[2] * g0 - w[1] * g1 + w[0] * g2;
  // R(q) -> q
  gq[0] += 2.f * (-qz * gR[0][1] + qz * gR[1][0] + qy * gR[0][2] - qy * gR[2][0] -
                  qx * gR[1][2] + qx * gR[2][1]);
  gq[1] += 2.f * (qy * gR[0][1] + qy * gR[1][0] + qz * gR[0][2] + qz * gR[2][0] -
                  qw * gR[1][2] + qw * gR[2][1]) -
           4.f * qx * (gR[1][1] + gR[2][2]);
  gq[2] += 2.f * (qx * gR[0][1] + qx * gR[1][0] + qw * gR[0][2] - qw * gR[2][0] +
                  qz * gR[1][2] + qz * gR[2][1]) -
           4.f * qy * (gR[0][0] + gR[2][2]);
  gq[3] += 2.f * (-qw * gR[0][1] + qw * gR[1][0] + qx * gR[0][2] + qx * gR[2][0] +
                  qy * gR[1][2] + qy * gR[2][1]) -
           4.f * qz * (gR[0][0] + gR[1][1]);
  // thrust: t = sum_i n_i|n_i| b_i
  for (int i = 0; i < nt; ++i) {
    const float4 dd = gdir[i], aa = garm[i];
    const float gfi = dd.x * gt[0] + dd.y * gt[1] + dd.z * gt[2] + aa.x * gt[3] +
                      aa.y * gt[4] + aa.z * gt[5];
    gs.n[i] += 2.f * fabsf(s.n[i]) * gfi;
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
  for (int i = 0; i < 3; ++i) out.p[i] = (add ? out.p[i] : 0.f) + a * x.p[i];
  for (int i = 0; i < 4; ++i) out.q[i] = (add ? out.q[i] : 0.f) + aq * x.q[i];
  for (int i = 0; i < 3; ++i) out.v[i] = (add ? out.v[i] : 0.f) + a * x.v[i];
  for (int i = 0; i < 3; ++i) out.w[i] = (add ? out.w[i] : 0.f) + a * x.w[i];
  for (int i = 0; i < MT; ++i) out.n[i] = (add ? out.n[i] : 0.f) + a * x.n[i];
}

template <int MT>
__device__ __forceinline__ void st_zero(St<MT> &x) {
  for (int i = 0; i < 3; ++i) x.p[i] = x.v[i] = x.w[i] = 0.f;
  for (int i = 0; i < 4; ++i) x.q[i] = 0.f;
  for (int i = 0; i < MT; ++i) x.n[i] = 0.f;
}

// lam: in, the adjoint of the sub-step's output s+; out, the adjoint of its input s.
//   z  = s + h/6 W k1 + h/3 W k2 + h/3 W k3 + h/6 W k4,  s+ = N(z)
//   y2 = s + h/2 W k1,  y3 = s + h/2 W k2,  y4 = s + h W k3,  k_i = rhs(y_i), y1 = s
// reverse:  lk4 = h/6 W lz,            ly4 = J(y4)^T lk4
//           lk3 = h/3 W lz + h W ly4,   ly3 = J(y3)^T lk3
//           lk2 = h/3 W lz + h/2 W ly3, ly2 = J(y2)^T lk2
//           lk1 = h/6 W lz + h/2 W ly2
//           ls  = lz + ly4 + ly3 + ly2 + J(s)^T lk1
template <int MT>
__device__ void step_vjp(const St<MT> &s, const float (&cs)[MT], const ParDiag &P,
                         const float4 *gdir, const float4 *garm, int nt, bool current_accel,
                         float h, St<MT> &lam, Grad &G, float (&gcs)[MT]) {
  const float hh = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
  St<MT> k, y2, y3, y4, z;
  rhs<MT, true, true>(s, cs, P, gdir, garm, nt, current_accel, k);
  axpy(z, s, h6, k);
  axpy(y2, s, hh, k);
  rhs<MT, true, true>(y2, cs, P, gdir, garm, nt, current_accel, k);
  axpy(z, z, h3, k);
  axpy(y3, s, hh, k);
  rhs<MT, true, true>(y3, cs, P, gdir, garm, nt, current_accel, k);
  axpy(z, z, h3, k);
  axpy(y4, s, h, k);
  rhs<MT, true, true>(y4, cs, P, gdir, garm, nt, current_accel, k);
  axpy(z, z, h6, k);

  // renormalisation q+ = z_q / |z_q|:  lz_q = (lam_q - q+ (q+ . lam_q)) / |z_q|
  const float nq = sqrtf(z.q[0] * z.q[0] + z.q[1] * z.q[1] + z.q[2] * z.q[2] + z.q[3] * z.q[3]);
  float qn[4], dot = 0.f;
  for (int i = 0; i < 4; ++i) {
    qn[i] = z.q[i] / nq;
    dot += qn[i] * lam.q[i];
  }
  St<MT> lz = lam;
  for (int i = 0; i < 4; ++i) lz.q[i] = (lam.q[i] - qn[i] * dot) / nq;

  St<MT> lk, ly;
  St<MT> &ls = lam;
  ls = lz;
  // stage 4
  wscale(lk, lz, h6, false);
  st_zero(ly);
  rhs_vjp<MT>(y4, cs, P, gdir, garm, nt, current_accel, lk, ly, G, gcs);
  wscale(ls, ly, 1.f, true);
  for (int i = 0; i < 4; ++i) ls.q[i] += 0.5f * ly.q[i];  // wscale halved the q part
  // stage 3
  wscale(lk, lz, h3, false);
  wscale(lk, ly, h, true);
  st_zero(ly);
  rhs_vjp<MT>(y3, cs, P, gdir, garm, nt, current_accel, lk, ly, G, gcs);
  wscale(ls, ly, 1.f, true);
  for (int i = 0; i < 4; ++i) ls.q[i] += 0.5f * ly.q[i];
  // stage 2
  wscale(lk, lz, h3, false);
  wscale(lk, ly, hh, true);
  st_zero(ly);
  rhs_vjp<MT>(y2, cs, P, gdir, garm, nt, current_accel, lk, ly, G, gcs);
  wscale(ls, ly, 1.f, true);
  for (int i = 0; i < 4; ++i) ls.q[i] += 0.5f * ly.q[i];
  // stage 1
  wscale(lk, lz, h6, false);
  wscale(lk, ly, hh, true);
  rhs_vjp<MT>(s, cs, P, gdir, garm, nt, current_accel, lk, ls, G, gcs);
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
    const float *a = reinterpret_cast<const float *>(fv.act) + (seg * fv.n + e) * MG_MAX_THR;
    for (int i = 0; i < nt; ++i) c[i] = a[i] * itau;
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

// One thread per env.  ckpt [n_ck][MG_NSTATE][n] (state at sub-steps 0, C, 2C, ...),
// dtraj [T][MG_NTRAJ][n] (loss adjoint of the state after each sub-step).  Outputs: dcoef
// [n][18] (M_A, Dl, Dq diagonals), dact [n_seg][n][8] accumulated, dstate0 [n][21] or null.
template <int MT>
__global__ void __launch_bounds__(kAdjThreads)
    k_adjoint(const FleetView fv, const int32_t *__restrict__ types, const float *__restrict__ ckpt,
              const float *__restrict__ dtraj, int32_t T, int32_t C, int64_t step0,
              float *__restrict__ dcoef, float *__restrict__ dact, float *__restrict__ dstate0) {
  __shared__ float4 sgeo[MG_MAX_TYPES][2 * MG_MAX_THR];
  for (int i = threadIdx.x; i < fv.n_types * 2 * MG_MAX_THR; i += blockDim.x) {
    const int t = i / (2 * MG_MAX_THR), j = i % (2 * MG_MAX_THR);
    sgeo[t][j] = j < MG_MAX_THR ? fv.geo[t].dir[j] : fv.geo[t].arm[j - MG_MAX_THR];
  }
  __syncthreads();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= fv.n) return;
  const int type = types[e];
  const float4 *gdir = sgeo[type], *garm = sgeo[type] + MG_MAX_THR;
  const int nt = fv.geo[type].n_thr;
  const bool ca = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);
  const float h = fv.dt;
  const int64_t n = fv.n;
  ParDiag P;
  load_par<true>(fv.pa, e, P);
  const LagEnv L = lag_env(P.itau, h);  // the forward's throttle-lag update (checkpoint replay)

  Grad G;
  for (int i = 0; i < 3; ++i) G.ma[i] = G.J[i] = 0.f;
  for (int i = 0; i < 6; ++i) G.mi[i] = G.dl[i] = G.dq[i] = 0.f;
  St<MT> lam;
  st_zero(lam);
  St<MT> S[kMaxSeg];
  float c[MT], gcs[MT];

  const int32_t n_ck = (T + C - 1) / C;
  for (int32_t sg = n_ck - 1; sg >= 0; --sg) {
    const int32_t t0 = sg * C, len = min(C, T - t0);
    // re-run the segment from its checkpoint
    const float *ck = ckpt + (int64_t)sg * MG_NSTATE * n + e;
    for (int i = 0; i < 3; ++i) S[0].p[i] = ck[(int64_t)(i)*n];
    for (int i = 0; i < 4; ++i) S[0].q[i] = ck[(int64_t)(3 + i) * n];
    for (int i = 0; i < 3; ++i) S[0].v[i] = ck[(int64_t)(7 + i) * n];
    for (int i = 0; i < 3; ++i) S[0].w[i] = ck[(int64_t)(10 + i) * n];
    for (int i = 0; i < MT; ++i) S[0].n[i] = ck[(int64_t)(13 + i) * n];
    for (int32_t j = 1; j < len; ++j) {
      S[j] = S[j - 1];
      commands_at<MT>(fv, e, step0 + t0 + j - 1, nt, P.itau, c);
      float b[MT];
      lag_segment<MT>(c, L, b);
      rk4_step_lag<MT, true, true>(S[j], b, L, P, gdir, garm, nt, ca, h);
    }
    // walk it backwards
    for (int32_t j = len - 1; j >= 0; --j) {
      const int64_t t = t0 + j;
      const float *g = dtraj + t * MG_NTRAJ * n + e;
      for (int i = 0; i < 3; ++i) lam.p[i] += g[(int64_t)i * n];
      for (int i = 0; i < 4; ++i) lam.q[i] += g[(int64_t)(3 + i) * n];
      for (int i = 0; i < 3; ++i) lam.v[i] += g[(int64_t)(7 + i) * n];
      for (int i = 0; i < 3; ++i) lam.w[i] += g[(int64_t)(10 + i) * n];
      commands_at<MT>(fv, e, step0 + t, nt, P.itau, c);
      for (int i = 0; i < MT; ++i) gcs[i] = 0.f;
      step_vjp<MT>(S[j], c, P, gdir, garm, nt, ca, h, lam, G, gcs);
      if (dact && fv.n_seg > 0) {
        int64_t seg = (step0 + t) / fv.hold;
        if (seg > fv.n_seg - 1) seg = fv.n_seg - 1;
        float *da = dact + (seg * n + e) * MG_MAX_THR;
        for (int i = 0; i < nt; ++i) da[i] += P.itau * gcs[i];
      }
    }
  }
  // coefficients: M_A enters through Q1 (translational), J = diag(I_o) + M_A,rot and
  // M^-1 = diag(1 / (m + M_A,lin), 1 / (I + M_A,rot)): d mi / d M_A = -mi^2.
  float *dc = dcoef + e * 18;
  for (int j = 0; j < 3; ++j) {
    dc[j] = G.ma[j] - P.mi[j] * P.mi[j] * G.mi[j];
    dc[3 + j] = G.J[j] - P.mi[3 + j] * P.mi[3 + j] * G.mi[3 + j];
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

}  // namespace

cudaError_t launch_checkpoint(const StatePlanes &st, int64_t n, float *ck, cudaStream_t stream) {
  k_checkpoint<<<(int)((n + 255) / 256), 256, 0, stream>>>(st, n, ck);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const FleetView &fv, const int32_t *types, bool eight,
                           const float *ckpt, const float *dtraj, int32_t T, int32_t C,
                           int64_t step0, float *dcoef, float *dact, float *dstate0,
                           cudaStream_t stream) {
  if (C < 1 || C > kMaxSeg || T < 1) return cudaErrorInvalidValue;
  // One warp per block while the fleet has fewer warps than the GPU has SMs x 4 (the backward
  // pass is latency-bound, so its warps should be spread over all SMs, each with its own L1 for
  // the threads' recompute buffers), larger blocks beyond.
  int n_sm = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t warps = (fv.n + 31) / 32;
  const int threads = warps <= 4 * (int64_t)n_sm ? 32 : kAdjThreads;
  const int grid = (int)((fv.n + threads - 1) / threads);
  if (eight)
    k_adjoint<8><<<grid, threads, 0, stream>>>(fv, types, ckpt, dtraj, T, C, step0, dcoef, dact,
                                              dstate0);
  else
    k_adjoint<6><<<grid, threads, 0, stream>>>(fv, types, ckpt, dtraj, T, C, step0, dcoef, dact,
                                              dstate0);
  return cudaGetLastError();
}

int adjoint_max_interval() { return kMaxSeg; }

}  // namespace mg
