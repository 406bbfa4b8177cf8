// Device-side building blocks of the fused Fossen step: Philox draws, the right-hand side of
// Eq. 1 (§METHOD) for one vehicle held in registers, and the RK4 sub-step.
//
// Formulation (same mathematics as Eq. 1, arranged for one thread per vehicle in FP32):
//   - Coriolis terms in Kirchhoff's vector form: with [P1;P2] = M_RB nu and [Q1;Q2] = M_A nu_r,
//       C_RB(nu) nu   = [w x P1 ; v x P1 + w x P2]
//       C_A(nu_r)nu_r = [w x Q1 ; v_r x Q1 + w x Q2]
//     which is what Fossen's momentum-block matrices multiply out to; the two are summed before
//     the cross products.
//   - Restoring vector from the third row of R(q): k = R^T e3, g = -[(W - B) k ; G x k],
//     G = W r_g - B r_b.
//   - The mass matrix M = M_RB + M_A is inverted once per parameter change (FP64 Cholesky, see
//     mg_setup.cu); the step multiplies by the stored FP32 inverse.
#pragma once

#include <type_traits>

#include "mg_internal.h"

namespace mg {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC 2011): ten
// rounds of two 32x32->64-bit products; the key is bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

// Draw block `block` of stream `stream` for env id `gid` under key `seed`.
__device__ __forceinline__ uint4 draw4(uint64_t seed, uint64_t gid, uint32_t stream,
                                       uint32_t block) {
  return philox4x32_10(make_uint4((uint32_t)gid, (uint32_t)(gid >> 32), stream, block),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Open-interval uniform from the top 23 bits: ((x >> 9) + 1/2) 2^-23 (exact in FP32).
__device__ __forceinline__ float u01f(uint32_t x) {
  return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f);
}
__device__ __forceinline__ double u01d(uint32_t x) {
  return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

// Counter streams of the draws (shared with the host-side documentation in mg.h).
enum : uint32_t { STREAM_PARAMS = 0, STREAM_CURRENT = 1, STREAM_RESET = 2, STREAM_CMD = 3 };

// Procedural throttle commands of segment seg for env id gid: c_i = 2u - 1 (stream 3, blocks
// 2 seg and 2 seg + 1 give thrusters 0..3 and 4..7).
template <int MT>
__device__ __forceinline__ void procedural_commands(uint64_t seed, uint64_t gid, int64_t seg,
                                                    float (&c)[MT]) {
  const uint4 a = draw4(seed, gid, STREAM_CMD, (uint32_t)(2 * seg));
  c[0] = 2.f * u01f(a.x) - 1.f; c[1] = 2.f * u01f(a.y) - 1.f;
  c[2] = 2.f * u01f(a.z) - 1.f; c[3] = 2.f * u01f(a.w) - 1.f;
  const uint4 b = draw4(seed, gid, STREAM_CMD, (uint32_t)(2 * seg + 1));
  c[4] = 2.f * u01f(b.x) - 1.f; c[5] = 2.f * u01f(b.y) - 1.f;
  if constexpr (MT > 6) {
    c[6] = 2.f * u01f(b.z) - 1.f;
    c[7] = 2.f * u01f(b.w) - 1.f;
  }
}

// Box-Muller pair from two open-interval uniforms (FP64).
__device__ __forceinline__ void box_muller(double u1, double u2, double &z0, double &z1) {
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Box-Muller in FP32, for the episode-start draws: the same uniforms (exact in FP32) and the
// same formula, each result within a few ulp of the FP64 form.  Resets run inside step-time
// kernels (auto-reset), where a warp with one resetting env would otherwise pay GB300's
// reduced-rate FP64 transcendentals for all 32 lanes.
__device__ __forceinline__ void box_muller_f(float u1, float u2, float &z0, float &z1) {
  const float r = sqrtf(-2.f * logf(u1));
  float s, c;
  sincospif(2.f * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Initial body velocity of episode ep of env id gid: nu = sigma N(0,1)^6 from stream 2 (blocks
// 2 ep, 2 ep + 1).
__device__ __forceinline__ void reset_nu(uint64_t seed, uint64_t gid, uint32_t ep, double sigma,
                                         float (&nu)[6]) {
  const uint4 a = draw4(seed, gid, STREAM_RESET, 2u * ep);
  const uint4 b = draw4(seed, gid, STREAM_RESET, 2u * ep + 1u);
  float z[6];
  box_muller_f(u01f(a.x), u01f(a.y), z[0], z[1]);
  box_muller_f(u01f(a.z), u01f(a.w), z[2], z[3]);
  box_muller_f(u01f(b.x), u01f(b.y), z[4], z[5]);
  const float sg = (float)sigma;
#pragma unroll
  for (int i = 0; i < 6; ++i) nu[i] = sg * z[i];
}

// New episode for env e (episode reset, §METHOD randomisation of the start): p = 0, q =
// identity, n = 0, nu from reset_nu at the env's episode counter; the counter is incremented and
// the non-finite flag cleared.
__device__ __forceinline__ void reset_env(const StatePlanes &st, int64_t e, uint64_t gid,
                                          uint64_t seed, double sigma, uint32_t *episode,
                                          uint32_t *flags, unsigned long long *nonfinite_count) {
  const uint32_t ep = episode[e];
  float nu[6];
  reset_nu(seed, gid, ep, sigma, nu);
  st.s0[e] = make_float4(0.f, 0.f, 0.f, 1.f);
  st.s1[e] = make_float4(0.f, 0.f, 0.f, nu[0]);
  st.s2[e] = make_float4(nu[1], nu[2], nu[3], nu[4]);
  st.s3[e] = make_float4(nu[5], 0.f, 0.f, 0.f);
  st.s4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  st.s5[e] = 0.f;
  episode[e] = ep + 1u;
  if (flags[e] & 1u) atomicAdd(nonfinite_count, ~0ull);  // decrement
  flags[e] = 0u;
}

// ---------------------------------------------------------------- per-env registers
template <int MT>
struct St {
  float p[3], q[4], v[3], w[3], n[MT];
};

// Diagonal-mass parameters (34 floats).
struct ParDiag {
  float m, ma0, ma1, ma2;   // mass, translational added mass
  float J0, J1, J2, wb;     // diag(I_o) + rotational added mass, W - B
  float dl[6], dq[6];       // linear, quadratic damping
  float G0, G1, G2, kT;     // W r_g - B r_b, thrust coefficient
  float vc0, vc1, vc2, itau;  // NED current, 1 / tau_m
  float mi[6];              // diagonal of M^-1
};

// General parameters: off-centre gravity (off-diagonal M_RB, full M^-1).
struct ParGen : ParDiag {
  float mrg0, mrg1, mrg2;   // m r_g
  float Ixy, Ixz, Iyz;      // off-diagonal of I_o = I_g - m S(r_g)^2
  float mo[15];             // off-diagonal of M^-1: 01 02 03 04 05 12 13 14 15 23 24 25 34 35 45
};

template <bool DIAG>
using Par = typename std::conditional<DIAG, ParDiag, ParGen>::type;

// Diagonal-mass step coefficients, formed from ParDiag once per launch.  With r_g = 0 and
// diagonal M_A, M = M_RB + M_A is diagonal, and Eq. 1's row i reads nu'_i = f_i / M_ii.  Every
// parameter that multiplies a term of f_i is stored pre-multiplied by (M^-1)_ii, so each row's
// chain of FMAs ends in nu'_i itself, and the Kirchhoff Coriolis terms are expanded into the
// products they reduce to when M_RB and M_A are diagonal (row indices i, i1 = i+1, i2 = i+2 mod 3;
// r = v - v_c^b):
//   translational, -(w x (m v + M_A r)) - M_A (w x v_c^b) with v_c^b = v - r:
//     w_i2 [(m + Ma_i) v_i1 + (Ma_i1 - Ma_i) r_i1] - w_i1 [(m + Ma_i) v_i2 + (Ma_i2 - Ma_i) r_i2],
//     and (m + Ma_i) / M_ii = 1, so the v terms carry no coefficient;
//   rotational, -(r x M_A r) - (w x J w):  (Ma_i1 - Ma_i2) r_i1 r_i2 + (J_i1 - J_i2) w_i1 w_i2.
// The same mathematics as the general path (rhs with ParGen), in fewer operations.  It includes
// the current-acceleration term M_A [w x v_c^b; 0] (the default model); a sim with that term
// switched off (MG_MODEL_NO_CURRENT_ACCEL) runs the general path.
struct StepDiag {
  // translational rows: mi kT, mi (W - B), mi (Ma_i1 - Ma_i), mi (Ma_i2 - Ma_i), mi Dl_i, mi Dq_i
  // (mi = 1 / M_ii)
  float At[3], Wt[3], bp[3], bm[3], dlt[3], dqt[3];
  // rotational rows: mi kT, mi (Ma_i1 - Ma_i2), mi (J_i1 - J_i2), mi Dl, mi Dq, mi G_i1, mi G_i2
  float Ar[3], B[3], C[3], dlr[3], dqr[3], Gp[3], Gm[3];
  float vc0, vc1, vc2, itau;  // NED current, 1 / tau_m
};

__device__ __forceinline__ StepDiag step_diag(const ParDiag &P) {
  StepDiag C;
  const float ma[3] = {P.ma0, P.ma1, P.ma2}, J[3] = {P.J0, P.J1, P.J2};
  const float G[3] = {P.G0, P.G1, P.G2};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
    const float mt = P.mi[i], mr = P.mi[3 + i];
    C.At[i] = mt * P.kT;
    C.Wt[i] = mt * P.wb;
    C.bp[i] = mt * (ma[i1] - ma[i]);
    C.bm[i] = mt * (ma[i2] - ma[i]);
    C.dlt[i] = mt * P.dl[i];
    C.dqt[i] = mt * P.dq[i];
    C.Ar[i] = mr * P.kT;
    C.B[i] = mr * (ma[i1] - ma[i2]);
    C.C[i] = mr * (J[i1] - J[i2]);
    C.dlr[i] = mr * P.dl[3 + i];
    C.dqr[i] = mr * P.dq[3 + i];
    C.Gp[i] = mr * G[i1];
    C.Gm[i] = mr * G[i2];
  }
  C.vc0 = P.vc0; C.vc1 = P.vc1; C.vc2 = P.vc2; C.itau = P.itau;
  return C;
}

// What the step's right-hand side reads: the diagonal-mass coefficients above, or the general
// parameters as loaded.
template <bool DIAG>
using Coef = typename std::conditional<DIAG, StepDiag, ParGen>::type;

template <bool DIAG>
__device__ __forceinline__ Coef<DIAG> make_coef(const Par<DIAG> &P) {
  if constexpr (DIAG) return step_diag(P);
  else return P;
}

__device__ __forceinline__ float4 ldg4(const float4 *p, int64_t e) { return __ldg(p + e); }

template <bool DIAG>
__device__ __forceinline__ void load_par(const ParamPlanes &pa, int64_t e, Par<DIAG> &P) {
  float4 a = ldg4(pa.d0, e), b = ldg4(pa.d1, e), c = ldg4(pa.d2, e), d = ldg4(pa.d3, e);
  float4 f = ldg4(pa.d4, e), g = ldg4(pa.d5, e), h = ldg4(pa.d6, e), i = ldg4(pa.d7, e);
  float2 j = __ldg(pa.d8 + e);
  P.m = a.x; P.ma0 = a.y; P.ma1 = a.z; P.ma2 = a.w;
  P.J0 = b.x; P.J1 = b.y; P.J2 = b.z; P.wb = b.w;
  P.dl[0] = c.x; P.dl[1] = c.y; P.dl[2] = c.z; P.dl[3] = c.w;
  P.dl[4] = d.x; P.dl[5] = d.y; P.dq[0] = d.z; P.dq[1] = d.w;
  P.dq[2] = f.x; P.dq[3] = f.y; P.dq[4] = f.z; P.dq[5] = f.w;
  P.G0 = g.x; P.G1 = g.y; P.G2 = g.z; P.kT = g.w;
  P.vc0 = h.x; P.vc1 = h.y; P.vc2 = h.z; P.itau = h.w;
  P.mi[0] = i.x; P.mi[1] = i.y; P.mi[2] = i.z; P.mi[3] = i.w; P.mi[4] = j.x; P.mi[5] = j.y;
  if constexpr (!DIAG) {
    float4 k0 = ldg4(pa.g0, e), k1 = ldg4(pa.g1, e), k2 = ldg4(pa.g2, e), k3 = ldg4(pa.g3, e);
    float4 k4 = ldg4(pa.g4, e);
    float k5 = __ldg(pa.g5 + e);
    P.mrg0 = k0.x; P.mrg1 = k0.y; P.mrg2 = k0.z; P.Ixy = k0.w;
    P.Ixz = k1.x; P.Iyz = k1.y; P.mo[0] = k1.z; P.mo[1] = k1.w;
    P.mo[2] = k2.x; P.mo[3] = k2.y; P.mo[4] = k2.z; P.mo[5] = k2.w;
    P.mo[6] = k3.x; P.mo[7] = k3.y; P.mo[8] = k3.z; P.mo[9] = k3.w;
    P.mo[10] = k4.x; P.mo[11] = k4.y; P.mo[12] = k4.z; P.mo[13] = k4.w;
    P.mo[14] = k5;
  }
}

// L2 = true loads through L2 only (ld.cg): needed when another SM may have written the state
// during the same kernel (work-queue schedule), so that no stale L1 line is read.
template <int MT, bool L2 = false>
__device__ __forceinline__ void load_state(const StatePlanes &sp, int64_t e, St<MT> &s) {
  const float4 a = L2 ? __ldcg(sp.s0 + e) : sp.s0[e], b = L2 ? __ldcg(sp.s1 + e) : sp.s1[e];
  const float4 c = L2 ? __ldcg(sp.s2 + e) : sp.s2[e], d = L2 ? __ldcg(sp.s3 + e) : sp.s3[e];
  const float4 f = L2 ? __ldcg(sp.s4 + e) : sp.s4[e];
  s.p[0] = a.x; s.p[1] = a.y; s.p[2] = a.z; s.q[0] = a.w;
  s.q[1] = b.x; s.q[2] = b.y; s.q[3] = b.z; s.v[0] = b.w;
  s.v[1] = c.x; s.v[2] = c.y; s.w[0] = c.z; s.w[1] = c.w;
  s.w[2] = d.x; s.n[0] = d.y; s.n[1] = d.z; s.n[2] = d.w;
  s.n[3] = f.x; s.n[4] = f.y; s.n[5] = f.z;
  if constexpr (MT > 6) {
    s.n[6] = f.w;
    s.n[7] = L2 ? __ldcg(sp.s5 + e) : sp.s5[e];
  }
}

template <int MT>
__device__ __forceinline__ void store_state(const StatePlanes &sp, int64_t e, const St<MT> &s) {
  sp.s0[e] = make_float4(s.p[0], s.p[1], s.p[2], s.q[0]);
  sp.s1[e] = make_float4(s.q[1], s.q[2], s.q[3], s.v[0]);
  sp.s2[e] = make_float4(s.v[1], s.v[2], s.w[0], s.w[1]);
  sp.s3[e] = make_float4(s.w[2], s.n[0], s.n[1], s.n[2]);
  if constexpr (MT > 6) {
    sp.s4[e] = make_float4(s.n[3], s.n[4], s.n[5], s.n[6]);
    sp.s5[e] = s.n[7];
  } else {
    sp.s4[e] = make_float4(s.n[3], s.n[4], s.n[5], 0.0f);
  }
}

// ---------------------------------------------------------------- right-hand side of Eq. 1
// d = f(s; c) with two storage conventions that save multiplies in the hot loop:
//   - cs[i] = c_i / tau_m (the command pre-divided by the lag constant once per segment), so
//     n_i' = cs_i - n_i / tau_m is a single FMA;
//   - d.q holds 2 q' (the 1/2 of q' = 1/2 q (x) (0, w) is folded into the RK4 weights).
// Every sum is written as a chain of FMAs (same terms as Eq. 1; only the rounding order differs
// from a term-by-term evaluation).  The diagonal-mass path reads the StepDiag coefficients (each
// row's chain ends in nu'_i, no separate M^-1 multiply); the general path reads ParGen and
// multiplies the generalised force by the full M^-1.
// gdir/garm: the block's vehicle type's thruster directions and moment arms (shared memory),
// zero past its thruster count; MIXED (fleets with several thruster counts) evaluates all MT
// thrusters, the absent ones contributing exact zeros (their command is zeroed by the caller and
// their lag state stays 0), so no warp branches on the count.  NH > 0 selects the vectored layout's
// allocation: thrusters [0, NH) horizontal (d_z = 0: no heave force), the rest vertical
// (d_x = d_y = 0, so r x d has no yaw component); the skipped products are exact zeros, so the
// result is bit-identical to the dense 6 x N allocation (NH = 0).
//
// XH (general path only): the env's off-diagonal hydrodynamic coefficients xh[MG_NXPARAM]
// (M_A above its diagonal, then D_l's off-diagonal entries, both row-major; mg.h) enter the
// added-mass momenta Q = M_A nu_r, the current term M_A [w x v_c^b; 0] and the damping D_l nu_r.
// LAGD = false leaves d.n unset (the caller integrates the linear throttle lag in closed form).
// The diagonal-mass path always includes the current-acceleration term (current_accel unused).
template <int MT, bool DIAG, bool MIXED, int NH = 0, bool XH = false, bool LAGD = true>
__device__ __forceinline__ void rhs(const St<MT> &s, const float (&cs)[MT], const Coef<DIAG> &P,
                                    const float4 *gdir, const float4 *garm, int nt,
                                    bool current_accel, St<MT> &d,
                                    const float *__restrict__ xh = nullptr) {
  static_assert(!(XH && DIAG), "the off-diagonal hydrodynamics use the general path");
  // Thrusters (Eq. 3 actions): F_i = kT n_i|n_i| along d_i at r_i; n_i' = (c_i - n_i) / tau_m.
  float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, t4 = 0.f, t5 = 0.f;
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    {
      const float f = s.n[i] * fabsf(s.n[i]);
      const float4 dd = gdir[i], aa = garm[i];
      if (NH == 0) {
        t0 = fmaf(f, dd.x, t0); t1 = fmaf(f, dd.y, t1); t2 = fmaf(f, dd.z, t2);
        t3 = fmaf(f, aa.x, t3); t4 = fmaf(f, aa.y, t4); t5 = fmaf(f, aa.z, t5);
      } else if (i < NH) {
        t0 = fmaf(f, dd.x, t0); t1 = fmaf(f, dd.y, t1);
        t3 = fmaf(f, aa.x, t3); t4 = fmaf(f, aa.y, t4); t5 = fmaf(f, aa.z, t5);
      } else {
        t2 = fmaf(f, dd.z, t2); t3 = fmaf(f, aa.x, t3); t4 = fmaf(f, aa.y, t4);
      }
      if constexpr (LAGD) d.n[i] = fmaf(-s.n[i], P.itau, cs[i]);
    }
  }
  (void)nt;

  // Attitude matrix R(q) = I + 2 q_w S(eps) + 2 S(eps)^2 (body -> NED), written out.
  const float qw = s.q[0], qx = s.q[1], qy = s.q[2], qz = s.q[3];
  const float tx = qx + qx, ty = qy + qy, tz = qz + qz;
  const float zdiag = fmaf(-qz, tz, 1.f);
  const float R00 = fmaf(-qy, ty, zdiag), R11 = fmaf(-qx, tx, zdiag);
  const float R22 = fmaf(-qx, tx, fmaf(-qy, ty, 1.f));
  const float xy = qx * ty, xz = qx * tz, yz = qy * tz;
  const float R01 = fmaf(-qw, tz, xy), R10 = fmaf(qw, tz, xy);
  const float R02 = fmaf(qw, ty, xz), R20 = fmaf(-qw, ty, xz);
  const float R12 = fmaf(-qw, tx, yz), R21 = fmaf(qw, tx, yz);

  const float v0 = s.v[0], v1 = s.v[1], v2 = s.v[2];
  const float w0 = s.w[0], w1 = s.w[1], w2 = s.w[2];

  if constexpr (DIAG) {
    (void)current_accel;
    // Velocity relative to the current (constant in NED): r = v - R^T v_c.
    const float r0 = fmaf(-R20, P.vc2, fmaf(-R10, P.vc1, fmaf(-R00, P.vc0, v0)));
    const float r1 = fmaf(-R21, P.vc2, fmaf(-R11, P.vc1, fmaf(-R01, P.vc0, v1)));
    const float r2 = fmaf(-R22, P.vc2, fmaf(-R12, P.vc1, fmaf(-R02, P.vc0, v2)));
    // Translational rows (StepDiag): thrust, (W - B) k_e with k_e = R^T e3 = (R20, R21, R22),
    // the expanded Coriolis terms, damping.
    {
      const float u0 = fmaf(P.bp[0], r1, v1), x0 = fmaf(P.bm[0], r2, v2);
      const float u1 = fmaf(P.bp[1], r2, v2), x1 = fmaf(P.bm[1], r0, v0);
      const float u2 = fmaf(P.bp[2], r0, v0), x2 = fmaf(P.bm[2], r1, v1);
      float a0 = fmaf(P.Wt[0], R20, P.At[0] * t0);
      float a1 = fmaf(P.Wt[1], R21, P.At[1] * t1);
      float a2 = fmaf(P.Wt[2], R22, P.At[2] * t2);
      a0 = fmaf(-w1, x0, fmaf(w2, u0, a0));
      a1 = fmaf(-w2, x1, fmaf(w0, u1, a1));
      a2 = fmaf(-w0, x2, fmaf(w1, u2, a2));
      d.v[0] = fmaf(-fmaf(P.dqt[0], fabsf(r0), P.dlt[0]), r0, a0);
      d.v[1] = fmaf(-fmaf(P.dqt[1], fabsf(r1), P.dlt[1]), r1, a1);
      d.v[2] = fmaf(-fmaf(P.dqt[2], fabsf(r2), P.dlt[2]), r2, a2);
    }
    // Rotational rows: thrust moment, G x k_e, Munk and gyroscopic products, damping.
    {
      float b0 = fmaf(-P.Gm[0], R21, fmaf(P.Gp[0], R22, P.Ar[0] * t3));
      float b1 = fmaf(-P.Gm[1], R22, fmaf(P.Gp[1], R20, P.Ar[1] * t4));
      float b2 = fmaf(-P.Gm[2], R20, fmaf(P.Gp[2], R21, P.Ar[2] * t5));
      b0 = fmaf(P.C[0] * w1, w2, fmaf(P.B[0] * r1, r2, b0));
      b1 = fmaf(P.C[1] * w2, w0, fmaf(P.B[1] * r2, r0, b1));
      b2 = fmaf(P.C[2] * w0, w1, fmaf(P.B[2] * r0, r1, b2));
      d.w[0] = fmaf(-fmaf(P.dqr[0], fabsf(w0), P.dlr[0]), w0, b0);
      d.w[1] = fmaf(-fmaf(P.dqr[1], fabsf(w1), P.dlr[1]), w1, b1);
      d.w[2] = fmaf(-fmaf(P.dqr[2], fabsf(w2), P.dlr[2]), w2, b2);
    }
  } else {
    // Current constant in NED, seen from the body: v_c^b = R^T v_c; relative velocity v_r.
    const float cb0 = fmaf(R20, P.vc2, fmaf(R10, P.vc1, R00 * P.vc0));
    const float cb1 = fmaf(R21, P.vc2, fmaf(R11, P.vc1, R01 * P.vc0));
    const float cb2 = fmaf(R22, P.vc2, fmaf(R12, P.vc1, R02 * P.vc0));
    const float r0 = v0 - cb0, r1 = v1 - cb1, r2 = v2 - cb2;

    // Momenta: Q1 = M_A,lin v_r; h = P1 + Q1 = m v + Q1 + w x m r_g;
    //          k = P2 + Q2 = (diag(I_o) + M_A,rot) w + off-diagonal I_o w + m r_g x v.
    float q0 = P.ma0 * r0, q1 = P.ma1 * r1, q2 = P.ma2 * r2;
    float k0 = P.J0 * w0, k1 = P.J1 * w1, k2 = P.J2 * w2;
    if constexpr (XH) {
      // off-diagonal added mass: Q_i += sum_{j != i} M_A,ij nu_r,j (upper triangle, mirrored)
      const float *A = xh;  // 01 02 03 04 05 12 13 14 15 23 24 25 34 35 45
      q0 = fmaf(A[0], r1, fmaf(A[1], r2, fmaf(A[2], w0, fmaf(A[3], w1, fmaf(A[4], w2, q0)))));
      q1 = fmaf(A[0], r0, fmaf(A[5], r2, fmaf(A[6], w0, fmaf(A[7], w1, fmaf(A[8], w2, q1)))));
      q2 = fmaf(A[1], r0, fmaf(A[5], r1, fmaf(A[9], w0, fmaf(A[10], w1, fmaf(A[11], w2, q2)))));
      k0 = fmaf(A[2], r0, fmaf(A[6], r1, fmaf(A[9], r2, fmaf(A[12], w1, fmaf(A[13], w2, k0)))));
      k1 = fmaf(A[3], r0, fmaf(A[7], r1, fmaf(A[10], r2, fmaf(A[12], w0, fmaf(A[14], w2, k1)))));
      k2 = fmaf(A[4], r0, fmaf(A[8], r1, fmaf(A[11], r2, fmaf(A[13], w0, fmaf(A[14], w1, k2)))));
    }
    float h0 = fmaf(P.m, v0, q0), h1 = fmaf(P.m, v1, q1), h2 = fmaf(P.m, v2, q2);
    const float a0 = fmaf(w1, P.mrg2, -w2 * P.mrg1);  // w x m r_g
    const float a1 = fmaf(w2, P.mrg0, -w0 * P.mrg2);
    const float a2 = fmaf(w0, P.mrg1, -w1 * P.mrg0);
    h0 += a0; h1 += a1; h2 += a2;
    k0 = fmaf(P.Ixy, w1, fmaf(P.Ixz, w2, fmaf(P.mrg1, v2, fmaf(-P.mrg2, v1, k0))));
    k1 = fmaf(P.Ixy, w0, fmaf(P.Iyz, w2, fmaf(P.mrg2, v0, fmaf(-P.mrg0, v2, k1))));
    k2 = fmaf(P.Ixz, w0, fmaf(P.Iyz, w1, fmaf(P.mrg0, v1, fmaf(-P.mrg1, v0, k2))));

    // Translational generalised force:
    //   kT t + (W - B) k_e - w x h - (Dl + Dq |v_r|) v_r [- M_A,lin (w x v_c^b)],
    // with k_e = R^T e3 = (R20, R21, R22) the restoring direction.
    float f0 = fmaf(P.wb, R20, P.kT * t0);
    float f1 = fmaf(P.wb, R21, P.kT * t1);
    float f2 = fmaf(P.wb, R22, P.kT * t2);
    f0 = fmaf(w2, h1, fmaf(-w1, h2, f0));
    f1 = fmaf(w0, h2, fmaf(-w2, h0, f1));
    f2 = fmaf(w1, h0, fmaf(-w0, h1, f2));
    f0 = fmaf(-fmaf(P.dq[0], fabsf(r0), P.dl[0]), r0, f0);
    f1 = fmaf(-fmaf(P.dq[1], fabsf(r1), P.dl[1]), r1, f1);
    f2 = fmaf(-fmaf(P.dq[2], fabsf(r2), P.dl[2]), r2, f2);
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;  // w x v_c^b
    if (current_accel) {
      c0 = fmaf(w1, cb2, -w2 * cb1);
      c1 = fmaf(w2, cb0, -w0 * cb2);
      c2 = fmaf(w0, cb1, -w1 * cb0);
      f0 = fmaf(-P.ma0, c0, f0);
      f1 = fmaf(-P.ma1, c1, f1);
      f2 = fmaf(-P.ma2, c2, f2);
    }
    if constexpr (XH) {
      // off-diagonal current term and linear damping of the translational rows
      const float *A = xh, *Dl = xh + 15;  // Dl: row-major off-diagonal, 5 per row
      f0 = fmaf(-A[0], c1, fmaf(-A[1], c2, f0));
      f1 = fmaf(-A[0], c0, fmaf(-A[5], c2, f1));
      f2 = fmaf(-A[1], c0, fmaf(-A[5], c1, f2));
      f0 = fmaf(-Dl[0], r1, fmaf(-Dl[1], r2, fmaf(-Dl[2], w0, fmaf(-Dl[3], w1,
               fmaf(-Dl[4], w2, f0)))));
      f1 = fmaf(-Dl[5], r0, fmaf(-Dl[6], r2, fmaf(-Dl[7], w0, fmaf(-Dl[8], w1,
               fmaf(-Dl[9], w2, f1)))));
      f2 = fmaf(-Dl[10], r0, fmaf(-Dl[11], r1, fmaf(-Dl[12], w0, fmaf(-Dl[13], w1,
               fmaf(-Dl[14], w2, f2)))));
    }
    // Rotational: kT t' - v_r x Q1 - w x k - v x (w x m r_g) - (Dl + Dq|w|) w + G x k_e.
    float f3 = fmaf(r2, q1, fmaf(-r1, q2, P.kT * t3));
    float f4 = fmaf(r0, q2, fmaf(-r2, q0, P.kT * t4));
    float f5 = fmaf(r1, q0, fmaf(-r0, q1, P.kT * t5));
    f3 = fmaf(w2, k1, fmaf(-w1, k2, f3));
    f4 = fmaf(w0, k2, fmaf(-w2, k0, f4));
    f5 = fmaf(w1, k0, fmaf(-w0, k1, f5));
    f3 = fmaf(v2, a1, fmaf(-v1, a2, f3));
    f4 = fmaf(v0, a2, fmaf(-v2, a0, f4));
    f5 = fmaf(v1, a0, fmaf(-v0, a1, f5));
    f3 = fmaf(-fmaf(P.dq[3], fabsf(w0), P.dl[3]), w0, f3);
    f4 = fmaf(-fmaf(P.dq[4], fabsf(w1), P.dl[4]), w1, f4);
    f5 = fmaf(-fmaf(P.dq[5], fabsf(w2), P.dl[5]), w2, f5);
    f3 = fmaf(-P.G2, R21, fmaf(P.G1, R22, f3));
    f4 = fmaf(-P.G0, R22, fmaf(P.G2, R20, f4));
    f5 = fmaf(-P.G1, R20, fmaf(P.G0, R21, f5));
    if constexpr (XH) {
      // off-diagonal current term and linear damping of the rotational rows
      const float *A = xh, *Dl = xh + 15;
      f3 = fmaf(-A[2], c0, fmaf(-A[6], c1, fmaf(-A[9], c2, f3)));
      f4 = fmaf(-A[3], c0, fmaf(-A[7], c1, fmaf(-A[10], c2, f4)));
      f5 = fmaf(-A[4], c0, fmaf(-A[8], c1, fmaf(-A[11], c2, f5)));
      f3 = fmaf(-Dl[15], r0, fmaf(-Dl[16], r1, fmaf(-Dl[17], r2, fmaf(-Dl[18], w1,
               fmaf(-Dl[19], w2, f3)))));
      f4 = fmaf(-Dl[20], r0, fmaf(-Dl[21], r1, fmaf(-Dl[22], r2, fmaf(-Dl[23], w0,
               fmaf(-Dl[24], w2, f4)))));
      f5 = fmaf(-Dl[25], r0, fmaf(-Dl[26], r1, fmaf(-Dl[27], r2, fmaf(-Dl[28], w0,
               fmaf(-Dl[29], w1, f5)))));
    }

    // nu' = M^-1 f.
    const float *o = P.mo;
    d.v[0] = P.mi[0] * f0 + o[0] * f1 + o[1] * f2 + o[2] * f3 + o[3] * f4 + o[4] * f5;
    d.v[1] = o[0] * f0 + P.mi[1] * f1 + o[5] * f2 + o[6] * f3 + o[7] * f4 + o[8] * f5;
    d.v[2] = o[1] * f0 + o[5] * f1 + P.mi[2] * f2 + o[9] * f3 + o[10] * f4 + o[11] * f5;
    d.w[0] = o[2] * f0 + o[6] * f1 + o[9] * f2 + P.mi[3] * f3 + o[12] * f4 + o[13] * f5;
    d.w[1] = o[3] * f0 + o[7] * f1 + o[10] * f2 + o[12] * f3 + P.mi[4] * f4 + o[14] * f5;
    d.w[2] = o[4] * f0 + o[8] * f1 + o[11] * f2 + o[13] * f3 + o[14] * f4 + P.mi[5] * f5;
  }

  // Kinematics: p' = R v; 2 q' = q (x) (0, w).
  d.p[0] = fmaf(R02, v2, fmaf(R01, v1, R00 * v0));
  d.p[1] = fmaf(R12, v2, fmaf(R11, v1, R10 * v0));
  d.p[2] = fmaf(R22, v2, fmaf(R21, v1, R20 * v0));
  d.q[0] = fmaf(-qz, w2, fmaf(-qy, w1, -qx * w0));
  d.q[1] = fmaf(qy, w2, fmaf(-qz, w1, qw * w0));
  d.q[2] = fmaf(-qx, w2, fmaf(qw, w1, qz * w0));
  d.q[3] = fmaf(qw, w2, fmaf(qx, w1, -qy * w0));
}

// y = x + a k, with the quaternion taking a / 2 (its derivative is stored doubled).  WN = false
// leaves the throttle states alone.
template <int MT, bool WN = true>
__device__ __forceinline__ void axpy(St<MT> &y, const St<MT> &x, float a, const St<MT> &k) {
  const float aq = 0.5f * a;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    y.p[i] = fmaf(a, k.p[i], x.p[i]);
    y.v[i] = fmaf(a, k.v[i], x.v[i]);
    y.w[i] = fmaf(a, k.w[i], x.w[i]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) y.q[i] = fmaf(aq, k.q[i], x.q[i]);
  if constexpr (WN) {
#pragma unroll
    for (int i = 0; i < MT; ++i) y.n[i] = fmaf(a, k.n[i], x.n[i]);
  }
}

// The throttle lag n' = (c - n) / tau_m is linear with the command held, so RK4 applied to it has
// closed forms: with g2 = -h / (2 tau_m), g3 = -h / tau_m and b = (h/2) c / tau_m the stage
// values are y2 = n + g2 n + b, y3 = n + g2 y2 + b, y4 = n + g3 y3 + 2 b, and the step gives
// n+ = P n + (1 - P) c with P = 1 + z + z^2/2 + z^3/6 + z^4/24, z = g3 (RK4's stability
// polynomial) — the same numbers as RK4's stage updates and weighted sum, in 6 operations per
// thruster instead of 11.
struct LagEnv {
  float g2, g3, P, lambda, hh;  // lambda = (1 - P) / (g2 tau_m): (1 - P) c = lambda b; hh = h/2
};

__device__ __forceinline__ LagEnv lag_env(float itau, float h) {
  LagEnv L;
  L.hh = 0.5f * h;
  L.g3 = -h * itau;
  L.g2 = 0.5f * L.g3;
  const float z = L.g3;
  L.P = fmaf(fmaf(fmaf(fmaf(z, 1.f / 24.f, 1.f / 6.f), z, 0.5f), z, 1.f), z, 1.f);
  L.lambda = (1.f - L.P) / (L.hh * itau);
  return L;
}

// Per command segment: b_i = (h/2) c_i / tau_m from cs_i = c_i / tau_m.
template <int MT>
__device__ __forceinline__ void lag_segment(const float (&cs)[MT], const LagEnv &L,
                                            float (&b)[MT]) {
#pragma unroll
  for (int i = 0; i < MT; ++i) b[i] = L.hh * cs[i];
}

// One sub-step (§METHOD): classical RK4 of size h, command held (cs = c / tau_m), then
// q <- q / |q|.
template <int MT, bool DIAG, bool MIXED, int NH = 0, bool XH = false>
__device__ __forceinline__ void rk4_step(St<MT> &s, const float (&cs)[MT], const Coef<DIAG> &P,
                                         const float4 *gdir, const float4 *garm, int nt,
                                         bool current_accel, float h,
                                         const float *__restrict__ xh = nullptr) {
  const float hh = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
  St<MT> k, y, acc;
  rhs<MT, DIAG, MIXED, NH, XH>(s, cs, P, gdir, garm, nt, current_accel, k, xh);
  axpy(acc, s, h6, k);
  axpy(y, s, hh, k);
  rhs<MT, DIAG, MIXED, NH, XH>(y, cs, P, gdir, garm, nt, current_accel, k, xh);
  axpy(acc, acc, h3, k);
  axpy(y, s, hh, k);
  rhs<MT, DIAG, MIXED, NH, XH>(y, cs, P, gdir, garm, nt, current_accel, k, xh);
  axpy(acc, acc, h3, k);
  axpy(y, s, h, k);
  rhs<MT, DIAG, MIXED, NH, XH>(y, cs, P, gdir, garm, nt, current_accel, k, xh);
  axpy(s, acc, h6, k);
  const float inv = rsqrtf(fmaf(s.q[0], s.q[0], fmaf(s.q[1], s.q[1],
                                fmaf(s.q[2], s.q[2], s.q[3] * s.q[3]))));
#pragma unroll
  for (int i = 0; i < 4; ++i) s.q[i] *= inv;
}

// One sub-step as rk4_step, with the throttle lag in the closed forms above (b from lag_segment
// for the held command; e = (1 - P) c recovered as lambda b).  Same RK4, different rounding of
// the lag state.
template <int MT, bool DIAG, bool MIXED, int NH = 0, bool XH = false>
__device__ __forceinline__ void rk4_step_lag(St<MT> &s, const float (&b)[MT], const LagEnv &L,
                                             const Coef<DIAG> &P, const float4 *gdir,
                                             const float4 *garm, int nt, bool current_accel,
                                             float h, const float *__restrict__ xh = nullptr) {
  const float hh = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
  St<MT> k, y, acc;
  rhs<MT, DIAG, MIXED, NH, XH, false>(s, b, P, gdir, garm, nt, current_accel, k, xh);
  axpy<MT, false>(acc, s, h6, k);
  axpy<MT, false>(y, s, hh, k);
#pragma unroll
  for (int i = 0; i < MT; ++i) y.n[i] = fmaf(L.g2, s.n[i], s.n[i] + b[i]);
  rhs<MT, DIAG, MIXED, NH, XH, false>(y, b, P, gdir, garm, nt, current_accel, k, xh);
  axpy<MT, false>(acc, acc, h3, k);
  axpy<MT, false>(y, s, hh, k);
#pragma unroll
  for (int i = 0; i < MT; ++i) y.n[i] = fmaf(L.g2, y.n[i], s.n[i] + b[i]);
  rhs<MT, DIAG, MIXED, NH, XH, false>(y, b, P, gdir, garm, nt, current_accel, k, xh);
  axpy<MT, false>(acc, acc, h3, k);
  axpy<MT, false>(y, s, h, k);
#pragma unroll
  for (int i = 0; i < MT; ++i) y.n[i] = fmaf(L.g3, y.n[i], fmaf(2.f, b[i], s.n[i]));
  rhs<MT, DIAG, MIXED, NH, XH, false>(y, b, P, gdir, garm, nt, current_accel, k, xh);
  axpy<MT, false>(s, acc, h6, k);
#pragma unroll
  for (int i = 0; i < MT; ++i) s.n[i] = fmaf(L.P, s.n[i], L.lambda * b[i]);
  const float inv = rsqrtf(fmaf(s.q[0], s.q[0], fmaf(s.q[1], s.q[1],
                                fmaf(s.q[2], s.q[2], s.q[3] * s.q[3]))));
#pragma unroll
  for (int i = 0; i < 4; ++i) s.q[i] *= inv;
}

}  // namespace mg
