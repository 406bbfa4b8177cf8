// Packed step: two vehicles per thread, every operation of the RK4 sub-step issued as one
// FP32x2 instruction (sm_100+ fma/mul/add .f32x2) over the pair.
//
// Device code of the packed step kernel (mg_pair.cu).
//
// A packed FP32x2 FMA is two correctly rounded FMAs: per component it is the same operation as
// fmaf, so evaluating the right-hand side of Eq. 1 (§METHOD) in the order of the scalar rhs()
// (mg_device.cuh) gives every vehicle the same bits as the one-vehicle-per-thread kernels.  The
// FMA pipe has the same throughput either way, but one packed instruction carries two
// vehicles' work through the same dependency latency, so a warp needs half the instructions in
// flight to keep the pipe busy — the sub-step's dependency chains, not the pipe, limit the
// scalar kernel at 65,536 vehicles.
//
// Covered: the diagonal-mass step (r_g = 0, diagonal M_A and D), 6, 8 or mixed thruster
// counts, dense or vectored allocation, current-acceleration term on or off.  A kernel pairs
// two vehicles per thread; when a thread has only one, it passes it twice and stores it once.
#pragma once

#include "mg_advance.cuh"

namespace mg {

// Register budget of the packed kernels: two vehicles' state, parameters and RK4 stages.
constexpr int kRegsPair = 255;

// ---------------------------------------------------------------- packed arithmetic
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 pabs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 psplat(float a) { return make_float2(a, a); }

template <int MT>
struct St2 {
  float2 p[3], q[4], v[3], w[3], n[MT];
};

// The 34 diagonal-mass parameters of ParDiag, one pair per field.  A packed instruction has no
// operand negation, so the parameters the right-hand side only uses negated are stored negated
// (damping, current) and G is kept in both signs; negation is exact, so this changes no bit.
struct Par2 {
  float2 m, ma0, ma1, ma2;
  float2 J0, J1, J2, wb;
  float2 ndl[6], ndq[6];        // -Dl, -Dq
  float2 G0, G1, G2, kT;
  float2 nG0, nG1, nG2;         // -G
  float2 nvc0, nvc1, nvc2, itau;  // -v_c (NED)
  float2 mi[6];
};

__device__ __forceinline__ float2 pk2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ void pack_par(const ParDiag &a, const ParDiag &b, Par2 &P) {
  P.m = pk2(a.m, b.m);
  P.ma0 = pk2(a.ma0, b.ma0); P.ma1 = pk2(a.ma1, b.ma1); P.ma2 = pk2(a.ma2, b.ma2);
  P.J0 = pk2(a.J0, b.J0); P.J1 = pk2(a.J1, b.J1); P.J2 = pk2(a.J2, b.J2);
  P.wb = pk2(a.wb, b.wb);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    P.ndl[i] = pk2(-a.dl[i], -b.dl[i]);
    P.ndq[i] = pk2(-a.dq[i], -b.dq[i]);
    P.mi[i] = pk2(a.mi[i], b.mi[i]);
  }
  P.G0 = pk2(a.G0, b.G0); P.G1 = pk2(a.G1, b.G1); P.G2 = pk2(a.G2, b.G2);
  P.nG0 = pk2(-a.G0, -b.G0); P.nG1 = pk2(-a.G1, -b.G1); P.nG2 = pk2(-a.G2, -b.G2);
  P.kT = pk2(a.kT, b.kT);
  P.nvc0 = pk2(-a.vc0, -b.vc0); P.nvc1 = pk2(-a.vc1, -b.vc1); P.nvc2 = pk2(-a.vc2, -b.vc2);
  P.itau = pk2(a.itau, b.itau);
}

template <int MT>
__device__ __forceinline__ void pack_state(const St<MT> &a, const St<MT> &b, St2<MT> &s) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.p[i] = make_float2(a.p[i], b.p[i]);
    s.v[i] = make_float2(a.v[i], b.v[i]);
    s.w[i] = make_float2(a.w[i], b.w[i]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) s.q[i] = make_float2(a.q[i], b.q[i]);
#pragma unroll
  for (int i = 0; i < MT; ++i) s.n[i] = make_float2(a.n[i], b.n[i]);
}

template <int MT>
__device__ __forceinline__ void unpack_state(const St2<MT> &s, St<MT> &a, St<MT> &b) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    a.p[i] = s.p[i].x; b.p[i] = s.p[i].y;
    a.v[i] = s.v[i].x; b.v[i] = s.v[i].y;
    a.w[i] = s.w[i].x; b.w[i] = s.w[i].y;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a.q[i] = s.q[i].x;
    b.q[i] = s.q[i].y;
  }
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    a.n[i] = s.n[i].x;
    b.n[i] = s.n[i].y;
  }
}

// Thruster geometry of one vehicle type in shared memory, each component duplicated into both
// halves of a pair: g[i] = {d_x, d_y, d_z, (r x d)_x, (r x d)_y, (r x d)_z}.
struct GeoPair {
  float2 g[MG_MAX_THR][6];
};

// Two geometry pairs from shared memory, re-read at every use: an ordinary load of this
// loop-invariant table is hoisted out of the sub-step loop and would hold ~50 registers for the
// whole launch; all lanes read the same address (a broadcast), so the re-reads are cheap.
__device__ __forceinline__ void lds_pairs(const float2 *p, float2 &a, float2 &b) {
  float4 v;
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(s));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}

__device__ __forceinline__ void stage_geo_pair(const Geo &src, GeoPair &dst, int i) {
  const float4 d = src.dir[i], a = src.arm[i];
  dst.g[i][0] = psplat(d.x); dst.g[i][1] = psplat(d.y); dst.g[i][2] = psplat(d.z);
  dst.g[i][3] = psplat(a.x); dst.g[i][4] = psplat(a.y); dst.g[i][5] = psplat(a.z);
}

// ---------------------------------------------------------------- right-hand side, packed
// Operation for operation the diagonal-mass rhs() of mg_device.cuh with LAGD = false (the
// throttle lag is integrated in closed form by the caller), d.q holding 2 q'.
template <int MT, int NH>
__device__ __forceinline__ void rhs2(const St2<MT> &s, const Par2 &P, const GeoPair &G,
                                     bool current_accel, St2<MT> &d) {
  const float2 Z = psplat(0.f), ONE = psplat(1.f);
  // Thrusters: F_i = kT n_i |n_i| along d_i at r_i (kT applied below).
  float2 t0 = Z, t1 = Z, t2 = Z, t3 = Z, t4 = Z, t5 = Z;
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const float2 f = pmul(s.n[i], pabs(s.n[i]));
    float2 g[6];
    if (NH == 0 || i < NH) lds_pairs(&G.g[i][0], g[0], g[1]);
    lds_pairs(&G.g[i][2], g[2], g[3]);
    lds_pairs(&G.g[i][4], g[4], g[5]);
    if (NH == 0) {
      t0 = pfma(f, g[0], t0); t1 = pfma(f, g[1], t1); t2 = pfma(f, g[2], t2);
      t3 = pfma(f, g[3], t3); t4 = pfma(f, g[4], t4); t5 = pfma(f, g[5], t5);
    } else if (i < NH) {
      t0 = pfma(f, g[0], t0); t1 = pfma(f, g[1], t1);
      t3 = pfma(f, g[3], t3); t4 = pfma(f, g[4], t4); t5 = pfma(f, g[5], t5);
    } else {
      t2 = pfma(f, g[2], t2); t3 = pfma(f, g[3], t3); t4 = pfma(f, g[4], t4);
    }
  }

  // R(q) = I + 2 q_w S(eps) + 2 S(eps)^2.
  const float2 qw = s.q[0], qx = s.q[1], qy = s.q[2], qz = s.q[3];
  const float2 nqw = pneg(qw), nqx = pneg(qx), nqy = pneg(qy), nqz = pneg(qz);
  const float2 tx = padd(qx, qx), ty = padd(qy, qy), tz = padd(qz, qz);
  const float2 zdiag = pfma(nqz, tz, ONE);
  const float2 R00 = pfma(nqy, ty, zdiag), R11 = pfma(nqx, tx, zdiag);
  const float2 R22 = pfma(nqx, tx, pfma(nqy, ty, ONE));
  const float2 xy = pmul(qx, ty), xz = pmul(qx, tz), yz = pmul(qy, tz);
  const float2 R01 = pfma(nqw, tz, xy), R10 = pfma(qw, tz, xy);
  const float2 R02 = pfma(qw, ty, xz), R20 = pfma(nqw, ty, xz);
  const float2 R12 = pfma(nqw, tx, yz), R21 = pfma(qw, tx, yz);

  const float2 v0 = s.v[0], v1 = s.v[1], v2 = s.v[2];
  const float2 w0 = s.w[0], w1 = s.w[1], w2 = s.w[2];
  const float2 nw0 = pneg(w0), nw1 = pneg(w1), nw2 = pneg(w2);

  // Current seen from the body (negated: ncb = R^T (-v_c) = -v_c^b), relative velocity.
  const float2 ncb0 = pfma(R20, P.nvc2, pfma(R10, P.nvc1, pmul(R00, P.nvc0)));
  const float2 ncb1 = pfma(R21, P.nvc2, pfma(R11, P.nvc1, pmul(R01, P.nvc0)));
  const float2 ncb2 = pfma(R22, P.nvc2, pfma(R12, P.nvc1, pmul(R02, P.nvc0)));
  const float2 r0 = padd(v0, ncb0), r1 = padd(v1, ncb1), r2 = padd(v2, ncb2);

  // Momenta: Q1 = M_A,lin v_r, h = m v + Q1, k = J w.
  const float2 q0 = pmul(P.ma0, r0), q1 = pmul(P.ma1, r1), q2 = pmul(P.ma2, r2);
  const float2 k0 = pmul(P.J0, w0), k1 = pmul(P.J1, w1), k2 = pmul(P.J2, w2);
  const float2 h0 = pfma(P.m, v0, q0), h1 = pfma(P.m, v1, q1), h2 = pfma(P.m, v2, q2);

  // Translational force.
  float2 f0 = pfma(P.wb, R20, pmul(P.kT, t0));
  float2 f1 = pfma(P.wb, R21, pmul(P.kT, t1));
  float2 f2 = pfma(P.wb, R22, pmul(P.kT, t2));
  f0 = pfma(w2, h1, pfma(nw1, h2, f0));
  f1 = pfma(w0, h2, pfma(nw2, h0, f1));
  f2 = pfma(w1, h0, pfma(nw0, h1, f2));
  f0 = pfma(pfma(P.ndq[0], pabs(r0), P.ndl[0]), r0, f0);
  f1 = pfma(pfma(P.ndq[1], pabs(r1), P.ndl[1]), r1, f1);
  f2 = pfma(pfma(P.ndq[2], pabs(r2), P.ndl[2]), r2, f2);
  if (current_accel) {
    // -c = -(w x v_c^b), from -v_c^b: e.g. -c_0 = -(w1 cb2 - w2 cb1) = w1 ncb2 + (-w2) ncb1.
    const float2 nc0 = pfma(w1, ncb2, pmul(nw2, ncb1));
    const float2 nc1 = pfma(w2, ncb0, pmul(nw0, ncb2));
    const float2 nc2 = pfma(w0, ncb1, pmul(nw1, ncb0));
    f0 = pfma(P.ma0, nc0, f0);
    f1 = pfma(P.ma1, nc1, f1);
    f2 = pfma(P.ma2, nc2, f2);
  }
  // Rotational force.
  float2 f3 = pfma(r2, q1, pfma(pneg(r1), q2, pmul(P.kT, t3)));
  float2 f4 = pfma(r0, q2, pfma(pneg(r2), q0, pmul(P.kT, t4)));
  float2 f5 = pfma(r1, q0, pfma(pneg(r0), q1, pmul(P.kT, t5)));
  f3 = pfma(w2, k1, pfma(nw1, k2, f3));
  f4 = pfma(w0, k2, pfma(nw2, k0, f4));
  f5 = pfma(w1, k0, pfma(nw0, k1, f5));
  f3 = pfma(pfma(P.ndq[3], pabs(w0), P.ndl[3]), w0, f3);
  f4 = pfma(pfma(P.ndq[4], pabs(w1), P.ndl[4]), w1, f4);
  f5 = pfma(pfma(P.ndq[5], pabs(w2), P.ndl[5]), w2, f5);
  f3 = pfma(P.nG2, R21, pfma(P.G1, R22, f3));
  f4 = pfma(P.nG0, R22, pfma(P.G2, R20, f4));
  f5 = pfma(P.nG1, R20, pfma(P.G0, R21, f5));

  // nu' = M^-1 f (diagonal).
  d.v[0] = pmul(P.mi[0], f0); d.v[1] = pmul(P.mi[1], f1); d.v[2] = pmul(P.mi[2], f2);
  d.w[0] = pmul(P.mi[3], f3); d.w[1] = pmul(P.mi[4], f4); d.w[2] = pmul(P.mi[5], f5);

  // Kinematics: p' = R v; 2 q' = q (x) (0, w).
  d.p[0] = pfma(R02, v2, pfma(R01, v1, pmul(R00, v0)));
  d.p[1] = pfma(R12, v2, pfma(R11, v1, pmul(R10, v0)));
  d.p[2] = pfma(R22, v2, pfma(R21, v1, pmul(R20, v0)));
  d.q[0] = pfma(nqz, w2, pfma(nqy, w1, pmul(nqx, w0)));
  d.q[1] = pfma(qy, w2, pfma(nqz, w1, pmul(qw, w0)));
  d.q[2] = pfma(nqx, w2, pfma(qw, w1, pmul(qz, w0)));
  d.q[3] = pfma(qw, w2, pfma(qx, w1, pmul(nqy, w0)));
}

// y = x + a k for p, q (with a / 2), v, w; the throttle states are handled by the caller.
template <int MT>
__device__ __forceinline__ void axpy2(St2<MT> &y, const St2<MT> &x, float a, const St2<MT> &k) {
  const float2 A = psplat(a), AQ = psplat(0.5f * a);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    y.p[i] = pfma(A, k.p[i], x.p[i]);
    y.v[i] = pfma(A, k.v[i], x.v[i]);
    y.w[i] = pfma(A, k.w[i], x.w[i]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) y.q[i] = pfma(AQ, k.q[i], x.q[i]);
}

// Lag constants of a pair (lag_env of each vehicle).
struct Lag2 {
  float2 g2, g3, P, lambda;
  float hh;
};

__device__ __forceinline__ Lag2 lag_pair(float2 itau, float h) {
  const LagEnv a = lag_env(itau.x, h), b = lag_env(itau.y, h);
  Lag2 L;
  L.g2 = make_float2(a.g2, b.g2);
  L.g3 = make_float2(a.g3, b.g3);
  L.P = make_float2(a.P, b.P);
  L.lambda = make_float2(a.lambda, b.lambda);
  L.hh = a.hh;
  return L;
}

// One sub-step: rk4_step_lag of mg_device.cuh on a pair.
template <int MT, int NH>
__device__ __forceinline__ void rk4_step_lag2(St2<MT> &s, const float2 (&b)[MT], const Lag2 &L,
                                              const Par2 &P, const GeoPair &G,
                                              bool current_accel, float h) {
  const float hh = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
  const float2 TWO = psplat(2.f);
  St2<MT> k, y, acc;
  rhs2<MT, NH>(s, P, G, current_accel, k);
  axpy2(acc, s, h6, k);
  axpy2(y, s, hh, k);
#pragma unroll
  for (int i = 0; i < MT; ++i) y.n[i] = pfma(L.g2, s.n[i], padd(s.n[i], b[i]));
  rhs2<MT, NH>(y, P, G, current_accel, k);
  axpy2(acc, acc, h3, k);
  axpy2(y, s, hh, k);
#pragma unroll
  for (int i = 0; i < MT; ++i) y.n[i] = pfma(L.g2, y.n[i], padd(s.n[i], b[i]));
  rhs2<MT, NH>(y, P, G, current_accel, k);
  axpy2(acc, acc, h3, k);
  axpy2(y, s, h, k);
#pragma unroll
  for (int i = 0; i < MT; ++i) y.n[i] = pfma(L.g3, y.n[i], pfma(TWO, b[i], s.n[i]));
  rhs2<MT, NH>(y, P, G, current_accel, k);
  axpy2(s, acc, h6, k);
#pragma unroll
  for (int i = 0; i < MT; ++i) s.n[i] = pfma(L.P, s.n[i], pmul(L.lambda, b[i]));
  const float2 nn = pfma(s.q[0], s.q[0], pfma(s.q[1], s.q[1],
                                              pfma(s.q[2], s.q[2], pmul(s.q[3], s.q[3]))));
  const float2 inv = make_float2(rsqrtf(nn.x), rsqrtf(nn.y));
#pragma unroll
  for (int i = 0; i < 4; ++i) s.q[i] = pmul(s.q[i], inv);
}

// Held command of segment seg for both vehicles, as b = (h/2) c / tau_m (lag_segment).
template <int MT>
__device__ __forceinline__ void pair_commands(const FleetView &fv, int64_t ea, int64_t eb,
                                              int64_t seg, int nt, float2 itau, float hh,
                                              float2 (&b)[MT]) {
  float ca[MT], cb[MT];
  load_commands<MT>(fv, ea, seg, nt, itau.x, ca);
  load_commands<MT>(fv, eb, seg, nt, itau.y, cb);
#pragma unroll
  for (int i = 0; i < MT; ++i) b[i] = make_float2(hh * ca[i], hh * cb[i]);
}

// advance_env for a pair (ea, eb): k sub-steps from action-cursor position step0.
template <int MT, bool L2, int NH>
__device__ __forceinline__ void advance_pair(const FleetView &fv, int64_t ea, int64_t eb, int nt,
                                             const GeoPair &G, int64_t step0, int32_t k,
                                             St<MT> &sa, St<MT> &sb) {
  const bool current_accel = !(fv.model_flags & MG_MODEL_NO_CURRENT_ACCEL);
  const float h = fv.dt;
  St2<MT> s;
  Par2 P;
  {
    load_state<MT, L2>(fv.st, ea, sa);
    load_state<MT, L2>(fv.st, eb, sb);
    pack_state<MT>(sa, sb, s);
    ParDiag pa, pb;
    load_par<true>(fv.pa, ea, pa);
    load_par<true>(fv.pa, eb, pb);
    pack_par(pa, pb, P);
  }
  int64_t seg = step0 / fv.hold;
  int32_t left = fv.hold - (int32_t)(step0 - seg * fv.hold);
  const Lag2 L = lag_pair(P.itau, h);
  float2 b[MT];
  pair_commands<MT>(fv, ea, eb, seg, nt, P.itau, L.hh, b);
  for (int32_t it = 0; it < k; ++it) {
    if (left == 0) {
      ++seg;
      left = fv.hold;
      pair_commands<MT>(fv, ea, eb, seg, nt, P.itau, L.hh, b);
    }
    rk4_step_lag2<MT, NH>(s, b, L, P, G, current_accel, h);
    --left;
  }
  unpack_state<MT>(s, sa, sb);
}

}  // namespace mg
