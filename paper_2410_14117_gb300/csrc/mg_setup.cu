// Set-up kernels, run when parameters or episodes change (not per sub-step):
//   - domain randomisation (§METHOD) from Philox4x32-10 draws, in FP64, stored FP32;
//   - derivation of what the step reads, including M^-1 of the 6x6 mass matrix M_RB + M_A of
//     Eq. 1 by an FP64 Cholesky factorisation (M is symmetric positive definite for any
//     physical vehicle; a non-positive pivot is counted and reported);
//   - episode reset, and conversions between the SoA planes and the record layouts of mg.h.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "mg_device.cuh"

namespace mg {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n) { return (int)((n + kThreads - 1) / kThreads); }

// Index of the j-th of the 27 randomised scalars in the parameter record, in draw order: m,
// I_g (3), M_A (6), D_l (6), D_q (6), W, B (record entries 0..23 in order), then r_b,z, k_T,
// tau_m.  A compile-time function, so that the unrolled draw loop addresses the record in
// registers.
static_assert(MG_P_M == 0 && MG_P_IG == 1 && MG_P_MA == 4 && MG_P_DL == 10 && MG_P_DQ == 16 &&
                  MG_P_W == 22 && MG_P_B == 23 && MG_P_TAU == MG_P_KT + 1,
              "randomised-scalar order assumes the record layout of mg.h");
__host__ __device__ constexpr int rand_idx(int j) {
  return j < 24 ? j : j == 24 ? MG_P_RB + 2 : j == 25 ? MG_P_KT : MG_P_TAU;
}
// Block size of the randomisation kernel: at ~150 registers two or three 128-thread blocks fit
// per SM, where one 256-thread block leaves 65,536 envs 1.7 waves.
constexpr int kRandThreads = 128;
// Background form: 64-thread blocks (two warps, ~10 K registers) striding over the fleet, so
// that one block fits beside a step kernel's resident blocks on every SM.
constexpr int kRandBgThreads = 64;

// derive() for an env whose mass matrix is diagonal (r_g = 0, no off-diagonal added mass): the
// same values derive() stores, without building the 6 x 6 matrices (FP64 runs at a 64th of the
// FP32 rate on this GPU).  I_o = I_g exactly and every off-diagonal entry is +0 when r_g = 0.
__device__ void derive_diag(const SetupView &v, int64_t e, const double *p) {
  const double m = p[MG_P_M];
  const double *ma = p + MG_P_MA;
  const double rg[3] = {p[MG_P_RG], p[MG_P_RG + 1], p[MG_P_RG + 2]};
  double Mjj[6], mi[6];
  bool spd = true;
  for (int i = 0; i < 3; ++i) {
    Mjj[i] = m + ma[i];
    Mjj[3 + i] = p[MG_P_IG + i] + ma[3 + i];
  }
  for (int j = 0; j < 6; ++j) {
    if (!(Mjj[j] > 0.0)) spd = false;
    mi[j] = Mjj[j] > 0.0 ? 1.0 / Mjj[j] : 0.0;
  }
  if (!spd) atomicAdd(v.n_not_spd, 1ull);
  const double W = p[MG_P_W], B = p[MG_P_B];
  const double G[3] = {W * rg[0] - B * p[MG_P_RB], W * rg[1] - B * p[MG_P_RB + 1],
                       W * rg[2] - B * p[MG_P_RB + 2]};
  const ParamPlanes &pa = v.pa;
  auto f = [](double x) { return (float)x; };
  pa.d0[e] = make_float4(f(m), f(ma[0]), f(ma[1]), f(ma[2]));
  pa.d1[e] = make_float4(f(Mjj[3]), f(Mjj[4]), f(Mjj[5]), f(W - B));
  pa.d2[e] = make_float4(f(p[MG_P_DL]), f(p[MG_P_DL + 1]), f(p[MG_P_DL + 2]),
                         f(p[MG_P_DL + 3]));
  pa.d3[e] = make_float4(f(p[MG_P_DL + 4]), f(p[MG_P_DL + 5]), f(p[MG_P_DQ]),
                         f(p[MG_P_DQ + 1]));
  pa.d4[e] = make_float4(f(p[MG_P_DQ + 2]), f(p[MG_P_DQ + 3]), f(p[MG_P_DQ + 4]),
                         f(p[MG_P_DQ + 5]));
  pa.d5[e] = make_float4(f(G[0]), f(G[1]), f(G[2]), f(p[MG_P_KT]));
  pa.d6[e] = make_float4(f(p[MG_P_VC]), f(p[MG_P_VC + 1]), f(p[MG_P_VC + 2]),
                         f(1.0 / p[MG_P_TAU]));
  pa.d7[e] = make_float4(f(mi[0]), f(mi[1]), f(mi[2]), f(mi[3]));
  pa.d8[e] = make_float2(f(mi[4]), f(mi[5]));
  pa.g0[e] = make_float4(f(m * rg[0]), f(m * rg[1]), f(m * rg[2]), 0.f);
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  pa.g1[e] = z;
  pa.g2[e] = z;
  pa.g3[e] = z;
  pa.g4[e] = z;
  pa.g5[e] = 0.f;
}

// Derive the step's parameter planes for env e from its FP64 record p[MG_NPARAM].
__device__ void derive(const SetupView &v, int64_t e, const double *p) {
  const double m = p[MG_P_M];
  const double rg[3] = {p[MG_P_RG], p[MG_P_RG + 1], p[MG_P_RG + 2]};
  const double *ma = p + MG_P_MA;
  const double r2 = rg[0] * rg[0] + rg[1] * rg[1] + rg[2] * rg[2];
  const int64_t xs = v.xh_stride ? v.xh_stride : v.n;
  if (r2 == 0.0) {
    bool xh_zero = true;
    if (v.xh)
      for (int t = 0; t < 15; ++t) xh_zero = xh_zero && v.xh[(int64_t)t * xs + e] == 0.f;
    if (xh_zero) {
      derive_diag(v, e, p);
      return;
    }
  }
  // I_o = I_g - m S(r_g)^2 = I_g + m (|r_g|^2 I - r_g r_g^T)  (inertia about the body origin)
  double Io[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Io[i][j] = (i == j ? p[MG_P_IG + i] + m * r2 : 0.0) - m * rg[i] * rg[j];

  // M = M_RB + M_A = [[m I + Ma_lin, -m S(r_g)], [m S(r_g), I_o + Ma_rot]], plus M_A's
  // off-diagonal entries from the extension (FP32 values, as the step reads them).
  double M[6][6];
  const double S[3][3] = {{0.0, -rg[2], rg[1]}, {rg[2], 0.0, -rg[0]}, {-rg[1], rg[0], 0.0}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      M[i][j] = (i == j) ? m + ma[i] : 0.0;
      M[i][3 + j] = -m * S[i][j];
      M[3 + i][j] = m * S[i][j];
      M[3 + i][3 + j] = Io[i][j] + ((i == j) ? ma[3 + i] : 0.0);
    }
  bool ma_off = false;
  if (v.xh) {
    int t = 0;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j, ++t) {
        const double a = (double)v.xh[(int64_t)t * xs + e];
        M[i][j] += a;
        M[j][i] += a;
        ma_off = ma_off || a != 0.0;
      }
  }

  // Cholesky M = L L^T; L^-1 by forward substitution; M^-1 = L^-T L^-1.  With r_g = 0 the
  // matrix is diagonal (diagonal M_A), its factor is diag(sqrt(M_jj)) and the inverse 1 / M_jj.
  double L[6][6] = {}, Li[6][6] = {}, Mi[6][6] = {};
  bool spd = true;
  const bool diagonal = (r2 == 0.0) && !ma_off;
  if (diagonal) {
    for (int j = 0; j < 6; ++j) {
      if (!(M[j][j] > 0.0)) spd = false;
      Mi[j][j] = M[j][j] > 0.0 ? 1.0 / M[j][j] : 0.0;
    }
  }
  for (int j = 0; j < 6 && !diagonal; ++j) {
    double d = M[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) {
      spd = false;
      d = 1.0;
    }
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < 6; ++i) {
      double s = M[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / L[j][j];
    }
  }
  for (int j = 0; j < 6 && !diagonal; ++j) {
    Li[j][j] = 1.0 / L[j][j];
    for (int i = j + 1; i < 6; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += L[i][k] * Li[k][j];
      Li[i][j] = -s / L[i][i];
    }
  }
  for (int i = 0; i < 6 && !diagonal; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int k = (i > j ? i : j); k < 6; ++k) s += Li[k][i] * Li[k][j];
      Mi[i][j] = s;
    }
  if (!spd) atomicAdd(v.n_not_spd, 1ull);
  if (!diagonal) atomicOr(v.any_offdiag, 1u);

  const double W = p[MG_P_W], B = p[MG_P_B];
  const double G[3] = {W * rg[0] - B * p[MG_P_RB], W * rg[1] - B * p[MG_P_RB + 1],
                       W * rg[2] - B * p[MG_P_RB + 2]};
  const ParamPlanes &pa = v.pa;
  auto f = [](double x) { return (float)x; };
  pa.d0[e] = make_float4(f(m), f(ma[0]), f(ma[1]), f(ma[2]));
  pa.d1[e] = make_float4(f(Io[0][0] + ma[3]), f(Io[1][1] + ma[4]), f(Io[2][2] + ma[5]),
                         f(W - B));
  pa.d2[e] = make_float4(f(p[MG_P_DL]), f(p[MG_P_DL + 1]), f(p[MG_P_DL + 2]),
                         f(p[MG_P_DL + 3]));
  pa.d3[e] = make_float4(f(p[MG_P_DL + 4]), f(p[MG_P_DL + 5]), f(p[MG_P_DQ]),
                         f(p[MG_P_DQ + 1]));
  pa.d4[e] = make_float4(f(p[MG_P_DQ + 2]), f(p[MG_P_DQ + 3]), f(p[MG_P_DQ + 4]),
                         f(p[MG_P_DQ + 5]));
  pa.d5[e] = make_float4(f(G[0]), f(G[1]), f(G[2]), f(p[MG_P_KT]));
  pa.d6[e] = make_float4(f(p[MG_P_VC]), f(p[MG_P_VC + 1]), f(p[MG_P_VC + 2]),
                         f(1.0 / p[MG_P_TAU]));
  pa.d7[e] = make_float4(f(Mi[0][0]), f(Mi[1][1]), f(Mi[2][2]), f(Mi[3][3]));
  pa.d8[e] = make_float2(f(Mi[4][4]), f(Mi[5][5]));
  pa.g0[e] = make_float4(f(m * rg[0]), f(m * rg[1]), f(m * rg[2]), f(Io[0][1]));
  pa.g1[e] = make_float4(f(Io[0][2]), f(Io[1][2]), f(Mi[0][1]), f(Mi[0][2]));
  pa.g2[e] = make_float4(f(Mi[0][3]), f(Mi[0][4]), f(Mi[0][5]), f(Mi[1][2]));
  pa.g3[e] = make_float4(f(Mi[1][3]), f(Mi[1][4]), f(Mi[1][5]), f(Mi[2][3]));
  pa.g4[e] = make_float4(f(Mi[2][4]), f(Mi[2][5]), f(Mi[3][4]), f(Mi[3][5]));
  pa.g5[e] = f(Mi[4][5]);
}

__device__ __forceinline__ void randomize_env(const SetupView &v, const float *__restrict__ nominal,
                                              uint64_t seed, double lo, double hi,
                                              double current_sigma, double rg_halfwidth,
                                              int64_t e) {
  const uint64_t gid = (uint64_t)(v.gid0 + e);
  const float *nom = nominal + (int64_t)v.types[e] * MG_NPARAM;
  double p[MG_NPARAM];
  for (int j = 0; j < MG_NPARAM; ++j) p[j] = (double)nom[j];
  uint4 x = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int j = 0; j < 27; ++j) {
    if (j % 4 == 0) x = draw4(seed, gid, STREAM_PARAMS, (uint32_t)(j / 4));
    const uint32_t w = (j % 4 == 0) ? x.x : (j % 4 == 1) ? x.y : (j % 4 == 2) ? x.z : x.w;
    const int idx = rand_idx(j);
    p[idx] = (double)nom[idx] * (lo + (hi - lo) * u01d(w));
  }
  const uint4 c = draw4(seed, gid, STREAM_CURRENT, 0u);
  double z0, z1, z2, z3;
  box_muller(u01d(c.x), u01d(c.y), z0, z1);
  box_muller(u01d(c.z), u01d(c.w), z2, z3);
  p[MG_P_VC] += current_sigma * z0;
  p[MG_P_VC + 1] += current_sigma * z1;
  p[MG_P_VC + 2] += current_sigma * z2;
  if (rg_halfwidth > 0.0) {  // off-centre gravity: nominal + U[-w, w] per axis
    const uint4 r = draw4(seed, gid, STREAM_PARAMS, 7u);
    p[MG_P_RG] += rg_halfwidth * (2.0 * u01d(r.x) - 1.0);
    p[MG_P_RG + 1] += rg_halfwidth * (2.0 * u01d(r.y) - 1.0);
    p[MG_P_RG + 2] += rg_halfwidth * (2.0 * u01d(r.z) - 1.0);
  }
  // Store FP32; derive from the stored values so that everything the step reads is consistent
  // with what mg_get_params reports.
  for (int j = 0; j < MG_NPARAM; ++j) {
    const float f = (float)p[j];
    v.raw[e * MG_NPARAM + j] = f;
    p[j] = (double)f;
  }
  derive(v, e, p);
}

// One env per thread.
__global__ void __launch_bounds__(kRandThreads)
    k_randomize(const SetupView v, const float *__restrict__ nominal, uint64_t seed,
                            double lo, double hi, double current_sigma, double rg_halfwidth) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < v.n) randomize_env(v, nominal, seed, lo, hi, current_sigma, rg_halfwidth, e);
}

// Background form: a grid smaller than the fleet strides over it, leaving room on every SM for
// a step kernel running concurrently on another stream.  Same per-env arithmetic.
__global__ void __launch_bounds__(kRandBgThreads)
    k_randomize_bg(const SetupView v, const float *__restrict__ nominal, uint64_t seed,
                   double lo, double hi, double current_sigma, double rg_halfwidth) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < v.n; e += stride)
    randomize_env(v, nominal, seed, lo, hi, current_sigma, rg_halfwidth, e);
}

__global__ void k_import_params(const SetupView v, const float *__restrict__ in) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= v.n) return;
  double p[MG_NPARAM];
  for (int j = 0; j < MG_NPARAM; ++j) {
    const float f = in[e * MG_NPARAM + j];
    v.raw[e * MG_NPARAM + j] = f;
    p[j] = (double)f;
  }
  derive(v, e, p);
}

// Off-diagonal hydrodynamics between the record layout [n][MG_NXPARAM] and the planes
// [MG_NXPARAM][n] the step reads (to_planes), or back.
__global__ void k_xh_transpose(const float *__restrict__ in, float *__restrict__ out, int64_t n,
                               bool to_planes, int64_t stride) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  for (int c = 0; c < MG_NXPARAM; ++c) {
    if (to_planes)
      out[(int64_t)c * stride + e] = in[e * MG_NXPARAM + c];
    else
      out[e * MG_NXPARAM + c] = in[(int64_t)c * stride + e];
  }
}

__global__ void k_export_params(const SetupView v, float *__restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= v.n) return;
  for (int j = 0; j < MG_NPARAM; ++j) out[e * MG_NPARAM + j] = v.raw[e * MG_NPARAM + j];
}

__global__ void k_reset(const StatePlanes st, int64_t n, int64_t gid0,
                        const uint8_t *__restrict__ mask, uint64_t seed, double sigma,
                        uint32_t *__restrict__ episode, uint32_t *__restrict__ flags,
                        unsigned long long *nonfinite_count) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n || (mask && !mask[e])) return;
  reset_env(st, e, (uint64_t)(gid0 + e), seed, sigma, episode, flags, nonfinite_count);
}

// State rows ([n][MG_NSTATE], 84 B each) <-> planes, staged through shared memory so that a
// block's rows move as one contiguous span (16-byte vectors when the row buffer is 16-byte
// aligned: a block's span starts at a multiple of kRowThreads x 84 B = 10,752 B).
constexpr int kRowThreads = 128;

__device__ __forceinline__ bool aligned16(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

__global__ void __launch_bounds__(kRowThreads)
    k_export_state(const StatePlanes st, int64_t n, float *__restrict__ out) {
  __shared__ __align__(16) float rows[kRowThreads * MG_NSTATE];
  const int64_t e0 = (int64_t)blockIdx.x * kRowThreads;
  const int t = (int)threadIdx.x;
  const int64_t e = e0 + t;
  if (e < n) {
    const float4 a = st.s0[e], b = st.s1[e], c = st.s2[e], d = st.s3[e], f = st.s4[e];
    const float r[MG_NSTATE] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z,
                                c.w, d.x, d.y, d.z, d.w, f.x, f.y, f.z, f.w, st.s5[e]};
#pragma unroll
    for (int j = 0; j < MG_NSTATE; ++j) rows[t * MG_NSTATE + j] = r[j];
  }
  __syncthreads();
  const int total = (int)(n - e0 < kRowThreads ? n - e0 : kRowThreads) * MG_NSTATE;
  float *o = out + e0 * MG_NSTATE;
  int done = 0;
  if (aligned16(out)) {
    done = total & ~3;
    float4 *o4 = reinterpret_cast<float4 *>(o);
    const float4 *r4 = reinterpret_cast<const float4 *>(rows);
    for (int i = t; i < done / 4; i += kRowThreads) o4[i] = r4[i];
  }
  for (int i = done + t; i < total; i += kRowThreads) o[i] = rows[i];
}

__global__ void __launch_bounds__(kRowThreads)
    k_import_state(const StatePlanes st, int64_t n, const float *__restrict__ in) {
  __shared__ __align__(16) float rows[kRowThreads * MG_NSTATE];
  const int64_t e0 = (int64_t)blockIdx.x * kRowThreads;
  const int t = (int)threadIdx.x;
  const int total = (int)(n - e0 < kRowThreads ? n - e0 : kRowThreads) * MG_NSTATE;
  const float *src = in + e0 * MG_NSTATE;
  int done = 0;
  if (aligned16(in)) {
    done = total & ~3;
    const float4 *i4 = reinterpret_cast<const float4 *>(src);
    float4 *r4 = reinterpret_cast<float4 *>(rows);
    for (int i = t; i < done / 4; i += kRowThreads) r4[i] = i4[i];
  }
  for (int i = done + t; i < total; i += kRowThreads) rows[i] = src[i];
  __syncthreads();
  const int64_t e = e0 + t;
  if (e >= n) return;
  const float *r = rows + t * MG_NSTATE;
  st.s0[e] = make_float4(r[0], r[1], r[2], r[3]);
  st.s1[e] = make_float4(r[4], r[5], r[6], r[7]);
  st.s2[e] = make_float4(r[8], r[9], r[10], r[11]);
  st.s3[e] = make_float4(r[12], r[13], r[14], r[15]);
  st.s4[e] = make_float4(r[16], r[17], r[18], r[19]);
  st.s5[e] = r[20];
}

__global__ void k_flags_to_bytes(const uint32_t *__restrict__ flags, int64_t n,
                                 uint8_t *__restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = (uint8_t)(flags[e] & 1u);
}

__global__ void k_philox(const uint32_t *__restrict__ ctr, const uint32_t *__restrict__ key,
                         uint32_t *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox4x32_10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2],
                                           ctr[4 * i + 3]),
                                make_uint2(key[2 * i], key[2 * i + 1]));
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

}  // namespace

cudaError_t launch_randomize(const SetupView &v, const float *nominal, uint64_t seed, double lo,
                             double hi, double current_sigma, double rg_halfwidth,
                             cudaStream_t stream, int background_blocks) {
  if (background_blocks > 0) {
    const int64_t full = (v.n + kRandBgThreads - 1) / kRandBgThreads;
    const int blocks = (int)std::min<int64_t>(full, background_blocks);
    k_randomize_bg<<<blocks, kRandBgThreads, 0, stream>>>(v, nominal, seed, lo, hi,
                                                          current_sigma, rg_halfwidth);
  } else {
    k_randomize<<<(int)((v.n + kRandThreads - 1) / kRandThreads), kRandThreads, 0, stream>>>(
        v, nominal, seed, lo, hi, current_sigma, rg_halfwidth);
  }
  return cudaGetLastError();
}

cudaError_t launch_xh_transpose(const float *in, float *out, int64_t n, bool to_planes,
                                cudaStream_t stream, int64_t stride) {
  if (stride < n) stride = n;
  k_xh_transpose<<<blocks_for(n), kThreads, 0, stream>>>(in, out, n, to_planes, stride);
  return cudaGetLastError();
}

cudaError_t launch_import_params(const SetupView &v, const float *in, cudaStream_t stream) {
  k_import_params<<<blocks_for(v.n), kThreads, 0, stream>>>(v, in);
  return cudaGetLastError();
}

cudaError_t launch_export_params(const SetupView &v, float *out, cudaStream_t stream) {
  k_export_params<<<blocks_for(v.n), kThreads, 0, stream>>>(v, out);
  return cudaGetLastError();
}

cudaError_t launch_reset(const StatePlanes &st, int64_t n, int64_t gid0, const uint8_t *mask,
                         uint64_t seed, double nu0_sigma, uint32_t *episode, uint32_t *flags,
                         unsigned long long *nonfinite_count, cudaStream_t stream) {
  k_reset<<<blocks_for(n), kThreads, 0, stream>>>(st, n, gid0, mask, seed, nu0_sigma, episode,
                                                  flags, nonfinite_count);
  return cudaGetLastError();
}

cudaError_t launch_export_state(const StatePlanes &st, int64_t n, float *out,
                                cudaStream_t stream) {
  k_export_state<<<(int)((n + kRowThreads - 1) / kRowThreads), kRowThreads, 0, stream>>>(st, n,
                                                                                      out);
  return cudaGetLastError();
}

cudaError_t launch_import_state(const StatePlanes &st, int64_t n, const float *in,
                                cudaStream_t stream) {
  k_import_state<<<(int)((n + kRowThreads - 1) / kRowThreads), kRowThreads, 0, stream>>>(st, n,
                                                                                      in);
  return cudaGetLastError();
}

cudaError_t launch_flags_to_bytes(const uint32_t *flags, int64_t n, uint8_t *out,
                                  cudaStream_t stream) {
  k_flags_to_bytes<<<blocks_for(n), kThreads, 0, stream>>>(flags, n, out);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                          cudaStream_t stream) {
  k_philox<<<blocks_for(n), kThreads, 0, stream>>>(ctr, key, out, n);
  return cudaGetLastError();
}

}  // namespace mg
