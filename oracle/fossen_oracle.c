/*
 * FP64 CPU oracle for the MarineGym vehicle step — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load this
 * library.  The product path (the CUDA library and its Python binding) never calls it and
 * shares no code with it.
 *
 * What it computes (§METHOD, Eq. 1 and the symbol list after it): the extended Fossen equation
 *
 *   tau = M_RB nu' + C_RB(nu) nu + g_RB(eta) + M_A nu' + C_A(nu) nu + D(nu) nu + g_A(eta)
 *
 * with eta the pose in NED and nu = (u,v,w,p,q,r) the body-frame velocity.  Readings of the
 * points the paper leaves open (all fixed once here and listed in the design notes):
 *   - attitude is a unit quaternion q = (w,x,y,z), Hamilton, body -> NED; the pose's Euler angles
 *     are only used by tests;
 *   - added-mass Coriolis and damping act on the velocity relative to a current that is constant
 *     in NED (nu_r = nu - [R^T v_c; 0]); with no current this is Eq. 1 exactly;
 *   - since nu_r' = nu' + [omega x v_c^b; 0] for such a current, the added-mass inertia term adds
 *     M_A [omega x v_c^b; 0] (switchable, flag ORC_NO_CURRENT_ACCEL);
 *   - tau comes from thrusters: F_i = k_T n_i |n_i| along unit direction d_i at position r_i, the
 *     throttle state n_i following the commanded throttle c_i (Eq. 3) with first-order lag tau_m;
 *   - one sub-step (§METHOD, "multiple sub-simulation steps") is one classical RK4 step of size
 *     h with the command held over the step, the attitude quaternion renormalised after the step.
 *
 * Plain on purpose: explicit 6x6 matrices, a general LU solve with partial pivoting, no blocking
 * or fusion.  The restoring vector is built from the weight and buoyancy forces rotated into the
 * body frame, the Coriolis matrices from Fossen's momentum-block parametrisation.
 *
 * Flat layouts: parameters [ORC_NPARAM], state [ORC_NSTATE], geometry [ORC_NGEO] — see the enum
 * below.  All arrays are row-major FP64.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
  P_M = 0, P_IG = 1, P_MA = 4, P_DL = 10, P_DQ = 16, P_W = 22, P_B = 23,
  P_RG = 24, P_RB = 27, P_KT = 30, P_TAU = 31, P_VC = 32, ORC_NPARAM = 35
};
enum { ORC_MAXTHR = 8, ORC_NGEO = 1 + 6 * ORC_MAXTHR, ORC_NSTATE = 21 };
enum { S_P = 0, S_Q = 3, S_NU = 7, S_N = 13 };
enum { ORC_NO_CURRENT_ACCEL = 1 };
/* Off-diagonal hydrodynamic extension (per env, optional): X_MA the 15 entries of M_A above its
 * diagonal, row-major ((0,1), (0,2), ..., (4,5)), mirrored below it; X_DL the 30 off-diagonal
 * entries of the linear damping D_l, row-major with the diagonal skipped.  The diagonals stay in
 * the parameter record; an all-zero extension is the diagonal model. */
enum { X_MA = 0, X_DL = 15, ORC_NXPARAM = 45 };

/* ------------------------------------------------------------------ small linear algebra */

/* S(a) with S(a) b = a x b. */
static void skew(const double a[3], double S[3][3]) {
  S[0][0] = 0.0;   S[0][1] = -a[2]; S[0][2] = a[1];
  S[1][0] = a[2];  S[1][1] = 0.0;   S[1][2] = -a[0];
  S[2][0] = -a[1]; S[2][1] = a[0];  S[2][2] = 0.0;
}

static void mat3_mul(const double A[3][3], const double B[3][3], double C[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
      C[i][j] = s;
    }
}

static void mat3_vec(const double A[3][3], const double x[3], double y[3]) {
  for (int i = 0; i < 3; ++i) y[i] = A[i][0] * x[0] + A[i][1] * x[1] + A[i][2] * x[2];
}

static void mat3T_vec(const double A[3][3], const double x[3], double y[3]) {
  for (int i = 0; i < 3; ++i) y[i] = A[0][i] * x[0] + A[1][i] * x[1] + A[2][i] * x[2];
}

static void mat6_vec(const double A[6][6], const double x[6], double y[6]) {
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
    for (int j = 0; j < 6; ++j) s += A[i][j] * x[j];
    y[i] = s;
  }
}

static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Solve A x = b (6x6) by Gaussian elimination with partial pivoting.  Returns 0, or -1 when a
 * pivot is exactly zero. */
static int solve6(const double Ain[6][6], const double bin[6], double x[6]) {
  double A[6][6], b[6];
  memcpy(A, Ain, sizeof A);
  memcpy(b, bin, sizeof b);
  for (int k = 0; k < 6; ++k) {
    int piv = k;
    for (int i = k + 1; i < 6; ++i)
      if (fabs(A[i][k]) > fabs(A[piv][k])) piv = i;
    if (A[piv][k] == 0.0) return -1;
    if (piv != k) {
      for (int j = 0; j < 6; ++j) { double t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t; }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < 6; ++i) {
      double f = A[i][k] / A[k][k];
      for (int j = k; j < 6; ++j) A[i][j] -= f * A[k][j];
      b[i] -= f * b[k];
    }
  }
  for (int i = 5; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < 6; ++j) s -= A[i][j] * x[j];
    x[i] = s / A[i][i];
  }
  return 0;
}

/* ------------------------------------------------------------------ model terms (Eq. 1) */

/* Attitude matrix R(q), body -> NED, from the quaternion (eta, eps):
 * R = I + 2 eta S(eps) + 2 S(eps)^2 (Fossen's Euler-parameter form).  Evaluated as written for
 * any q, unit or not. */
void orc_rotation(const double q[4], double R[9]) {
  double eps[3] = {q[1], q[2], q[3]}, S[3][3], S2[3][3];
  skew(eps, S);
  mat3_mul(S, S, S2);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      R[3 * i + j] = (i == j ? 1.0 : 0.0) + 2.0 * q[0] * S[i][j] + 2.0 * S2[i][j];
}

/* Rigid-body inertia M_RB about the body origin (Eq. 1, first term): mass m, inertia I_g about
 * the centre of gravity r_g (parallel-axis shift to the origin). */
void orc_mass_rb(const double *par, double M[36]) {
  double m = par[P_M], rg[3] = {par[P_RG], par[P_RG + 1], par[P_RG + 2]};
  double S[3][3], S2[3][3];
  skew(rg, S);
  mat3_mul(S, S, S2);
  memset(M, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i) {
    M[6 * i + i] = m;
    for (int j = 0; j < 3; ++j) {
      M[6 * i + (3 + j)] = -m * S[i][j];
      M[6 * (3 + i) + j] = m * S[i][j];
      double Ig = (i == j) ? par[P_IG + i] : 0.0;
      M[6 * (3 + i) + (3 + j)] = Ig - m * S2[i][j];
    }
  }
}

/* Added mass M_A (Eq. 1, hydrodynamic term): the diagonal from the parameter record, the
 * symmetric off-diagonal part from the extension x (NULL: none). */
void orc_mass_a_x(const double *par, const double *x, double M[36]) {
  memset(M, 0, 36 * sizeof(double));
  for (int i = 0; i < 6; ++i) M[6 * i + i] = par[P_MA + i];
  if (!x) return;
  int t = X_MA;
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      M[6 * i + j] = x[t];
      M[6 * j + i] = x[t];
      ++t;
    }
}

void orc_mass_a(const double *par, double M[36]) { orc_mass_a_x(par, NULL, M); }

/* Coriolis-centripetal matrix of a 6x6 inertia M evaluated at velocity x, in the momentum-block
 * form  C(x) = [[0, -S(M11 x1 + M12 x2)], [-S(M11 x1 + M12 x2), -S(M21 x1 + M22 x2)]]. */
static void coriolis_of(const double M[36], const double x[6], double C[36]) {
  double a1[3], a2[3];
  for (int i = 0; i < 3; ++i) {
    a1[i] = 0.0;
    a2[i] = 0.0;
    for (int j = 0; j < 6; ++j) {
      a1[i] += M[6 * i + j] * x[j];
      a2[i] += M[6 * (3 + i) + j] * x[j];
    }
  }
  double S1[3][3], S2[3][3];
  skew(a1, S1);
  skew(a2, S2);
  memset(C, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      C[6 * i + (3 + j)] = -S1[i][j];
      C[6 * (3 + i) + j] = -S1[i][j];
      C[6 * (3 + i) + (3 + j)] = -S2[i][j];
    }
}

/* C_RB(nu) (Eq. 1). */
void orc_coriolis_rb(const double *par, const double nu[6], double C[36]) {
  double M[36];
  orc_mass_rb(par, M);
  coriolis_of(M, nu, C);
}

/* C_A(nu_r) (Eq. 1), evaluated on the current-relative velocity. */
void orc_coriolis_a_x(const double *par, const double *x, const double nu_r[6], double C[36]) {
  double M[36];
  orc_mass_a_x(par, x, M);
  coriolis_of(M, nu_r, C);
}

void orc_coriolis_a(const double *par, const double nu_r[6], double C[36]) {
  orc_coriolis_a_x(par, NULL, nu_r, C);
}

/* D(nu_r) (Eq. 1): linear plus quadratic damping, D = D_l + diag(Dq |nu_r|), with D_l's
 * diagonal from the parameter record and its off-diagonal entries from the extension x (NULL:
 * none). */
void orc_damping_x(const double *par, const double *x, const double nu_r[6], double D[36]) {
  memset(D, 0, 36 * sizeof(double));
  for (int i = 0; i < 6; ++i) D[6 * i + i] = par[P_DL + i] + par[P_DQ + i] * fabs(nu_r[i]);
  if (!x) return;
  int t = X_DL;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j)
      if (j != i) D[6 * i + j] = x[t++];
}

void orc_damping(const double *par, const double nu_r[6], double D[36]) {
  orc_damping_x(par, NULL, nu_r, D);
}

/* Restoring vector g_RB(eta) + g_A(eta) (Eq. 1): weight W acts down (+z NED) at r_g, buoyancy B
 * acts up at r_b; both rotated into the body frame by R(q)^T; g is minus the generalised force. */
void orc_restoring(const double *par, const double q[4], double g[6]) {
  double Rf[9], R[3][3];
  orc_rotation(q, Rf);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = Rf[3 * i + j];
  double fgn[3] = {0.0, 0.0, par[P_W]}, fbn[3] = {0.0, 0.0, -par[P_B]};
  double fg[3], fb[3];
  mat3T_vec(R, fgn, fg);
  mat3T_vec(R, fbn, fb);
  double rg[3] = {par[P_RG], par[P_RG + 1], par[P_RG + 2]};
  double rb[3] = {par[P_RB], par[P_RB + 1], par[P_RB + 2]};
  double mg[3], mb[3];
  cross3(rg, fg, mg);
  cross3(rb, fb, mb);
  for (int i = 0; i < 3; ++i) {
    g[i] = -(fg[i] + fb[i]);
    g[3 + i] = -(mg[i] + mb[i]);
  }
}

/* Thruster wrench (the tau of Eq. 1 from the throttle actions of Eq. 3): thruster i pushes with
 * F_i = k_T n_i |n_i| along d_i from r_i. */
void orc_thrust(const double *par, const double *geo, const double *n, double tau[6]) {
  int nthr = (int)geo[0];
  const double *r = geo + 1, *d = geo + 1 + 3 * ORC_MAXTHR;
  for (int i = 0; i < 6; ++i) tau[i] = 0.0;
  for (int i = 0; i < nthr; ++i) {
    double F = par[P_KT] * n[i] * fabs(n[i]);
    double f[3] = {F * d[3 * i], F * d[3 * i + 1], F * d[3 * i + 2]}, mo[3];
    cross3(r + 3 * i, f, mo);
    for (int k = 0; k < 3; ++k) {
      tau[k] += f[k];
      tau[3 + k] += mo[k];
    }
  }
}

/* State derivative f(s; c).  s = (p, q, nu, n); x: the off-diagonal extension or NULL.
 * Returns 0, or -1 if M is singular. */
int orc_rhs_x(const double *par, const double *x, const double *geo, const double *s,
              const double *c, int flags, double *ds) {
  const double *q = s + S_Q, *nu = s + S_NU, *n = s + S_N;
  int nthr = (int)geo[0];
  double Rf[9], R[3][3];
  orc_rotation(q, Rf);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = Rf[3 * i + j];

  /* current, constant in NED, seen in the body frame; relative velocity */
  double vcn[3] = {par[P_VC], par[P_VC + 1], par[P_VC + 2]}, vcb[3];
  mat3T_vec(R, vcn, vcb);
  double nu_r[6];
  for (int i = 0; i < 3; ++i) {
    nu_r[i] = nu[i] - vcb[i];
    nu_r[3 + i] = nu[3 + i];
  }

  double Mrb[36], Ma[36], Crb[36], Ca[36], D[36], g[6], tau[6];
  orc_mass_rb(par, Mrb);
  orc_mass_a_x(par, x, Ma);
  orc_coriolis_rb(par, nu, Crb);
  orc_coriolis_a_x(par, x, nu_r, Ca);
  orc_damping_x(par, x, nu_r, D);
  orc_restoring(par, q, g);
  orc_thrust(par, geo, n, tau);

  double crb[6], ca[6], dd[6];
  mat6_vec((const double(*)[6])Crb, nu, crb);
  mat6_vec((const double(*)[6])Ca, nu_r, ca);
  mat6_vec((const double(*)[6])D, nu_r, dd);

  /* added-mass inertia of the current: M_A (nu_r' - nu') = M_A [omega x v_c^b; 0] */
  double ac[6] = {0, 0, 0, 0, 0, 0};
  if (!(flags & ORC_NO_CURRENT_ACCEL)) {
    double wx[6] = {0, 0, 0, 0, 0, 0};
    cross3(nu + 3, vcb, wx);
    mat6_vec((const double(*)[6])Ma, wx, ac);
  }

  double M[6][6], rhs[6], nudot[6];
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j) M[i][j] = Mrb[6 * i + j] + Ma[6 * i + j];
    rhs[i] = tau[i] - crb[i] - ca[i] - dd[i] - g[i] - ac[i];
  }
  if (solve6((const double(*)[6])M, rhs, nudot) != 0) return -1;

  /* kinematics: p' = R(q) v, q' = T(q) omega with T(q) = 1/2 [-eps^T; eta I + S(eps)] */
  double pd[3];
  mat3_vec((const double(*)[3])R, nu, pd);
  double eta = q[0], eps[3] = {q[1], q[2], q[3]}, Se[3][3];
  skew(eps, Se);
  double qd[4];
  qd[0] = -0.5 * (eps[0] * nu[3] + eps[1] * nu[4] + eps[2] * nu[5]);
  for (int i = 0; i < 3; ++i) {
    double t = eta * nu[3 + i];
    for (int j = 0; j < 3; ++j) t += Se[i][j] * nu[3 + j];
    qd[1 + i] = 0.5 * t;
  }

  for (int i = 0; i < 3; ++i) ds[S_P + i] = pd[i];
  for (int i = 0; i < 4; ++i) ds[S_Q + i] = qd[i];
  for (int i = 0; i < 6; ++i) ds[S_NU + i] = nudot[i];
  /* first-order throttle lag n' = (c - n) / tau_m */
  for (int i = 0; i < ORC_MAXTHR; ++i)
    ds[S_N + i] = (i < nthr) ? (c[i] - n[i]) / par[P_TAU] : 0.0;
  return 0;
}

int orc_rhs(const double *par, const double *geo, const double *s, const double *c, int flags,
            double *ds) {
  return orc_rhs_x(par, NULL, geo, s, c, flags, ds);
}

/* One sub-step: classical RK4 of size h with the command held, then q <- q / |q|. */
int orc_rk4_step_x(const double *par, const double *x, const double *geo, const double *s,
                   const double *c, double h, int flags, double *out) {
  double k1[ORC_NSTATE], k2[ORC_NSTATE], k3[ORC_NSTATE], k4[ORC_NSTATE], y[ORC_NSTATE];
  int err = 0;
  err |= orc_rhs_x(par, x, geo, s, c, flags, k1);
  for (int i = 0; i < ORC_NSTATE; ++i) y[i] = s[i] + 0.5 * h * k1[i];
  err |= orc_rhs_x(par, x, geo, y, c, flags, k2);
  for (int i = 0; i < ORC_NSTATE; ++i) y[i] = s[i] + 0.5 * h * k2[i];
  err |= orc_rhs_x(par, x, geo, y, c, flags, k3);
  for (int i = 0; i < ORC_NSTATE; ++i) y[i] = s[i] + h * k3[i];
  err |= orc_rhs_x(par, x, geo, y, c, flags, k4);
  for (int i = 0; i < ORC_NSTATE; ++i)
    out[i] = s[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  double nq = sqrt(out[S_Q] * out[S_Q] + out[S_Q + 1] * out[S_Q + 1] +
                   out[S_Q + 2] * out[S_Q + 2] + out[S_Q + 3] * out[S_Q + 3]);
  for (int i = 0; i < 4; ++i) out[S_Q + i] /= nq;
  return err;
}

int orc_rk4_step(const double *par, const double *geo, const double *s, const double *c,
                 double h, int flags, double *out) {
  return orc_rk4_step_x(par, NULL, geo, s, c, h, flags, out);
}

/* Fleet rollout.  For env e and step j (0-based), the command is cmd[seg][e][*] with
 * seg = min(j / hold, n_seg - 1).  par [n][NPARAM], types [n] index geo [n_types][NGEO],
 * s [n][NSTATE] is advanced in place; traj, if not NULL, receives the state after every step,
 * [n_steps][n][NSTATE].  nthreads <= 0 keeps the OpenMP default.  Returns the number of envs
 * whose solve failed. */
int64_t orc_rollout_x(int64_t n, const double *par, const double *xpar /*[n][NXPARAM] or NULL*/,
                      const double *geo, const int32_t *types, double *s, const double *cmd,
                      int32_t n_seg, int32_t hold, int32_t n_steps, double h, int32_t flags,
                      double *traj, int32_t nthreads) {
  int64_t fails = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : fails)
#endif
  for (int64_t e = 0; e < n; ++e) {
    const double *pe = par + e * ORC_NPARAM;
    const double *xe = xpar ? xpar + e * ORC_NXPARAM : NULL;
    const double *ge = geo + (int64_t)types[e] * ORC_NGEO;
    double *se = s + e * ORC_NSTATE, next[ORC_NSTATE];
    int bad = 0;
    for (int32_t j = 0; j < n_steps; ++j) {
      int32_t seg = j / hold;
      if (seg > n_seg - 1) seg = n_seg - 1;
      const double *c = cmd + ((int64_t)seg * n + e) * ORC_MAXTHR;
      bad |= orc_rk4_step_x(pe, xe, ge, se, c, h, flags, next);
      memcpy(se, next, sizeof next);
      if (traj) memcpy(traj + ((int64_t)j * n + e) * ORC_NSTATE, se, sizeof next);
    }
    fails += bad ? 1 : 0;
  }
  return fails;
}

int64_t orc_rollout(int64_t n, const double *par, const double *geo, const int32_t *types,
                    double *s, const double *cmd, int32_t n_seg, int32_t hold, int32_t n_steps,
                    double h, int32_t flags, double *traj, int32_t nthreads) {
  return orc_rollout_x(n, par, NULL, geo, types, s, cmd, n_seg, hold, n_steps, h, flags, traj,
                       nthreads);
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ counter-based RNG
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC 2011): 10 rounds of two 32x32->64 multiplies on a 4-word counter, a 2-word key bumped by
 * the Weyl constants between rounds.  Used for the domain-randomisation draws (§METHOD). */
static const uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;
static const uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PH_M0 * c[0];
    uint64_t p1 = (uint64_t)PH_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += PH_W0;
    k1 += PH_W1;
  }
  memcpy(out, c, sizeof c);
}

/* Open-interval uniform from the top 23 bits: ((x >> 9) + 1/2) * 2^-23, exact in FP32. */
static double u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Box-Muller pair from two uniforms. */
static void box_muller(double u1, double u2, double *z0, double *z1) {
  const double two_pi = 6.283185307179586476925286766559;
  double rad = sqrt(-2.0 * log(u1));
  *z0 = rad * cos(two_pi * u2);
  *z1 = rad * sin(two_pi * u2);
}

static void draw(uint64_t seed, uint64_t gid, uint32_t stream, uint32_t block, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)gid, (uint32_t)(gid >> 32), stream, block};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  orc_philox4x32_10(ctr, key, x);
  for (int i = 0; i < 4; ++i) u[i] = u01(x[i]);
}

static const int RAND_IDX[27] = {
    P_M, P_IG, P_IG + 1, P_IG + 2,
    P_MA, P_MA + 1, P_MA + 2, P_MA + 3, P_MA + 4, P_MA + 5,
    P_DL, P_DL + 1, P_DL + 2, P_DL + 3, P_DL + 4, P_DL + 5,
    P_DQ, P_DQ + 1, P_DQ + 2, P_DQ + 3, P_DQ + 4, P_DQ + 5,
    P_W, P_B, P_RB + 2, P_KT, P_TAU};

/* Domain randomisation (§METHOD; §EXPERIMENTS "domain randomization"): every scalar of the
 * randomised set is the nominal value times U[lo, hi] (uniform j of stream 0, block j/4, word
 * j%4); the NED current is the nominal one plus current_sigma * N(0,1)^3 (stream 1, block 0,
 * Box-Muller on words (0,1) and (2,3)); with rg_halfwidth > 0 the centre of gravity is the
 * nominal one plus rg_halfwidth * (2u - 1) per axis (stream 0, block 7, words 0..2).
 * Counter = (gid lo, gid hi, stream, block), key = seed. */
void orc_randomize(int64_t n, uint64_t seed, double lo, double hi, double current_sigma,
                   double rg_halfwidth, const double *nominal /*[n_types][NPARAM]*/,
                   const int32_t *types, int64_t gid0, double *par /*[n][NPARAM]*/) {
  for (int64_t e = 0; e < n; ++e) {
    uint64_t gid = (uint64_t)(gid0 + e);
    const double *nom = nominal + (int64_t)types[e] * ORC_NPARAM;
    double *pe = par + e * ORC_NPARAM;
    memcpy(pe, nom, ORC_NPARAM * sizeof(double));
    double u[4];
    for (int j = 0; j < 27; ++j) {
      if (j % 4 == 0) draw(seed, gid, 0u, (uint32_t)(j / 4), u);
      pe[RAND_IDX[j]] = nom[RAND_IDX[j]] * (lo + (hi - lo) * u[j % 4]);
    }
    double z[4];
    draw(seed, gid, 1u, 0u, u);
    box_muller(u[0], u[1], &z[0], &z[1]);
    box_muller(u[2], u[3], &z[2], &z[3]);
    for (int i = 0; i < 3; ++i) pe[P_VC + i] = nom[P_VC + i] + current_sigma * z[i];
    if (rg_halfwidth > 0.0) {
      draw(seed, gid, 0u, 7u, u);
      for (int i = 0; i < 3; ++i) pe[P_RG + i] = nom[P_RG + i] + rg_halfwidth * (2.0 * u[i] - 1.0);
    }
  }
}

/* Episode start for env gid at its episode-th reset: p = 0, q = identity, n = 0,
 * nu = nu0_sigma * N(0,1)^6 (stream 2, blocks 2*episode and 2*episode+1, Box-Muller on word
 * pairs (0,1), (2,3) of the first block and (0,1) of the second). */
void orc_reset_state(uint64_t seed, double nu0_sigma, int64_t gid, uint32_t episode,
                     double *s /*[NSTATE]*/) {
  double u[4], z[6];
  memset(s, 0, ORC_NSTATE * sizeof(double));
  s[S_Q] = 1.0;
  draw(seed, (uint64_t)gid, 2u, 2u * episode, u);
  box_muller(u[0], u[1], &z[0], &z[1]);
  box_muller(u[2], u[3], &z[2], &z[3]);
  draw(seed, (uint64_t)gid, 2u, 2u * episode + 1u, u);
  box_muller(u[0], u[1], &z[4], &z[5]);
  for (int i = 0; i < 6; ++i) s[S_NU + i] = nu0_sigma * z[i];
}

/* Procedural commands: throttle c_i = 2u - 1 for segment seg of env gid (stream 3, blocks 2*seg
 * and 2*seg+1 give the 8 thrusters), zero past n_thr. */
void orc_commands(uint64_t cmd_seed, int64_t gid, uint32_t seg, int32_t n_thr,
                  double *c /*[8]*/) {
  double u[8];
  draw(cmd_seed, (uint64_t)gid, 3u, 2u * seg, u);
  draw(cmd_seed, (uint64_t)gid, 3u, 2u * seg + 1u, u + 4);
  for (int i = 0; i < ORC_MAXTHR; ++i) c[i] = (i < n_thr) ? 2.0 * u[i] - 1.0 : 0.0;
}

/* ------------------------------------------------------------------ task layer (§EXPERIMENTS)
 * Four tasks: 0 station-keeping at a target point, 1 circle, 2 helix, 3 lemniscate tracking.
 * Readings (the paper names the tasks and gives Eq. 2 and Eq. 4, but no trajectory parameters):
 *   - every reference lies in NED around the env's centre c = (cx, cy, cz) with phase phi0:
 *       circle      p_r(t) = c + (R cos(w t + phi0), R sin(w t + phi0), 0)
 *       helix       p_r(t) = c + (R cos(w t + phi0), R sin(w t + phi0), vz t)
 *       lemniscate  p_r(t) = c + R (cos s, sin s cos s, 0) / (1 + sin^2 s),  s = w t + phi0
 *       station     p_r(t) = c
 *   - the attitude reference is level with heading psi_r, so the attitude error is
 *     (phi, theta, wrap(psi - psi_r)) from the zyx Euler angles of q;
 *   - Eq. 2: station keeping observes {eta^e, nu}; tracking observes the errors to the next m
 *     reference points p_r(t + i dt_look), i = 1..m, and nu; eta^e = (p - p_r, attitude error);
 *   - Eq. 4: the position error is |p - p_r(t)|; for tracking tasks the sum over the episode's
 *     evaluation points (one per task step) is accumulated. */
static double wrap_pi(double a) {
  const double two_pi = 6.283185307179586476925286766559;
  a = fmod(a + 3.14159265358979323846, two_pi);
  if (a < 0) a += two_pi;
  return a - 3.14159265358979323846;
}

void orc_euler_zyx(const double q[4], double e[3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  double sp = 2.0 * (w * y - z * x);
  if (sp > 1.0) sp = 1.0;
  if (sp < -1.0) sp = -1.0;
  e[0] = atan2(2.0 * (w * x + y * z), 1.0 - 2.0 * (x * x + y * y));
  e[1] = asin(sp);
  e[2] = atan2(2.0 * (w * z + x * y), 1.0 - 2.0 * (y * y + z * z));
}

void orc_task_reference(int32_t task, const double *c /*cx cy cz phi0*/, double radius,
                        double omega, double vz, double t, double p[3]) {
  const double s = omega * t + c[3];
  p[0] = c[0];
  p[1] = c[1];
  p[2] = c[2];
  if (task == 1 || task == 2) {
    p[0] += radius * cos(s);
    p[1] += radius * sin(s);
    if (task == 2) p[2] += vz * t;
  } else if (task == 3) {
    const double d = 1.0 + sin(s) * sin(s);
    p[0] += radius * cos(s) / d;
    p[1] += radius * sin(s) * cos(s) / d;
  }
}

/* Observation (Eq. 2) and position error (Eq. 4) of one env at task time t.  obs receives
 * 6 m + 6 values (m = 1 for station keeping): for i = 1..m the position error p - p_r(t + i dt)
 * and the attitude error, then nu.  Returns |p - p_r(t)|. */
double orc_task_observe(int32_t task, const double *s, const double *c, double radius,
                        double omega, double vz, double psi_r, int32_t m, double dt_look,
                        double t, double *obs) {
  double e[3], pr[3];
  orc_euler_zyx(s + S_Q, e);
  const double att[3] = {e[0], e[1], wrap_pi(e[2] - psi_r)};
  const int32_t mm = task == 0 ? 1 : m;
  for (int32_t i = 0; i < mm; ++i) {
    orc_task_reference(task, c, radius, omega, vz, task == 0 ? t : t + (i + 1) * dt_look, pr);
    for (int k = 0; k < 3; ++k) {
      obs[6 * i + k] = s[S_P + k] - pr[k];
      obs[6 * i + 3 + k] = att[k];
    }
  }
  for (int k = 0; k < 6; ++k) obs[6 * mm + k] = s[S_NU + k];
  orc_task_reference(task, c, radius, omega, vz, t, pr);
  double d2 = 0.0;
  for (int k = 0; k < 3; ++k) d2 += (s[S_P + k] - pr[k]) * (s[S_P + k] - pr[k]);
  return sqrt(d2);
}

/* ------------------------------------------------------------------ split integration
 * The paper's own arrangement of Eq. 1 (§METHOD): the rigid-body term is integrated by the
 * physics engine, while the hydrodynamic term (added mass, added-mass Coriolis, damping,
 * buoyancy) is computed by a separate module and applied to the body as an external force.
 * Reading of one sub-step of size h (the engine's semi-implicit Euler; the added-mass force
 * needs nu', which is not known yet, so the previous sub-step's acceleration a stands in):
 *
 *   tau_h = -( M_A (a + [w x v_c^b; 0]) + C_A(nu_r) nu_r + D(nu_r) nu_r + g_A(eta) )
 *   nu'   = M_RB^-1 ( tau + tau_h - C_RB(nu) nu - g_RB(eta) )
 *   nu+ = nu + h nu',   p+ = p + h R(q) v+,   q+ = (q + h/2 q (x) (0, w+)) / |.|,
 *   n+  = n + h (c - n) / tau_m,   a+ = nu'
 *
 * g_RB is the weight part of the restoring vector (acting at r_g), g_A the buoyancy part (at
 * r_b); the current term M_A [w x v_c^b; 0] follows the coupled reading and shares its flag.
 * a = 0 at an episode start.  M_RB is the full rigid-body inertia of Eq. 1 (r_g may be off the
 * origin, and the solve is the general one); x is the off-diagonal extension of M_A and D_l
 * (NULL: the diagonal model), as in the coupled step. */
static void restoring_parts(const double *par, const double q[4], double g_rb[6],
                            double g_a[6]) {
  double Rf[9], R[3][3];
  orc_rotation(q, Rf);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = Rf[3 * i + j];
  double fgn[3] = {0.0, 0.0, par[P_W]}, fbn[3] = {0.0, 0.0, -par[P_B]};
  double fg[3], fb[3];
  mat3T_vec(R, fgn, fg);
  mat3T_vec(R, fbn, fb);
  double rg[3] = {par[P_RG], par[P_RG + 1], par[P_RG + 2]};
  double rb[3] = {par[P_RB], par[P_RB + 1], par[P_RB + 2]};
  double mg[3], mb[3];
  cross3(rg, fg, mg);
  cross3(rb, fb, mb);
  for (int i = 0; i < 3; ++i) {
    g_rb[i] = -fg[i];
    g_rb[3 + i] = -mg[i];
    g_a[i] = -fb[i];
    g_a[3 + i] = -mb[i];
  }
}

int orc_split_step_x(const double *par, const double *x, const double *geo, const double *s,
                     const double *a, const double *c, double h, int flags, double *out,
                     double *a_out) {
  const double *p = s + S_P, *q = s + S_Q, *nu = s + S_NU, *n = s + S_N;
  int nthr = (int)geo[0];
  double Rf[9], R[3][3];
  orc_rotation(q, Rf);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = Rf[3 * i + j];
  double vcn[3] = {par[P_VC], par[P_VC + 1], par[P_VC + 2]}, vcb[3];
  mat3T_vec(R, vcn, vcb);
  double nu_r[6];
  for (int i = 0; i < 3; ++i) {
    nu_r[i] = nu[i] - vcb[i];
    nu_r[3 + i] = nu[3 + i];
  }

  /* hydrodynamic module: an external generalised force */
  double Ma[36], Ca[36], D[36], g_rb[6], g_a[6];
  orc_mass_a_x(par, x, Ma);
  orc_coriolis_a_x(par, x, nu_r, Ca);
  orc_damping_x(par, x, nu_r, D);
  restoring_parts(par, q, g_rb, g_a);
  double acc[6];
  for (int i = 0; i < 6; ++i) acc[i] = a[i];
  if (!(flags & ORC_NO_CURRENT_ACCEL)) {
    double wx[3];
    cross3(nu + 3, vcb, wx);
    for (int i = 0; i < 3; ++i) acc[i] += wx[i];
  }
  double ma[6], ca[6], dd[6], tau_h[6];
  mat6_vec((const double(*)[6])Ma, acc, ma);
  mat6_vec((const double(*)[6])Ca, nu_r, ca);
  mat6_vec((const double(*)[6])D, nu_r, dd);
  for (int i = 0; i < 6; ++i) tau_h[i] = -(ma[i] + ca[i] + dd[i] + g_a[i]);

  /* rigid body: M_RB nu' = tau + tau_h - C_RB(nu) nu - g_RB */
  double Mrb[36], Crb[36], crb[6], tau[6], rhs[6], nudot[6];
  orc_mass_rb(par, Mrb);
  orc_coriolis_rb(par, nu, Crb);
  mat6_vec((const double(*)[6])Crb, nu, crb);
  orc_thrust(par, geo, n, tau);
  for (int i = 0; i < 6; ++i) rhs[i] = tau[i] + tau_h[i] - crb[i] - g_rb[i];
  if (solve6((const double(*)[6])Mrb, rhs, nudot) != 0) return -1;

  /* semi-implicit Euler: velocities first, then the pose with the new velocities */
  double nu1[6];
  for (int i = 0; i < 6; ++i) nu1[i] = nu[i] + h * nudot[i];
  double pd[3];
  mat3_vec((const double(*)[3])R, nu1, pd);
  for (int i = 0; i < 3; ++i) out[S_P + i] = p[i] + h * pd[i];
  const double *w = nu1 + 3;
  double qd[4];
  qd[0] = -0.5 * (q[1] * w[0] + q[2] * w[1] + q[3] * w[2]);
  qd[1] = 0.5 * (q[0] * w[0] + q[2] * w[2] - q[3] * w[1]);
  qd[2] = 0.5 * (q[0] * w[1] + q[3] * w[0] - q[1] * w[2]);
  qd[3] = 0.5 * (q[0] * w[2] + q[1] * w[1] - q[2] * w[0]);
  double q1[4], nq = 0.0;
  for (int i = 0; i < 4; ++i) {
    q1[i] = q[i] + h * qd[i];
    nq += q1[i] * q1[i];
  }
  nq = sqrt(nq);
  for (int i = 0; i < 4; ++i) out[S_Q + i] = q1[i] / nq;
  for (int i = 0; i < 6; ++i) {
    out[S_NU + i] = nu1[i];
    a_out[i] = nudot[i];
  }
  for (int i = 0; i < ORC_MAXTHR; ++i)
    out[S_N + i] = (i < nthr) ? n[i] + h * (c[i] - n[i]) / par[P_TAU] : 0.0;
  return 0;
}

int orc_split_step(const double *par, const double *geo, const double *s, const double *a,
                   const double *c, double h, int flags, double *out, double *a_out) {
  return orc_split_step_x(par, NULL, geo, s, a, c, h, flags, out, a_out);
}

/* Fleet rollout of the split scheme; as orc_rollout_x, with the acceleration memory acc [n][6]
 * advanced in place alongside s. */
int64_t orc_split_rollout_x(int64_t n, const double *par, const double *xpar,
                            const double *geo, const int32_t *types, double *s, double *acc,
                            const double *cmd, int32_t n_seg, int32_t hold, int32_t n_steps,
                            double h, int32_t flags, int32_t nthreads) {
  int64_t fails = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : fails)
#endif
  for (int64_t e = 0; e < n; ++e) {
    const double *pe = par + e * ORC_NPARAM;
    const double *xe = xpar ? xpar + e * ORC_NXPARAM : NULL;
    const double *ge = geo + (int64_t)types[e] * ORC_NGEO;
    double *se = s + e * ORC_NSTATE, *ae = acc + e * 6, next[ORC_NSTATE], an[6];
    int bad = 0;
    for (int32_t j = 0; j < n_steps; ++j) {
      int32_t seg = j / hold;
      if (seg > n_seg - 1) seg = n_seg - 1;
      const double *c = cmd + ((int64_t)seg * n + e) * ORC_MAXTHR;
      bad |= orc_split_step_x(pe, xe, ge, se, ae, c, h, flags, next, an);
      memcpy(se, next, sizeof next);
      memcpy(ae, an, sizeof an);
    }
    fails += bad ? 1 : 0;
  }
  return fails;
}
