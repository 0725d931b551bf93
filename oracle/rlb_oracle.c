/*
 * FP64 CPU oracle of the relativistic lattice Boltzmann model with improved dissipation
 * (Mendoza, Karlin, Succi, Herrmann, arXiv:1301.3423).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the GPU library is checked
 * against.  It shares no code with the GPU path; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.
 *
 * Everything is serial double precision, written in the order the paper states the method:
 *   - pull streaming by the integer lattice vectors v_i (Eq. (rlb:disc), left-hand side);
 *   - moments N^mu = sum_i f_i p_i^mu and T^{mu nu} = sum_i f_i p_i^mu p_i^nu (Sec. II.D);
 *   - Landau matching T^{a b} U_b = eps U^a, n = U_mu N^mu, eps = 3 n T (Eqs. (eigenproblem),
 *     (densitycal), Sec. II.D), solved by plain power iteration from the Eckart vector N/|N|;
 *   - relaxation time tau' from eta/s (Sec. II.D transport coefficients, Sec. III entropy);
 *   - discrete equilibrium f_i^eq = w_i sum_k a_k J_k(p_i) (Eq. (eq:disc1)) with the projections
 *     a_k = int f^eq J_k d^3p/p0 (Eq. (coeff)) taken from the closed-form Maxwell-Juttner moments
 *     and J_k the Gram-Schmidt polynomials of Sec. II.B (orders 0-3, or 0-2 for the second-order
 *     model); the explicit App. B forms (Eqs. (eq:equi3rd), (eq:equi2nd)) are kept as a
 *     cross-check: written out in powers of p they lose up to ~1e-12 to cancellation at T ~ 2 and
 *     p0 ~ 11, the orthogonal-basis sum about 1e-14;
 *   - Anderson-Witting BGK collision f_i <- f_i - (p_i^mu U_mu)/(tau' p_i^0) (f_i - f_i^eq)
 *     (Eq. (rlb:disc), right-hand side, with delta t' = 1).
 *
 * Boundaries, per axis: periodic, copy-out (a pull source beyond the end is the nearest edge cell)
 * or bounce-back wall.  The paper asks for weights equal under p -> -p (spatial part) so that the
 * classical bounce-back rule conserves mass and energy at solid walls (Sec. II.C); it states no
 * rule for links longer than one cell.  Here a population whose pull source lies beyond a
 * bounce-back wall is replaced by the same cell's post-collision population of the reversed
 * momentum (same p0, -v), i.e. every population that would leave through the wall comes back
 * reversed into the cell it left.
 *
 * Conventions: lattice units delta x = delta t' = 1, metric diag(+,-,-,-),
 * p_i^mu = p0_i (1, v_i / R) (Eq. (eq:mrecon2)).  Populations are stored f[i][z][y][x].
 * The stored state is post-collision; a step is pull, then collide.
 *
 * Pins (tests/test_oracle_*.py, tests/test_lattice.py): the equilibrium against the closed-form
 * Maxwell-Juttner moments and the appendix forms, Landau matching against a dense eigen-solver,
 * one step against an independent numpy step, conservation, stationarity, the shear-wave rate,
 * the Riemann impulse, bounce-back conservation and no-slip, the reference-temperature relaxation
 * time against a fixed tau', and the sampled one-step routine (ora_init_step_cells) against init
 * plus one whole-lattice step at corners, face-adjacent and random cells for every boundary type.  The weight tables are read from
 * the lattice/ text files, rebuilt from the moment conditions of Eqs. (eqs:eqs) because the paper
 * does not print its own: results that depend on which valid table is used (beyond the moment
 * conditions) are parity unpinned against the paper.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include "gs_basis.h"

#define ORA_QMAX 128
#define ORA_HBARC_GEV_FM 0.1973269804 /* CODATA hbar*c, converts T*time into a pure number */

enum { ORA_OK = 0, ORA_EINVAL = 1, ORA_ENONCONV = 4 };

/* ---------------------------------------------------------------------------------------------
 * Equilibrium: App. B.  Both functions return f_i^eq / w_i for one 4-momentum (p0, px, py, pz)
 * in the frame where the fluid has 4-velocity U = (U0, Ux, Uy, Uz), density n and temperature T.
 * ------------------------------------------------------------------------------------------- */

/* Eq. (eq:equi3rd): the 30-polynomial (third-order) projection, written out as printed. */
double ora_feq3_over_w(double n, double T, const double U[4], double p0, double px, double py, double pz) {
  const double U0 = U[0], Ux = U[1], Uy = U[2], Uz = U[3];
  const double s = px * Ux + py * Uy + pz * Uz;
  const double T2 = T * T, T3 = T2 * T;
  const double U02 = U0 * U0, Ux2 = Ux * Ux, Uy2 = Uy * Uy;
  const double a1 = p0 * p0 * p0 * (T * U0 - 1.0) * (T2 * (4.0 * U02 - 3.0 * (Ux2 + Uy2 + 1.0)) - 2.0 * T * U0 + 1.0);
  const double a2 =
      p0 * p0 *
      (T3 * (-2.0 * U02 * (3.0 * px * Ux + 3.0 * py * Uy + 2.0 * pz * Uz) +
             (Ux2 + Uy2 + 1.0) * (3.0 * px * Ux + 3.0 * py * Uy + pz * Uz) + 36.0 * U02 * U0 -
             6.0 * U0 * (3.0 * Ux2 + 3.0 * Uy2 + 4.0)) +
       3.0 * T2 * (2.0 * U0 * s - 22.0 * U02 + 7.0 * (Ux2 + Uy2) + 9.0) - 3.0 * T * (s - 14.0 * U0) - 15.0);
  const double a3 =
      3.0 * p0 *
      (T3 * (U02 * U0 * (px * px + py * py - 24.0) -
             U0 * (px * px * (2.0 * Ux2 + Uy2 + 1.0) + 2.0 * px * Ux * (py * Uy + pz * Uz) +
                   py * (py * Ux2 + 2.0 * py * Uy2 + py + 2.0 * pz * Uy * Uz) - 12.0) +
             12.0 * U02 * s - 2.0 * s) +
       T2 * (px * px * (-U02 + 2.0 * Ux2 + Uy2 + 1.0) + 2.0 * px * Ux * (py * Uy + pz * Uz - 11.0 * U0) +
             py * py * (-U02 + Ux2 + 2.0 * Uy2 + 1.0) + 2.0 * py * Uy * (pz * Uz - 11.0 * U0) -
             22.0 * pz * U0 * Uz + 56.0 * U02 - 14.0) +
       2.0 * T * (6.0 * s - 25.0 * U0) + 20.0);
  const double a4 =
      T * (px * px * px * T2 * Ux * (-3.0 * U02 + 4.0 * Ux2 + 3.0 * Uy2 + 3.0) +
           px * px * T *
               (3.0 * (U02 - 2.0 * Ux2 - Uy2 - 1.0) * (-py * T * Uy + 6.0 * T * U0 - 7.0) +
                pz * T * Uz * (-U02 + 4.0 * Ux2 + Uy2 + 1.0)) +
           3.0 * px * Ux *
               (T * (T * (py * py * (-U02 + Ux2 + 2.0 * Uy2 + 1.0) + 2.0 * py * Uy * (pz * Uz - 6.0 * U0) -
                          12.0 * pz * U0 * Uz + 24.0 * U02 - 4.0) +
                     14.0 * py * Uy + 14.0 * pz * Uz - 48.0 * U0) +
                30.0) +
           py * py * py * T2 * Uy * (-3.0 * U02 + 3.0 * Ux2 + 4.0 * Uy2 + 3.0) +
           py * py * T *
               (pz * T * Uz * (-U02 + Ux2 + 4.0 * Uy2 + 1.0) +
                3.0 * (6.0 * T * U0 - 7.0) * (U02 - Ux2 - 2.0 * Uy2 - 1.0)) +
           6.0 * py * Uy * (T * (2.0 * T * (-3.0 * pz * U0 * Uz + 6.0 * U02 - 1.0) + 7.0 * pz * Uz - 24.0 * U0) + 15.0) +
           6.0 * pz * Uz * (2.0 * T2 * (6.0 * U02 - 1.0) - 24.0 * T * U0 + 15.0) -
           24.0 * U0 * (T2 * (2.0 * U02 - 1.0) - 5.0 * T * U0 + 5.0));
  return n / (12.0 * T) * (a1 - a2 - a3 + a4 - 30.0 * (T2 - 2.0));
}

/* Eq. (eq:equi2nd): the 14-polynomial (second-order) projection, written out as printed. */
double ora_feq2_over_w(double n, double T, const double U[4], double p0, double px, double py, double pz) {
  const double U0 = U[0], Ux = U[1], Uy = U[2], Uz = U[3];
  const double s = px * Ux + py * Uy + pz * Uz;
  const double T2 = T * T;
  const double br =
      p0 * p0 * (T2 * (2.0 * U0 * U0 - Ux * Ux - Uy * Uy - 1.0) - 2.0 * T * U0 + 1.0) +
      2.0 * p0 * (T * (T * (U0 * (s - 4.0 * U0) + 1.0) - s + 7.0 * U0) - 4.0) +
      T2 * (px * px * (-U0 * U0 + 2.0 * Ux * Ux + Uy * Uy + 1.0) + 2.0 * px * Ux * (py * Uy + pz * Uz - 4.0 * U0) +
            py * py * (-U0 * U0 + Ux * Ux + 2.0 * Uy * Uy + 1.0) + 2.0 * py * Uy * (pz * Uz - 4.0 * U0) +
            8.0 * U0 * (U0 - pz * Uz) - 2.0) +
      2.0 * T * (5.0 * s - 8.0 * U0) + 12.0;
  return n / (4.0 * T) * br;
}

/* f_i^eq for every population of one cell through the explicit App. B form (cross-check only). */
void ora_equilibrium_appendix_cell(int order, int q, const int* v, const double* p0, const double* w, double n,
                                   double T, const double U[4], double* feq) {
  const double R = (order == 3) ? sqrt(41.0) : 3.0;
  for (int i = 0; i < q; ++i) {
    const double px = p0[i] * v[3 * i + 0] / R, py = p0[i] * v[3 * i + 1] / R, pz = p0[i] * v[3 * i + 2] / R;
    const double e = (order == 3) ? ora_feq3_over_w(n, T, U, p0[i], px, py, pz)
                                  : ora_feq2_over_w(n, T, U, p0[i], px, py, pz);
    feq[i] = w[i] * e;
  }
}

/* ---------------------------------------------------------------------------------------------
 * Equilibrium as the projection of Sec. II.B.  The orthogonal polynomials P_k (unnormalised J_k)
 * come from exact Gram-Schmidt over the monomials p0^e px^a py^b pz^c (e <= 1) listed in
 * gs_basis.h; a_k J_k(p) = (<f^eq, P_k> / <P_k, P_k>) P_k(p) with <f^eq, m> the Maxwell-Juttner
 * moment of the monomial m.
 * ------------------------------------------------------------------------------------------- */
static int gs_size(int order) { return order == 3 ? ORA_GS3_N : ORA_GS2_N; }
static const int (*gs_mono(int order))[4] { return order == 3 ? ora_gs3_mono : ora_gs2_mono; }
static long double gs_coef(int order, int k, int j) { return order == 3 ? ora_gs3_coef[k][j] : ora_gs2_coef[k][j]; }
static long double gs_norm(int order, int k) { return order == 3 ? ora_gs3_norm[k] : ora_gs2_norm[k]; }

/* P_k(p_i) for every population (tab[i][k], i < q, k < gs_size), evaluated in long double and
 * rounded once.  Returns the number of basis polynomials. */
int ora_gs_table(int order, int q, const int* v, const double* p0, double* tab) {
  const int nm = gs_size(order);
  const int(*mono)[4] = gs_mono(order);
  const long double R = sqrtl(order == 3 ? 41.0L : 9.0L);
  for (int i = 0; i < q; ++i) {
    const long double p[4] = {p0[i], p0[i] * (long double)v[3 * i] / R, p0[i] * (long double)v[3 * i + 1] / R,
                              p0[i] * (long double)v[3 * i + 2] / R};
    long double m[ORA_GS3_N];
    for (int j = 0; j < nm; ++j) {
      long double x = 1.0L;
      for (int e = 0; e < mono[j][0]; ++e) x *= p[0];
      for (int e = 0; e < mono[j][1]; ++e) x *= p[1];
      for (int e = 0; e < mono[j][2]; ++e) x *= p[2];
      for (int e = 0; e < mono[j][3]; ++e) x *= p[3];
      m[j] = x;
    }
    for (int k = 0; k < nm; ++k) {
      long double s = 0.0L;
      for (int j = 0; j < nm; ++j) s += gs_coef(order, k, j) * m[j];
      tab[(size_t)i * nm + k] = (double)s;
    }
  }
  return nm;
}

/* Maxwell-Juttner moment of the monomial p0^e px^a py^b pz^c (degree <= 3) over d^3p/p0:
 * n/(2T) for degree 0 (a Lorentz scalar, its rest-frame value), then N^mu = n U^mu,
 * T^{mu nu} = -n T eta^{mu nu} + 4 n T U^mu U^nu, P^{mu nu l} = -4 n T^2 (eta^{mu nu} U^l +
 * eta^{mu l} U^nu + eta^{nu l} U^mu) + 24 n T^2 U^mu U^nu U^l (Sec. II.C). */
static double mj_moment(double n, double T, const double U[4], const int mono[4]) {
  int idx[3], k = 0;
  for (int e = 0; e < mono[0]; ++e) idx[k++] = 0;
  for (int e = 0; e < mono[1]; ++e) idx[k++] = 1;
  for (int e = 0; e < mono[2]; ++e) idx[k++] = 2;
  for (int e = 0; e < mono[3]; ++e) idx[k++] = 3;
#define ETA(a, b) ((a) != (b) ? 0.0 : ((a) == 0 ? 1.0 : -1.0))
  switch (k) {
    case 0: return n / (2.0 * T);
    case 1: return n * U[idx[0]];
    case 2: return -n * T * ETA(idx[0], idx[1]) + 4.0 * n * T * U[idx[0]] * U[idx[1]];
    default:
      return -4.0 * n * T * T *
                 (ETA(idx[0], idx[1]) * U[idx[2]] + ETA(idx[0], idx[2]) * U[idx[1]] + ETA(idx[1], idx[2]) * U[idx[0]]) +
             24.0 * n * T * T * U[idx[0]] * U[idx[1]] * U[idx[2]];
  }
#undef ETA
}

/* f_i^eq = w_i sum_k a_k J_k(p_i) for every population of one cell (Eqs. (coeff), (eq:disc1));
 * gs = the table of ora_gs_table for this lattice. */
void ora_equilibrium_cell(int order, int q, const double* w, const double* gs, double n, double T, const double U[4],
                          double* feq) {
  const int nm = gs_size(order);
  const int(*mono)[4] = gs_mono(order);
  double b[ORA_GS3_N], a[ORA_GS3_N];
  for (int j = 0; j < nm; ++j) b[j] = mj_moment(n, T, U, mono[j]);
  for (int k = 0; k < nm; ++k) {
    double s = 0.0;
    for (int j = 0; j < nm; ++j) s += (double)gs_coef(order, k, j) * b[j];
    a[k] = s / (double)gs_norm(order, k); /* <f^eq, P_k> / <P_k, P_k> */
  }
  for (int i = 0; i < q; ++i) {
    double s = 0.0;
    for (int k = 0; k < nm; ++k) s += a[k] * gs[(size_t)i * nm + k];
    feq[i] = w[i] * s;
  }
}

/* N^mu = sum_i f_i p_i^mu, T^{mu nu} = sum_i f_i p_i^mu p_i^nu (Eqs. (moments:dis1), (moments:dis2)). */
void ora_moments_cell(int order, int q, const int* v, const double* p0, const double* f, double N[4], double Tm[16]) {
  const double R = (order == 3) ? sqrt(41.0) : 3.0;
  for (int a = 0; a < 4; ++a) N[a] = 0.0;
  for (int a = 0; a < 16; ++a) Tm[a] = 0.0;
  for (int i = 0; i < q; ++i) {
    const double p[4] = {p0[i], p0[i] * v[3 * i] / R, p0[i] * v[3 * i + 1] / R, p0[i] * v[3 * i + 2] / R};
    for (int a = 0; a < 4; ++a) {
      N[a] += f[i] * p[a];
      for (int b = 0; b < 4; ++b) Tm[4 * a + b] += f[i] * p[a] * p[b];
    }
  }
}

/* Landau matching (Eq. (eigenproblem) and Sec. II.D): U is the timelike eigenvector of
 * T^a_b = T^{a c} eta_{c b} with U^0 > 0, U.U = 1; eps its eigenvalue; n = U_mu N^mu.
 * Power iteration U <- V / sqrt(V.V), V^a = T^{a c} U_c, started from N / sqrt(N.N).
 * Stops when max |dU| <= 4 * 2^-52 * U^0, or when the change has stalled at round-off, or after
 * 500 iterations.  Returns ORA_ENONCONV if a Minkowski norm is not positive. */
int ora_landau_cell(const double N[4], const double Tm[16], double U[4], double* eps, double* n) {
  const double eta[4] = {1.0, -1.0, -1.0, -1.0};
  double NN = N[0] * N[0] - N[1] * N[1] - N[2] * N[2] - N[3] * N[3];
  if (!(NN > 0.0) || !(N[0] > 0.0)) return ORA_ENONCONV;
  for (int a = 0; a < 4; ++a) U[a] = N[a] / sqrt(NN);
  double prev = INFINITY, e = 0.0;
  for (int it = 0; it < 500; ++it) {
    double V[4];
    for (int a = 0; a < 4; ++a) {
      V[a] = 0.0;
      for (int c = 0; c < 4; ++c) V[a] += Tm[4 * a + c] * eta[c] * U[c];
    }
    const double VV = V[0] * V[0] - V[1] * V[1] - V[2] * V[2] - V[3] * V[3];
    if (!(VV > 0.0) || !(V[0] > 0.0)) return ORA_ENONCONV;
    e = sqrt(VV);
    double d = 0.0;
    for (int a = 0; a < 4; ++a) {
      const double un = V[a] / e;
      d = fmax(d, fabs(un - U[a]));
      U[a] = un;
    }
    if (d <= 4.0 * 2.220446049250313e-16 * U[0]) break;
    if (d >= prev && d <= 1e-11 * U[0]) break; /* stalled at round-off */
    prev = d;
  }
  *eps = e;
  *n = U[0] * N[0] - U[1] * N[1] - U[2] * N[2] - U[3] * N[3];
  if (!(*n > 0.0)) return ORA_ENONCONV;
  return ORA_OK;
}

/* Relaxation time in lattice units.  The paper gives eta = (2/3) P (tau' - dt'/2) and, undoing the
 * time dilatation, (tau - dt/2)/R (Sec. II.D, Sec. III); entropy s = 4n (Sec. III, dropping the
 * n ln(n/n_eq) term).  With P = nT and the physical unit conversion kappa = T_unit * dx / (hbar c):
 * tau' = 1/2 + 6 (eta/s) / (R kappa T). */
double ora_tau_prime(double eta_over_s, double R, double kappa, double T) {
  return 0.5 + 6.0 * eta_over_s / (R * kappa * T);
}

/* Source coordinate of a pull along one axis (bc 0 periodic, 1 copy-out; a bounce-back axis, 2,
 * never gets here with s outside [0, n): see beyond_wall). */
static inline long wrap_index(long s, long n, int bc) {
  if (bc == 0) { /* periodic */
    s %= n;
    if (s < 0) s += n;
    return s;
  }
  if (s < 0) return 0; /* copy-out: nearest edge cell */
  if (s >= n) return n - 1;
  return s;
}

/* 1 if the pull source (x, y, z) - v_i lies beyond a bounce-back wall. */
static inline int beyond_wall(const int* bc, long x, long y, long z, int nx, int ny, int nz, const int* vi) {
  const long s[3] = {x - vi[0], y - vi[1], z - vi[2]};
  const long n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a)
    if (bc[a] == 2 && (s[a] < 0 || s[a] >= n[a])) return 1;
  return 0;
}

/* Index of the population with the reversed momentum (same p0, -v) of population i. */
static int reversed_population(int q, const int* v, const double* p0, int i) {
  for (int j = 0; j < q; ++j)
    if (v[3 * j] == -v[3 * i] && v[3 * j + 1] == -v[3 * i + 1] && v[3 * j + 2] == -v[3 * i + 2] && p0[j] == p0[i])
      return j;
  return -1;
}

/* Moments, Landau matching, relaxation time, equilibrium and collision of one cell whose pulled
 * populations are ft[q].  Writes fo[q] (if collide), fld[6] = n, eps, U0..U3 and dn[5] = N^0,
 * T^00, T^0x, T^0y, T^0z (if non-NULL).  Returns ORA_OK or ORA_ENONCONV (then fo = ft, fld = NaN). */
static int collide_cell(int order, int q, const int* v, const double* p0, const double* w, const double* gs,
                        double eta_over_s,
                        double tau_prime, int tau_local_T, double T_ref, double kappa, int collide,
                        const double* ft, double* fo, double* fld, double* dn) {
  const double R = (order == 3) ? sqrt(41.0) : 3.0;
  double N[4], Tm[16], U[4], eps = NAN, n = NAN, feq[ORA_QMAX];
  ora_moments_cell(order, q, v, p0, ft, N, Tm);
  if (dn) {
    dn[0] = N[0];
    for (int b = 0; b < 4; ++b) dn[1 + b] = Tm[b];
  }
  if (ora_landau_cell(N, Tm, U, &eps, &n) != ORA_OK) {
    if (fld)
      for (int k = 0; k < 6; ++k) fld[k] = NAN;
    if (collide)
      for (int i = 0; i < q; ++i) fo[i] = ft[i];
    return ORA_ENONCONV;
  }
  const double T = eps / (3.0 * n); /* equation of state eps = 3 n T */
  if (fld) {
    fld[0] = n;
    fld[1] = eps;
    for (int a = 0; a < 4; ++a) fld[2 + a] = U[a];
  }
  if (!collide) return ORA_OK;
  const double tau = (tau_prime > 0.5) ? tau_prime : ora_tau_prime(eta_over_s, R, kappa, tau_local_T ? T : T_ref);
  ora_equilibrium_cell(order, q, w, gs, n, T, U, feq);
  for (int i = 0; i < q; ++i) {
    /* p_i^mu U_mu / p_i^0 = U0 - (v_i . U) / R */
    const double pu = U[0] - (v[3 * i] * U[1] + v[3 * i + 1] * U[2] + v[3 * i + 2] * U[3]) / R;
    fo[i] = ft[i] - pu / tau * (ft[i] - feq[i]);
  }
  return ORA_OK;
}

/*
 * One time step on the whole lattice (Eq. (rlb:disc)): pull f~_i(x) = fin_i(x - v_i), moments,
 * Landau matching, tau', equilibrium, collision; writes fout.  If fields != NULL it receives the
 * Landau fields of the pulled (pre-collision) populations: fields[k][cell], k = n, eps, U0..U3.
 * If dens != NULL it receives the conserved densities N^0, T^00, T^0x, T^0y, T^0z per cell.
 * collide = 0 only pulls and evaluates (fields / dens); pull = 0 reads each cell in place.
 * tau_prime > 0.5 fixes tau'; otherwise tau' follows eta/s with the local (tau_local_T = 1) or the
 * reference temperature.  bc[a] per axis: 0 periodic, 1 copy-out, 2 bounce-back wall.  Returns the
 * number of cells where Landau matching failed (those cells are copied without collision and get
 * NaN fields), or -1 if a bounce-back wall is asked for and a population has no reversed partner.
 */
long ora_step(int order, int q, const int* v, const double* p0, const double* w, const double* gs, int nx, int ny,
              int nz,
              const int* bc, double eta_over_s, double tau_prime, int tau_local_T, double T_ref, double dx_fm,
              double T_unit_GeV, int pull, int collide, const double* fin, double* fout, double* fields,
              double* dens) {
  const double kappa = T_unit_GeV * dx_fm / ORA_HBARC_GEV_FM;
  const size_t cells = (size_t)nx * ny * nz;
  long bad = 0;
  double ft[ORA_QMAX], fo[ORA_QMAX], fld[6], dn[5];
  int rev[ORA_QMAX];
  for (int i = 0; i < q; ++i) {
    rev[i] = reversed_population(q, v, p0, i);
    if (rev[i] < 0 && (bc[0] == 2 || bc[1] == 2 || bc[2] == 2)) return -1;
  }
  for (long z = 0; z < nz; ++z)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x) {
        const size_t c = ((size_t)z * ny + y) * nx + x;
        for (int i = 0; i < q; ++i) {
          if (pull && beyond_wall(bc, x, y, z, nx, ny, nz, v + 3 * i)) {
            ft[i] = fin[(size_t)rev[i] * cells + c]; /* bounced back at the wall */
            continue;
          }
          long sx = x, sy = y, sz = z;
          if (pull) {
            sx = wrap_index(x - v[3 * i + 0], nx, bc[0]);
            sy = wrap_index(y - v[3 * i + 1], ny, bc[1]);
            sz = wrap_index(z - v[3 * i + 2], nz, bc[2]);
          }
          ft[i] = fin[(size_t)i * cells + ((size_t)sz * ny + sy) * nx + sx];
        }
        if (collide_cell(order, q, v, p0, w, gs, eta_over_s, tau_prime, tau_local_T, T_ref, kappa, collide, ft, fo,
                         fld, dn) != ORA_OK)
          ++bad;
        if (fields)
          for (int k = 0; k < 6; ++k) fields[k * cells + c] = fld[k];
        if (dens)
          for (int k = 0; k < 5; ++k) dens[k * cells + c] = dn[k];
        if (collide)
          for (int i = 0; i < q; ++i) fout[(size_t)i * cells + c] = fo[i];
      }
  return bad;
}

/*
 * Sampled cells of one step taken from the equilibrium of given fields: every population of the
 * lattice starts as f_i^eq(n, T, u) of its cell; for each listed cell the populations after one
 * step are written to out[k][q].  Needs only the fields (n, T double[cells], u double[3][cells]),
 * so it can check single cells of lattices too large for ora_step.  Returns the number of listed
 * cells where Landau matching failed, or -1 for invalid fields.
 */
long ora_init_step_cells(int order, int q, const int* v, const double* p0, const double* w, const double* gs, int nx,
                         int ny, int nz,
                         const int* bc, double eta_over_s, double tau_prime, int tau_local_T, double T_ref,
                         double dx_fm, double T_unit_GeV, const double* n, const double* T, const double* u,
                         long nsample, const long* sample, double* out) {
  const double kappa = T_unit_GeV * dx_fm / ORA_HBARC_GEV_FM;
  const size_t cells = (size_t)nx * ny * nz;
  const int nm = gs_size(order);
  long bad = 0;
  double ft[ORA_QMAX], feq[ORA_QMAX];
  for (long k = 0; k < nsample; ++k) {
    const long c = sample[k];
    const long x = c % nx, y = (c / nx) % ny, z = c / ((long)nx * ny);
    for (int i = 0; i < q; ++i) {
      /* source cell and source population (the reversed one, in place, beyond a wall) */
      int src_i = i;
      size_t s;
      if (beyond_wall(bc, x, y, z, nx, ny, nz, v + 3 * i)) {
        src_i = reversed_population(q, v, p0, i);
        if (src_i < 0) return -1;
        s = (size_t)c;
      } else {
        const long sx = wrap_index(x - v[3 * i + 0], nx, bc[0]);
        const long sy = wrap_index(y - v[3 * i + 1], ny, bc[1]);
        const long sz = wrap_index(z - v[3 * i + 2], nz, bc[2]);
        s = ((size_t)sz * ny + sy) * nx + sx;
      }
      const double ux = u[s], uy = u[cells + s], uz = u[2 * cells + s];
      const double u2 = ux * ux + uy * uy + uz * uz;
      if (!(u2 < 1.0) || !(T[s] > 0.0) || !(n[s] > 0.0)) return -1;
      const double g = 1.0 / sqrt(1.0 - u2);
      const double U[4] = {g, g * ux, g * uy, g * uz};
      /* population src_i of the source cell: its equilibrium, evaluated for that population only */
      ora_equilibrium_cell(order, 1, w + src_i, gs + (size_t)src_i * nm, n[s], T[s], U, feq);
      ft[i] = feq[0];
    }
    if (collide_cell(order, q, v, p0, w, gs, eta_over_s, tau_prime, tau_local_T, T_ref, kappa, 1, ft, out + k * q,
                     NULL, NULL) != ORA_OK)
      ++bad;
  }
  return bad;
}

/* f_i = f_i^eq(n, T, u) on every cell; U = gamma (1, u).  Returns ORA_EINVAL if |u| >= 1. */
int ora_init(int order, int q, const double* w, const double* gs, long cells, const double* n, const double* T,
             const double* u, double* f) {
  double feq[ORA_QMAX];
  for (long c = 0; c < cells; ++c) {
    const double ux = u[c], uy = u[cells + c], uz = u[2 * cells + c];
    const double u2 = ux * ux + uy * uy + uz * uz;
    if (!(u2 < 1.0) || !(T[c] > 0.0) || !(n[c] > 0.0)) return ORA_EINVAL;
    const double g = 1.0 / sqrt(1.0 - u2);
    const double U[4] = {g, g * ux, g * uy, g * uz};
    ora_equilibrium_cell(order, q, w, gs, n[c], T[c], U, feq);
    for (int i = 0; i < q; ++i) f[(size_t)i * cells + c] = feq[i];
  }
  return ORA_OK;
}
