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
 *   - discrete equilibrium f_i^eq = w_i * (explicit polynomial of App. B, Eq. (eq:equi3rd) for the
 *     third-order model, Eq. (eq:equi2nd) for the second-order model);
 *   - Anderson-Witting BGK collision f_i <- f_i - (p_i^mu U_mu)/(tau' p_i^0) (f_i - f_i^eq)
 *     (Eq. (rlb:disc), right-hand side, with delta t' = 1).
 *
 * Conventions: lattice units delta x = delta t' = 1, metric diag(+,-,-,-),
 * p_i^mu = p0_i (1, v_i / R) (Eq. (eq:mrecon2)).  Populations are stored f[i][z][y][x].
 * The stored state is post-collision; a step is pull, then collide.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

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

/* f_i^eq for every population of one cell (Eq. (eq:disc1) through its explicit form). */
void ora_equilibrium_cell(int order, int q, const int* v, const double* p0, const double* w, double n, double T,
                          const double U[4], double* feq) {
  const double R = (order == 3) ? sqrt(41.0) : 3.0;
  for (int i = 0; i < q; ++i) {
    const double px = p0[i] * v[3 * i + 0] / R, py = p0[i] * v[3 * i + 1] / R, pz = p0[i] * v[3 * i + 2] / R;
    const double e = (order == 3) ? ora_feq3_over_w(n, T, U, p0[i], px, py, pz)
                                  : ora_feq2_over_w(n, T, U, p0[i], px, py, pz);
    feq[i] = w[i] * e;
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

/*
 * One time step on the whole lattice (Eq. (rlb:disc)): pull f~_i(x) = fin_i(x - v_i), moments,
 * Landau matching, tau', equilibrium, collision; writes fout.  If fields != NULL it receives the
 * Landau fields of the pulled (pre-collision) populations: fields[k][cell], k = n, eps, U0..U3.
 * If dens != NULL it receives the conserved densities N^0, T^00, T^0x, T^0y, T^0z per cell.
 * collide = 0 only pulls and evaluates (fields / dens); pull = 0 reads each cell in place.
 * tau_prime > 0.5 fixes tau'; otherwise tau' follows eta/s with the local (tau_local_T = 1) or the
 * reference temperature.  Returns the number of cells where Landau matching failed (those cells
 * are copied without collision and get NaN fields).
 */
long ora_step(int order, int q, const int* v, const double* p0, const double* w, int nx, int ny, int nz,
              const int* bc, double eta_over_s, double tau_prime, int tau_local_T, double T_ref, double dx_fm,
              double T_unit_GeV, int pull, int collide, const double* fin, double* fout, double* fields,
              double* dens) {
  const double R = (order == 3) ? sqrt(41.0) : 3.0;
  const double kappa = T_unit_GeV * dx_fm / ORA_HBARC_GEV_FM;
  const size_t cells = (size_t)nx * ny * nz;
  long bad = 0;
  double ft[ORA_QMAX], feq[ORA_QMAX];
  for (long z = 0; z < nz; ++z)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x) {
        const size_t c = ((size_t)z * ny + y) * nx + x;
        for (int i = 0; i < q; ++i) {
          long sx = x, sy = y, sz = z;
          if (pull) {
            sx = wrap_index(x - v[3 * i + 0], nx, bc[0]);
            sy = wrap_index(y - v[3 * i + 1], ny, bc[1]);
            sz = wrap_index(z - v[3 * i + 2], nz, bc[2]);
          }
          ft[i] = fin[(size_t)i * cells + ((size_t)sz * ny + sy) * nx + sx];
        }
        double N[4], Tm[16], U[4], eps = NAN, n = NAN;
        ora_moments_cell(order, q, v, p0, ft, N, Tm);
        if (dens) {
          dens[0 * cells + c] = N[0];
          for (int b = 0; b < 4; ++b) dens[(1 + b) * cells + c] = Tm[b];
        }
        const int st = ora_landau_cell(N, Tm, U, &eps, &n);
        if (st != ORA_OK) {
          ++bad;
          if (fields)
            for (int k = 0; k < 6; ++k) fields[k * cells + c] = NAN;
          if (collide)
            for (int i = 0; i < q; ++i) fout[(size_t)i * cells + c] = ft[i];
          continue;
        }
        const double T = eps / (3.0 * n); /* equation of state eps = 3 n T */
        if (fields) {
          fields[0 * cells + c] = n;
          fields[1 * cells + c] = eps;
          for (int a = 0; a < 4; ++a) fields[(2 + a) * cells + c] = U[a];
        }
        if (!collide) continue;
        const double tau =
            (tau_prime > 0.5) ? tau_prime : ora_tau_prime(eta_over_s, R, kappa, tau_local_T ? T : T_ref);
        ora_equilibrium_cell(order, q, v, p0, w, n, T, U, feq);
        for (int i = 0; i < q; ++i) {
          /* p_i^mu U_mu / p_i^0 = U0 - (v_i . U) / R */
          const double pu = U[0] - (v[3 * i] * U[1] + v[3 * i + 1] * U[2] + v[3 * i + 2] * U[3]) / R;
          fout[(size_t)i * cells + c] = ft[i] - pu / tau * (ft[i] - feq[i]);
        }
      }
  return bad;
}

/* f_i = f_i^eq(n, T, u) on every cell; U = gamma (1, u).  Returns ORA_EINVAL if |u| >= 1. */
int ora_init(int order, int q, const int* v, const double* p0, const double* w, long cells, const double* n,
             const double* T, const double* u, double* f) {
  double feq[ORA_QMAX];
  for (long c = 0; c < cells; ++c) {
    const double ux = u[c], uy = u[cells + c], uz = u[2 * cells + c];
    const double u2 = ux * ux + uy * uy + uz * uz;
    if (!(u2 < 1.0) || !(T[c] > 0.0) || !(n[c] > 0.0)) return ORA_EINVAL;
    const double g = 1.0 / sqrt(1.0 - u2);
    const double U[4] = {g, g * ux, g * uy, g * uz};
    ora_equilibrium_cell(order, q, v, p0, w, n[c], T[c], U, feq);
    for (int i = 0; i < q; ++i) f[(size_t)i * cells + c] = feq[i];
  }
  return ORA_OK;
}
