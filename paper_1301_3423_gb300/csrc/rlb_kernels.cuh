// Kernels of the relativistic lattice Boltzmann step (arXiv:1301.3423) for sm_103a.
//
// One thread owns one cell.  A step (Eq. (rlb:disc)) is a single fused pass per cell:
//   pull    f~_i(x) = f_i(x - v_i)                     one read per population
//   moments N^mu, T^{mu nu} over mirror pairs         (Sec. II.D)
//   Landau  T^{ab} U_b = eps U^a, n = U.N, T = eps/(3n) (Eq. (eigenproblem))
//   tau'    from eta/s and T                           (Sec. II.D, Sec. III)
//   f^eq    E(p0, t), t = v.U/R, as a cubic in t per energy level (App. B, Eq. (eq:equi3rd) /
//           (eq:equi2nd) regrouped)
//   collide f_i - (U0 - t_i)/tau' (f_i - w_i E_i)      one write per population
// The cells of a step are split over two launches: rows whose y and z are interior (constant
// offsets, or x wrapped only, per 32-aligned warp segment) and the boundary rows (k_step_shell_rows;
// k_step_shell per cell for lattices shorter than the stencil reach).  Batched steps use the same
// split across many lattices (k_step_batch).
//
// The quadrature is a compile-time table (generated rlb_quadrature.h), so every per-population
// constant (velocity components, energy, weight, mirror partner) is an immediate.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "rlb_common.h"
#include "rlb_quadrature.h"

namespace rlb {

// ---------------------------------------------------------------------------------------------
// compile-time loop
// ---------------------------------------------------------------------------------------------
template <int... Is, class F>
__device__ __forceinline__ void sfor_impl(std::integer_sequence<int, Is...>, F& f) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  sfor_impl(std::make_integer_sequence<int, N>{}, f);
}
template <int I>
using ic = std::integral_constant<int, I>;

// ---------------------------------------------------------------------------------------------
// storage formats
// ---------------------------------------------------------------------------------------------
struct StoreF64 {
  using T = double;
  using A = double;                 // arithmetic of the step
  static constexpr bool kKeep = false;  // 128 doubles do not fit the register file: reload
  template <class L, int I>
  __device__ static __forceinline__ A load(const T* p, const StepParams&) { return __ldg(p); }
  template <class L, int I>
  __device__ static __forceinline__ void store(T* p, A v, const StepParams&) { *p = v; }
  template <class L, int I>
  __device__ static __forceinline__ double to_f64(T v, const StepParams&) { return v; }
  template <class L, int I>
  __device__ static __forceinline__ T from_f64(double v, const StepParams&) { return v; }
};

struct StoreF32 {
  using T = float;
  using A = float;
  static constexpr bool kKeep = true;   // all populations of a cell live in registers
  // Each population is read once per step: cached in L2 only, leaving L1 to the register spills
  // (measured 4.7 % faster at 256^3 than loads that also allocate in L1).
  template <class L, int I>
  __device__ static __forceinline__ A load(const T* p, const StepParams&) { return __ldcg(p); }
  template <class L, int I>
  __device__ static __forceinline__ void store(T* p, A v, const StepParams&) { *p = v; }
  template <class L, int I>
  __device__ static __forceinline__ double to_f64(T v, const StepParams&) { return (double)v; }
  template <class L, int I>
  __device__ static __forceinline__ T from_f64(double v, const StepParams&) { return (float)v; }
};

// Half-precision deviation d_i = f_i / w_i - n_ref / 2 from the weight-scaled rest equilibrium.
struct StoreF16Dev {
  using T = __half;
  using A = float;
  static constexpr bool kKeep = true;
  template <class L, int I>
  __device__ static __forceinline__ A load(const T* p, const StepParams& sp) {
    constexpr float w = (float)L::W[I];
    return w * (__half2float(__ldg(p)) + sp.half_nref);
  }
  template <class L, int I>
  __device__ static __forceinline__ void store(T* p, A v, const StepParams& sp) {
    constexpr float iw = (float)(1.0 / L::W[I]);
    *p = __float2half_rn(fmaf(v, iw, -sp.half_nref));
  }
  // the deviation d_i itself (the step kernels work in deviation space)
  template <class L, int I>
  __device__ static __forceinline__ A load_dev(const T* p, const StepParams&) { return __half2float(__ldg(p)); }
  template <class L, int I>
  __device__ static __forceinline__ void store_dev(T* p, A d, const StepParams&) { *p = __float2half_rn(d); }
  template <class L, int I>
  __device__ static __forceinline__ double to_f64(T v, const StepParams& sp) {
    constexpr double w = L::W[I];
    return w * ((double)__half2float(v) + (double)sp.half_nref);
  }
  template <class L, int I>
  __device__ static __forceinline__ T from_f64(double v, const StepParams& sp) {
    constexpr double iw = 1.0 / L::W[I];
    return __float2half_rn((float)(v * iw - (double)sp.half_nref));
  }
};

// ---------------------------------------------------------------------------------------------
// cell geometry and the pull source index
// ---------------------------------------------------------------------------------------------
struct Cell {
  int c, x, y, z;
};

__device__ __forceinline__ Cell make_cell(int c, const StepParams& p) {
  Cell r;
  r.c = c;
  const int yz = c / p.nx;
  r.x = c - yz * p.nx;
  r.z = yz / p.ny;
  r.y = yz - r.z * p.ny;
  return r;
}

// Source coordinate of x - v along an axis of n cells: periodic wrap or copy-out clamp.
// GENERAL handles n < |v| (a full modulo); otherwise one conditional wrap suffices.
template <int V, bool GENERAL>
__device__ __forceinline__ int src_coord(int x, int n, int bc) {
  if constexpr (V == 0) {
    return x;
  } else {
    int s = x - V;
    if (bc) return (V > 0) ? max(s, 0) : min(s, n - 1);
    if constexpr (GENERAL) {
      s %= n;
      return s < 0 ? s + n : s;
    } else {
      if constexpr (V > 0) return s < 0 ? s + n : s;
      else return s >= n ? s - n : s;
    }
  }
}

// src_coord with the shift v known only at run time (one conditional wrap: n >= |v|).
__device__ __forceinline__ int src_coord_rt(int x, int v, int n, int bc) {
  const int s = x - v;
  if ((unsigned)s < (unsigned)n) return s;
  if (bc) return s < 0 ? 0 : n - 1;
  return s < 0 ? s + n : s - n;
}

// The populations' velocities as a table in constant memory, for loops over the populations with
// a run-time index.
template <class L>
struct VelTab {
  signed char v[L::Q][3];
};
template <class L>
constexpr VelTab<L> make_vel_tab() {
  VelTab<L> t{};
  for (int i = 0; i < L::Q; ++i) {
    t.v[i][0] = (signed char)L::VX[i];
    t.v[i][1] = (signed char)L::VY[i];
    t.v[i][2] = (signed char)L::VZ[i];
  }
  return t;
}
template <class L>
__constant__ VelTab<L> kVelTab = make_vel_tab<L>();

// Pull offsets of one shell row (fixed y, z): for every population the constant offset plus the
// row's y and z wrap (or clamp) shifts, worked out once per row by the warp's 32 lanes (four
// populations each) into roff[Q]; the warp's cells then add only their x shift.  Lattices with
// bounce-back walls take shell_row_offset per population instead.
template <class L>
__device__ __forceinline__ void shell_row_table(long long* roff, const Cell& cl, const StepParams& p) {
  for (int i = threadIdx.x & 31; i < L::Q; i += 32) {
    const int vy = kVelTab<L>.v[i][1], vz = kVelTab<L>.v[i][2];
    long long o = p.off[i];
    o += (long long)(src_coord_rt(cl.y, vy, p.ny, p.bc[1]) - (cl.y - vy)) * p.nx;
    o += (long long)(src_coord_rt(cl.z, vz, p.nz, p.bc[2]) - (cl.z - vz)) * p.nxy;
    roff[i] = o;
  }
  __syncwarp();
}

// True if the pull source of population I lies beyond a bounce-back wall (then the cell takes its
// own population of the reversed momentum, I ^ 1: mirror pairs are adjacent).
template <class L, int I>
__device__ __forceinline__ bool beyond_wall(const Cell& cl, const StepParams& p) {
  constexpr int vx = L::VX[I], vy = L::VY[I], vz = L::VZ[I];
  bool b = false;
  if constexpr (vx != 0) b = b || (p.bc[0] == kBounceBack && (unsigned)(cl.x - vx) >= (unsigned)p.nx);
  if constexpr (vy != 0) b = b || (p.bc[1] == kBounceBack && (unsigned)(cl.y - vy) >= (unsigned)p.ny);
  if constexpr (vz != 0) b = b || (p.bc[2] == kBounceBack && (unsigned)(cl.z - vz) >= (unsigned)p.nz);
  return b;
}

// WALLS = false compiles the bounce-back test out: kernels for lattices without walls pay nothing.
template <class L, int I, bool GENERAL, bool WALLS>
__device__ __forceinline__ long long pull_index(const Cell& cl, const StepParams& p) {
  constexpr int vx = L::VX[I], vy = L::VY[I], vz = L::VZ[I];
  if constexpr (WALLS) {
    if (p.has_wall && beyond_wall<L, I>(cl, p)) return (long long)(I ^ 1) * p.cells + cl.c;
  }
  const int sx = src_coord<vx, GENERAL>(cl.x, p.nx, p.bc[0]);
  const int sy = src_coord<vy, GENERAL>(cl.y, p.ny, p.bc[1]);
  const int sz = src_coord<vz, GENERAL>(cl.z, p.nz, p.bc[2]);
  return (long long)I * p.cells + (long long)(sz * p.nxy + sy * p.nx + sx);
}


// Pull offset of population I from the cell's own index when only the x coordinate can leave the
// lattice (rows whose y and z are interior): the constant offset with x wrapped or clamped, or the
// cell's own reversed population beyond a bounce-back wall in x.
template <class L, int I, bool WALLS>
__device__ __forceinline__ long long x_row_offset(const Cell& cl, const StepParams& p) {
  constexpr int vx = L::VX[I];
  if constexpr (WALLS && vx != 0) {
    if (p.bc[0] == kBounceBack && (unsigned)(cl.x - vx) >= (unsigned)p.nx) return (long long)(I ^ 1) * p.cells;
  }
  return p.off[I] + (src_coord<vx, false>(cl.x, p.nx, p.bc[0]) - (cl.x - vx));
}

// ---------------------------------------------------------------------------------------------
// moments N^mu, T^{mu nu} (Eqs. (moments:dis1), (moments:dis2)), accumulated over mirror pairs:
// for a pair (v, -v) at energy p0, s1 = p0 (f+ +- f-), s2 = p0^2 (f+ +- f-).
// ---------------------------------------------------------------------------------------------
template <class A>
struct Mom {
  A N0, Nx, Ny, Nz, T00, T0x, T0y, T0z, Txx, Tyy, Tzz, Txy, Txz, Tyz;
};

// Moments of the weights alone, sum_i w_i k_i for the moment kernels k_i of N^0, T^00 and T^ab:
// in deviation space (f_i = w_i (d_i + c)) the constant c contributes c times these.  The odd
// moments cancel exactly between mirror partners.
template <class L>
struct RestSums {
  static constexpr double sum(int e, int a, int b) {  // sum_i w_i p0^e (v_a v_b / R^2 if a >= 0)
    double s = 0.0;
    for (int i = 0; i < L::Q; ++i) {
      const double p = L::P0[L::LEV[i]];
      const double v[3] = {(double)L::VX[i], (double)L::VY[i], (double)L::VZ[i]};
      double t = L::W[i] * (e == 1 ? p : p * p);
      if (a >= 0) t *= v[a] * v[b] * L::INV_R2;
      s += t;
    }
    return s;
  }
  static constexpr double N0 = sum(1, -1, -1), T00 = sum(2, -1, -1), Txx = sum(2, 0, 0), Tyy = sum(2, 1, 1),
                          Txy = sum(2, 0, 1), Txz = sum(2, 0, 2), Tyz = sum(2, 1, 2);
};

template <class L, class A>
__device__ __forceinline__ void add_rest_sums(Mom<A>& m, A c) {
  m.N0 = fma(A(RestSums<L>::N0), c, m.N0);
  m.T00 = fma(A(RestSums<L>::T00), c, m.T00);
  m.Txx = fma(A(RestSums<L>::Txx), c, m.Txx);
  m.Tyy = fma(A(RestSums<L>::Tyy), c, m.Tyy);
  m.Txy = fma(A(RestSums<L>::Txy), c, m.Txy);
  m.Txz = fma(A(RestSums<L>::Txz), c, m.Txz);
  m.Tyz = fma(A(RestSums<L>::Tyz), c, m.Tyz);
}

// DEV = true: get returns deviations d_i = f_i / w_i - c, and the moments are those of
// f_i = w_i (d_i + c).
template <class L, class A, bool DEV = false, class Get>
__device__ __forceinline__ Mom<A> moments(Get&& get, A c = A(0)) {
  Mom<A> m;
  m.N0 = m.Nx = m.Ny = m.Nz = A(0);
  m.T00 = m.T0x = m.T0y = m.T0z = A(0);
  m.Txx = m.Tyy = m.Txy = m.Txz = m.Tyz = A(0);
  static_for<L::NDP>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int first = L::DP_FIRST[k];
    constexpr int np = L::DP_NPAIR[k];
    A s1p = A(0), s1m = A(0), s2p = A(0), s2m = A(0);
    static_for<np>([&](auto J) {
      constexpr int ip = first + 2 * decltype(J)::value;
      constexpr double wk = DEV ? L::W[ip] : 1.0;  // mirror partners share the weight
      constexpr double p0 = L::P0[L::LEV[ip]];
      const A fa = get(ic<ip>{});
      const A fb = get(ic<ip + 1>{});
      const A sp = fa + fb, sm = fa - fb;
      s1p = fma(A(wk * p0), sp, s1p);
      s1m = fma(A(wk * p0), sm, s1m);
      s2p = fma(A(wk * p0 * p0), sp, s2p);
      s2m = fma(A(wk * p0 * p0), sm, s2m);
    });
    constexpr int vx = L::VX[first], vy = L::VY[first], vz = L::VZ[first];
    constexpr double ir = L::INV_R, ir2 = L::INV_R2;
    m.N0 += s1p;
    m.T00 += s2p;
    if constexpr (vx != 0) {
      m.Nx = fma(A(vx * ir), s1m, m.Nx);
      m.T0x = fma(A(vx * ir), s2m, m.T0x);
      m.Txx = fma(A(vx * vx * ir2), s2p, m.Txx);
    }
    if constexpr (vy != 0) {
      m.Ny = fma(A(vy * ir), s1m, m.Ny);
      m.T0y = fma(A(vy * ir), s2m, m.T0y);
      m.Tyy = fma(A(vy * vy * ir2), s2p, m.Tyy);
    }
    if constexpr (vz != 0) {
      m.Nz = fma(A(vz * ir), s1m, m.Nz);
      m.T0z = fma(A(vz * ir), s2m, m.T0z);
    }
    if constexpr (vx != 0 && vy != 0) m.Txy = fma(A(vx * vy * ir2), s2p, m.Txy);
    if constexpr (vx != 0 && vz != 0) m.Txz = fma(A(vx * vz * ir2), s2p, m.Txz);
    if constexpr (vy != 0 && vz != 0) m.Tyz = fma(A(vy * vz * ir2), s2p, m.Tyz);
  });
  if constexpr (DEV) add_rest_sums<L, A>(m, c);
  // |v|^2 = R^2 for every velocity, so the spatial trace of T equals T^00.
  m.Tzz = m.T00 - m.Txx - m.Tyy;
  return m;
}

template <class A, class B>
__device__ __forceinline__ Mom<B> convert(const Mom<A>& a) {
  return Mom<B>{B(a.N0),  B(a.Nx),  B(a.Ny),  B(a.Nz),  B(a.T00), B(a.T0x), B(a.T0y),
                B(a.T0z), B(a.Txx), B(a.Tyy), B(a.Tzz), B(a.Txy), B(a.Txz), B(a.Tyz)};
}

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }

// ---------------------------------------------------------------------------------------------
// Landau matching (Eq. (eigenproblem), Sec. II.D).  U is the timelike eigenvector of
// T^a_b = T^{ac} eta_{cb}.  Shifted power iteration started from the Eckart vector N/|N|:
//   V = T.(eta U),  rho = U.V,  W = V + (rho/3) U,  U <- W / |W|.
// The shift rho/3 moves the spacelike eigenvalues -P_k to rho/3 - P_k, which vanish in local
// equilibrium (eps = 3P), so the contraction factor is the relative pressure anisotropy instead
// of P/eps = 1/3.  eps is the Rayleigh quotient U.V, n = U.N.  Each lane stops once converged (a
// warp runs as long as its slowest cell).
// ---------------------------------------------------------------------------------------------
template <class A>
struct Landau {
  A U0, Ux, Uy, Uz, eps, n;
  bool ok;    // a timelike frame with eps > 0 and n > 0
  bool conv;  // the last update moved U by at most tol * U0 (false: stopped at MAXIT)
};

// Shifted power iteration from the start vector (U0, Ux, Uy, Uz), at most MAXIT updates; a lane
// stops once an update moves U by at most tol * U0.
template <class A, int MAXIT>
__device__ __forceinline__ Landau<A> landau_from(const Mom<A>& m, A U0, A Ux, A Uy, A Uz, const A tol) {
  Landau<A> r;
  r.ok = false;
  r.conv = false;
  for (int it = 0; it < MAXIT; ++it) {
    const A V0 = m.T00 * U0 - m.T0x * Ux - m.T0y * Uy - m.T0z * Uz;
    const A Vx = m.T0x * U0 - m.Txx * Ux - m.Txy * Uy - m.Txz * Uz;
    const A Vy = m.T0y * U0 - m.Txy * Ux - m.Tyy * Uy - m.Tyz * Uz;
    const A Vz = m.T0z * U0 - m.Txz * Ux - m.Tyz * Uy - m.Tzz * Uz;
    const A s = (U0 * V0 - Ux * Vx - Uy * Vy - Uz * Vz) * A(1.0 / 3.0);
    const A W0 = fma(s, U0, V0), Wx = fma(s, Ux, Vx), Wy = fma(s, Uy, Vy), Wz = fma(s, Uz, Vz);
    const A WW = W0 * W0 - Wx * Wx - Wy * Wy - Wz * Wz;
    if (!(WW > A(0)) || !(W0 > A(0))) return r;
    const A iw = rsqrt_(WW);
    const A n0 = W0 * iw, nx = Wx * iw, ny = Wy * iw, nz = Wz * iw;
    const A d = fmax(fmax(fabs(n0 - U0), fabs(nx - Ux)), fmax(fabs(ny - Uy), fabs(nz - Uz)));
    U0 = n0; Ux = nx; Uy = ny; Uz = nz;
    if (d <= tol * U0) {
      r.conv = true;
      break;
    }
  }
  const A V0 = m.T00 * U0 - m.T0x * Ux - m.T0y * Uy - m.T0z * Uz;
  const A Vx = m.T0x * U0 - m.Txx * Ux - m.Txy * Uy - m.Txz * Uz;
  const A Vy = m.T0y * U0 - m.Txy * Ux - m.Tyy * Uy - m.Tyz * Uz;
  const A Vz = m.T0z * U0 - m.Txz * Ux - m.Tyz * Uy - m.Tzz * Uz;
  r.eps = U0 * V0 - Ux * Vx - Uy * Vy - Uz * Vz;
  r.n = U0 * m.N0 - Ux * m.Nx - Uy * m.Ny - Uz * m.Nz;
  r.U0 = U0; r.Ux = Ux; r.Uy = Uy; r.Uz = Uz;
  r.ok = (r.eps > A(0)) && (r.n > A(0)) && isfinite(r.eps) && isfinite(r.n);
  return r;
}

// Landau matching from the Eckart vector N / |N|; double stops at 8e-16 U0 (a few units in the last
// place), float at 3e-7 U0.
template <class A, int MAXIT>
__device__ __forceinline__ Landau<A> landau(const Mom<A>& m) {
  const A NN = m.N0 * m.N0 - m.Nx * m.Nx - m.Ny * m.Ny - m.Nz * m.Nz;
  if (!(NN > A(0)) || !(m.N0 > A(0))) {
    Landau<A> r;
    r.ok = false;
    r.conv = false;
    return r;
  }
  const A is = rsqrt_(NN);
  const A tol = std::is_same<A, double>::value ? A(8e-16) : A(3e-7);
  return landau_from<A, MAXIT>(m, m.N0 * is, m.Nx * is, m.Ny * is, m.Nz * is, tol);
}

// The double-precision solve of a float step, kept out of line: it runs for few cells and would
// otherwise grow the step kernel's hot code (a call keeps the caller's register allocation that of
// the float path).  It starts from the Eckart vector and stops at 1e-12 U0: the populations are
// float, so more digits carry no information, while the double arithmetic still removes the
// gamma^2 cancellation in U.U = 1.
static __device__ __noinline__ Landau<double> landau_fp64_out_of_line(const Mom<double> m) {
  const double NN = m.N0 * m.N0 - m.Nx * m.Nx - m.Ny * m.Ny - m.Nz * m.Nz;
  if (!(NN > 0.0) || !(m.N0 > 0.0)) {
    Landau<double> r;
    r.ok = false;
    r.conv = false;
    return r;
  }
  const double is = rsqrt(NN);
  Landau<double> r = landau_from<double, 40>(m, m.N0 * is, m.Nx * is, m.Ny * is, m.Nz * is, 1e-12);
  r.ok = r.ok && r.conv;  // no frame to 1e-12 in 40 double updates: reported, not used
  return r;
}

// Landau matching in the step's arithmetic A.  Reduced-precision paths switch to double for cells
// whose Eckart Lorentz factor exceeds gamma_thr (or always, if asked): the solve loses about
// gamma^2 digits to cancellation in U.U = 1.
// A double solve that stops at MAXIT without meeting its tolerance is accepted only if the last
// update was below 1e-10 U0 (round-off can keep the last digits moving); a float solve that does
// not converge in 8 updates is redone in double.
template <class A>
__device__ __forceinline__ Landau<A> landau_step(const Mom<A>& m, const StepParams& p) {
  if constexpr (std::is_same<A, double>::value) {
    Landau<double> r = landau<double, 40>(m);
    if (r.ok && !r.conv) {
      const Landau<double> again = landau_from<double, 1>(m, r.U0, r.Ux, r.Uy, r.Uz, 1e-10);
      r.ok = again.ok && again.conv;
    }
    return r;
  } else {
    const float NN = m.N0 * m.N0 - m.Nx * m.Nx - m.Ny * m.Ny - m.Nz * m.Nz;
    Landau<float> r;
    const bool dbl = p.landau_fp64 || m.N0 * m.N0 > p.gamma_thr2 * NN;
    if (!dbl) {
      r = landau<float, 8>(m);
      if (r.conv || !r.ok) return r;
    }
    const Landau<double> d = landau_fp64_out_of_line(convert<A, double>(m));
    return Landau<A>{(A)d.U0, (A)d.Ux, (A)d.Uy, (A)d.Uz, (A)d.eps, (A)d.n, d.ok, d.conv};
  }
}

template <class A>
__device__ __forceinline__ A tau_prime(A T, const StepParams& p) {
  if constexpr (std::is_same<A, double>::value) {
    if (p.tau_is_fixed) return p.tau_fixed;
    const double Tt = p.tau_local ? T : p.T_ref;
    return 0.5 + p.tau_coef / Tt;
  } else {
    if (p.tau_is_fixed) return p.tau_fixed_f;
    const float Tt = p.tau_local ? T : p.T_ref_f;
    return 0.5f + p.tau_coef_f / Tt;
  }
}

// ---------------------------------------------------------------------------------------------
// Equilibrium in factored form.  The projection of the Maxwell-Juttner distribution onto the
// polynomials of degree <= order depends on p only through p0 and s = p.U (rotational symmetry
// about U), so f_i^eq = w_i E(p0_i, t_i) with s = p0 t, t = v.U/R, and, with x = T U0 - 1:
//   order 3:  E = n/(12T) [c00 + p0 (c10 + c01 t) + p0^2 (c20 + c11 t + c02 t^2) + p0^3 (x + T t)^3]
//   order 2:  E = n/(4T)  [c00 + p0 (c10 + c01 t) + p0^2 (x + T t)^2]
// which is App. B's Eq. (eq:equi3rd) / (eq:equi2nd) regrouped.
// ---------------------------------------------------------------------------------------------
template <int ORDER, class A>
struct EqCoef {
  A c00, c10, c01, c20, c11, c02, x, T, pref;
};

template <int ORDER, class A>
__device__ __forceinline__ EqCoef<ORDER, A> eq_coef(A n, A T, A U0) {
  EqCoef<ORDER, A> c;
  const A x = fma(T, U0, A(-1));
  const A x2 = x * x, T2 = T * T;
  c.x = x;
  c.T = T;
  if constexpr (ORDER == 3) {
    const A pref = n / (A(12) * T);
    c.pref = pref;
    c.c00 = A(-6) * pref * (fma(x2, fma(A(8), x, A(4)), fma(A(4), x, A(-2))) + T2 * fma(A(-4), x, A(1)));
    c.c10 = A(6) * pref * (fma(x2, fma(A(12), x, A(8)), fma(A(5), x, A(-1))) + T2 * fma(A(-6), x, A(1)));
    c.c01 = A(6) * pref * T * (fma(A(12), x2, A(3)) - A(2) * T2);
    c.c20 = A(-3) * pref * x * (fma(x, fma(A(6), x, A(3)), A(2)) - A(2) * T2);
    c.c11 = A(-6) * pref * T * (fma(x, fma(A(6), x, A(1)), A(1)) - T2);
    c.c02 = A(-3) * pref * T2 * fma(A(6), x, A(-1));
  } else {
    const A pref = n / (A(4) * T);
    c.pref = pref;
    c.c00 = A(2) * pref * (fma(A(4), x2, A(2)) - T2);
    c.c10 = A(-2) * pref * (fma(x, fma(A(4), x, A(1)), A(1)) - T2);
    c.c01 = A(-2) * pref * T * fma(A(4), x, A(-1));
    c.c20 = c.c11 = c.c02 = A(0);
  }
  return c;
}

// Pull offset of population I from the cell's own index in a shell row: the constant offset plus
// the y and z wrap (or clamp) shifts of the row, plus the x shift unless the warp's x segment is
// interior; the cell's own reversed population beyond a bounce-back wall.
template <class L, int I, bool WALLS>
__device__ __forceinline__ long long shell_row_offset(const Cell& cl, const StepParams& p, const bool xfast) {
  constexpr int vx = L::VX[I], vy = L::VY[I], vz = L::VZ[I];
  if constexpr (WALLS) {
    if (p.has_wall && beyond_wall<L, I>(cl, p)) return (long long)(I ^ 1) * p.cells;
  }
  long long o = p.off[I];
  if constexpr (vy != 0) o += (long long)(src_coord<vy, false>(cl.y, p.ny, p.bc[1]) - (cl.y - vy)) * p.nx;
  if constexpr (vz != 0) o += (long long)(src_coord<vz, false>(cl.z, p.nz, p.bc[2]) - (cl.z - vz)) * p.nxy;
  if constexpr (vx != 0) {
    if (!xfast) o += src_coord<vx, false>(cl.x, p.nx, p.bc[0]) - (cl.x - vx);
  }
  return o;
}

// The equilibrium as a polynomial in t per energy level l (p0 = p0_l):
//   E(p0_l, t) = a_l + t (b_l + t (c_l + t d_l)),
//   order 3: a = c00 + p0 c10 + p0^2 c20 + pref p0^3 x^3,  b = p0 c01 + p0^2 c11 + 3 pref p0^3 x^2 T,
//            c = p0^2 c02 + 3 pref p0^3 x T^2,             d = pref p0^3 T^3;
//   order 2: a = c00 + p0 c10 + pref p0^2 x^2,  b = p0 c01 + 2 pref p0^2 x T,  c = pref p0^2 T^2,  d = 0.
// The same regrouping of App. B's forms: the per-cell work moves from the 48 (15) directions to
// the 4 (3) energy levels, and each population costs a cubic (quadratic) Horner step in t.
template <class L, class A>
struct LevCoef {
  A a[L::NLEV], b[L::NLEV], c[L::NLEV], d[L::NLEV];
};

// shift: subtracted from every a_l (deviation space evaluates E - c)
template <class L, class A>
__device__ __forceinline__ LevCoef<L, A> level_coef(const EqCoef<L::ORDER, A>& q, A shift = A(0)) {
  LevCoef<L, A> r;
  static_for<L::NLEV>([&](auto K) {
    constexpr int l = decltype(K)::value;
    constexpr double pd = L::P0[l];
    const A p = A(pd), p2 = A(pd * pd);
    if constexpr (L::ORDER == 3) {
      const A pp3 = A(pd * pd * pd) * q.pref;  // pref p0^3
      const A ppx = pp3 * q.x;
      r.d[l] = pp3 * (q.T * q.T * q.T);
      r.c[l] = fma(A(3) * ppx, q.T * q.T, p2 * q.c02);
      r.b[l] = fma(A(3) * ppx * q.x, q.T, fma(p2, q.c11, p * q.c01));
      r.a[l] = fma(ppx * q.x, q.x, fma(p2, q.c20, fma(p, q.c10, q.c00 - shift)));
    } else {
      const A pp2 = p2 * q.pref;  // pref p0^2
      r.d[l] = A(0);
      r.c[l] = pp2 * (q.T * q.T);
      r.b[l] = fma(A(2) * pp2 * q.x, q.T, p * q.c01);
      r.a[l] = fma(pp2 * q.x, q.x, fma(p, q.c10, q.c00 - shift));
    }
  });
  return r;
}

// Collision of one cell (Eq. (rlb:disc) right-hand side, delta t' = 1):
//   f*_i = f_i + omega_i (w_i E_i - f_i),  omega_i = p_i.U / (tau' p0_i) = (U0 - t_i) / tau'.
// DEV = true: get / put carry deviations d_i = f_i / w_i - c, and the collision is
// d_i + omega_i ((E_i - c) - d_i).
template <class L, class A, bool DEV = false, class Get, class Put>
__device__ __forceinline__ void collide(const Landau<A>& lw, A T, A inv_tau, Get&& get, Put&& put, A c = A(0)) {
  const LevCoef<L, A> e = level_coef<L, A>(eq_coef<L::ORDER, A>(lw.n, T, lw.U0), DEV ? c : A(0));
  const A a = lw.U0 * inv_tau;
  static_for<L::NDP>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int first = L::DP_FIRST[k];
    constexpr int np = L::DP_NPAIR[k];
    constexpr int vx = L::VX[first], vy = L::VY[first], vz = L::VZ[first];
    constexpr double ir = L::INV_R;
    A t = A(0);  // direction +v: t; mirror -v: -t
    if constexpr (vx != 0) t = fma(A(vx * ir), lw.Ux, t);
    if constexpr (vy != 0) t = fma(A(vy * ir), lw.Uy, t);
    if constexpr (vz != 0) t = fma(A(vz * ir), lw.Uz, t);
    const A omp = fma(-t, inv_tau, a), omm = fma(t, inv_tau, a);
    static_for<np>([&](auto J) {
      constexpr int ip = first + 2 * decltype(J)::value;
      constexpr int l = L::LEV[ip];
      constexpr double wd = L::W[ip];
      const A w = A(wd);
      A Ep, Em;
      if constexpr (L::ORDER == 3) {
        Ep = fma(t, fma(t, fma(t, e.d[l], e.c[l]), e.b[l]), e.a[l]);
        Em = fma(-t, fma(-t, fma(-t, e.d[l], e.c[l]), e.b[l]), e.a[l]);
      } else {
        Ep = fma(t, fma(t, e.c[l], e.b[l]), e.a[l]);
        Em = fma(-t, fma(-t, e.c[l], e.b[l]), e.a[l]);
      }
      const A fp = get(ic<ip>{}), fm = get(ic<ip + 1>{});
      if constexpr (DEV) {
        put(ic<ip>{}, fma(omp, Ep - fp, fp));
        put(ic<ip + 1>{}, fma(omm, Em - fm, fm));
        (void)w;
      } else {
        put(ic<ip>{}, fma(omp, fma(w, Ep, -fp), fp));
        put(ic<ip + 1>{}, fma(omm, fma(w, Em, -fm), fm));
      }
    });
  });
}

// ---------------------------------------------------------------------------------------------
// Float arithmetic in mirror pairs.  Populations i (direction +v) and i + 1 (direction -v) share
// energy and weight, so their work is one float2 operation (sm_100+ paired FP32 FMA):
// moments accumulate per sign with sign-symmetric constants, and the equilibrium and collision of
// the pair are evaluated together with t2 = (t, -t).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Sums of the direction pairs [DPB, DPE) in paired arithmetic: the 13 independent moments before
// the weights' own moments (deviation space) and the trace identity are added (finish_moments_f2).
template <class L, bool DEV = false, int DPB = 0, int DPE = L::NDP, class Get2>
__device__ __forceinline__ Mom<float> moments_f2_part(Get2&& get2) {
  const float2 z = f2(0.f, 0.f);
  float2 N0 = z, Nx = z, Ny = z, Nz = z, T00 = z, T0x = z, T0y = z, T0z = z, Txx = z, Tyy = z, Txy = z, Txz = z, Tyz = z;
  static_for<DPE - DPB>([&](auto K) {
    constexpr int k = DPB + decltype(K)::value;
    constexpr int first = L::DP_FIRST[k];
    constexpr int np = L::DP_NPAIR[k];
    float2 S1 = z, S2 = z;  // (sum over energies for +v, for -v)
    static_for<np>([&](auto J) {
      constexpr int ip = first + 2 * decltype(J)::value;
      constexpr double wk = DEV ? L::W[ip] : 1.0;  // mirror partners share the weight
      constexpr float p0 = (float)(wk * L::P0[L::LEV[ip]]);
      constexpr float p02 = (float)(wk * L::P0[L::LEV[ip]] * L::P0[L::LEV[ip]]);
      const float2 f = get2(ic<ip>{});
      S1 = ffma2(f2(p0, p0), f, S1);
      S2 = ffma2(f2(p02, p02), f, S2);
    });
    constexpr int vx = L::VX[first], vy = L::VY[first], vz = L::VZ[first];
    constexpr double ir = L::INV_R, ir2 = L::INV_R2;
    N0 = fadd2(N0, S1);
    T00 = fadd2(T00, S2);
    if constexpr (vx != 0) {
      constexpr float c = (float)(vx * ir);
      constexpr float cc = (float)(vx * vx * ir2);
      Nx = ffma2(f2(c, -c), S1, Nx);
      T0x = ffma2(f2(c, -c), S2, T0x);
      Txx = ffma2(f2(cc, cc), S2, Txx);
    }
    if constexpr (vy != 0) {
      constexpr float c = (float)(vy * ir);
      constexpr float cc = (float)(vy * vy * ir2);
      Ny = ffma2(f2(c, -c), S1, Ny);
      T0y = ffma2(f2(c, -c), S2, T0y);
      Tyy = ffma2(f2(cc, cc), S2, Tyy);
    }
    if constexpr (vz != 0) {
      constexpr float c = (float)(vz * ir);
      Nz = ffma2(f2(c, -c), S1, Nz);
      T0z = ffma2(f2(c, -c), S2, T0z);
    }
    if constexpr (vx != 0 && vy != 0) {
      constexpr float cc = (float)(vx * vy * ir2);
      Txy = ffma2(f2(cc, cc), S2, Txy);
    }
    if constexpr (vx != 0 && vz != 0) {
      constexpr float cc = (float)(vx * vz * ir2);
      Txz = ffma2(f2(cc, cc), S2, Txz);
    }
    if constexpr (vy != 0 && vz != 0) {
      constexpr float cc = (float)(vy * vz * ir2);
      Tyz = ffma2(f2(cc, cc), S2, Tyz);
    }
  });
  Mom<float> m;
  m.N0 = N0.x + N0.y;
  m.Nx = Nx.x + Nx.y;
  m.Ny = Ny.x + Ny.y;
  m.Nz = Nz.x + Nz.y;
  m.T00 = T00.x + T00.y;
  m.T0x = T0x.x + T0x.y;
  m.T0y = T0y.x + T0y.y;
  m.T0z = T0z.x + T0z.y;
  m.Txx = Txx.x + Txx.y;
  m.Tyy = Tyy.x + Tyy.y;
  m.Txy = Txy.x + Txy.y;
  m.Txz = Txz.x + Txz.y;
  m.Tyz = Tyz.x + Tyz.y;
  m.Tzz = 0.f;
  return m;
}

// The weights' own moments times c (deviation space) and T^zz from the trace identity.
template <class L, bool DEV = false>
__device__ __forceinline__ void finish_moments_f2(Mom<float>& m, float c = 0.f) {
  if constexpr (DEV) add_rest_sums<L, float>(m, c);
  m.Tzz = m.T00 - m.Txx - m.Tyy;
}

template <class L, bool DEV = false, class Get2>
__device__ __forceinline__ Mom<float> moments_f2(Get2&& get2, float c = 0.f) {
  Mom<float> m = moments_f2_part<L, DEV>(get2);
  finish_moments_f2<L, DEV>(m, c);
  return m;
}

// Collision of the direction pairs [DPB, DPE) (all of them by default).
template <class L, bool DEV = false, int DPB = 0, int DPE = L::NDP, class Get2, class Put2>
__device__ __forceinline__ void collide_f2(const Landau<float>& lw, float T, float inv_tau, Get2&& get2, Put2&& put2,
                                           float c = 0.f) {
  const LevCoef<L, float> e1 = level_coef<L, float>(eq_coef<L::ORDER, float>(lw.n, T, lw.U0), DEV ? c : 0.f);
  // the coefficients as (x, x) pairs once per cell, the operands of the paired Horner steps
  struct {
    float2 a[L::NLEV], b[L::NLEV], c[L::NLEV], d[L::NLEV];
  } e;
  static_for<L::NLEV>([&](auto K) {
    constexpr int l = decltype(K)::value;
    e.a[l] = f2(e1.a[l], e1.a[l]);
    e.b[l] = f2(e1.b[l], e1.b[l]);
    e.c[l] = f2(e1.c[l], e1.c[l]);
    e.d[l] = f2(e1.d[l], e1.d[l]);
  });
  const float a = lw.U0 * inv_tau;
  const float2 Uxp = f2(lw.Ux, lw.Ux), Uyp = f2(lw.Uy, lw.Uy), Uzp = f2(lw.Uz, lw.Uz);
  const float2 itp = f2(inv_tau, inv_tau), nap = f2(-a, -a);
  static_for<DPE - DPB>([&](auto K) {
    constexpr int k = DPB + decltype(K)::value;
    constexpr int first = L::DP_FIRST[k];
    constexpr int np = L::DP_NPAIR[k];
    constexpr int vx = L::VX[first], vy = L::VY[first], vz = L::VZ[first];
    constexpr double ir = L::INV_R;
    float2 tt = f2(0.f, 0.f);  // (t, -t), t = v.U / R
    if constexpr (vx != 0) tt = ffma2(f2((float)(vx * ir), (float)(-vx * ir)), Uxp, tt);
    if constexpr (vy != 0) tt = ffma2(f2((float)(vy * ir), (float)(-vy * ir)), Uyp, tt);
    if constexpr (vz != 0) tt = ffma2(f2((float)(vz * ir), (float)(-vz * ir)), Uzp, tt);
    const float2 nom = ffma2(itp, tt, nap);  // -(U0 - t) / tau' for +v, -(U0 + t) / tau' for -v
    static_for<np>([&](auto J) {
      constexpr int ip = first + 2 * decltype(J)::value;
      constexpr int l = L::LEV[ip];
      constexpr float nw = DEV ? -1.f : (float)(-L::W[ip]);
      float2 E;
      if constexpr (L::ORDER == 3)
        E = ffma2(tt, ffma2(tt, ffma2(tt, e.d[l], e.c[l]), e.b[l]), e.a[l]);
      else
        E = ffma2(tt, ffma2(tt, e.c[l], e.b[l]), e.a[l]);
      const float2 f = get2(ic<ip>{});
      const float2 d = ffma2(f2(nw, nw), E, f);  // f - w E (deviation space: d - (E - c))
      put2(ic<ip>{}, ffma2(nom, d, f));        // f - omega (f - w E)
    });
  });
}

// ---------------------------------------------------------------------------------------------
// the fused step kernel
// ---------------------------------------------------------------------------------------------
// Compiler-level barrier: values read from memory before it are read again after it.
__device__ __forceinline__ void reload_barrier() { asm volatile("" ::: "memory"); }

// Moments, Landau matching, relaxation time, equilibrium and collision of one cell (steps a2-a7)
// whose pulled populations get(I) returns (deviations d_i for half-deviation storage); store(I, v)
// writes post-collision population I.  Shared by every step kernel, whatever it pulls from
// (registers, global memory or a shared-memory stage).  RELOAD = true makes the collision read
// every population again through get instead of keeping the moment pass's values in registers
// (for populations staged in shared memory).  A cell without a Landau frame is counted in status
// (valid lanes only) and streamed without collision.
template <class L, class S, bool PACKED, bool RELOAD = false, class Get, class Store>
__device__ __forceinline__ void relax_cell(Get&& get, Store&& store, const StepParams& p, int* __restrict__ status,
                                           const bool valid) {
  using A = typename S::A;
  constexpr bool DEV = std::is_same<S, StoreF16Dev>::value;
  const A c_dev = DEV ? A(p.half_nref) : A(0);
  auto get2 = [&](auto I) -> float2 {
    constexpr int i = decltype(I)::value;
    return make_float2((float)get(ic<i>{}), (float)get(ic<i + 1>{}));
  };
  Mom<A> m;
  if constexpr (PACKED) m = moments_f2<L, DEV>(get2, (float)c_dev);
  else m = moments<L, A, DEV>(get, c_dev);
  if constexpr (RELOAD) reload_barrier();
  const Landau<A> lw = landau_step<A>(m, p);
  if (!lw.ok) {
    // no Landau frame: record it and stream the populations without collision
    if (valid) {
      atomicAdd(&status[kStatusNonconv], 1);
      static_for<L::Q>([&](auto I) { store(I, get(I)); });
    }
    return;
  }
  const A T = lw.eps / (A(3) * lw.n);
  const A inv_tau = A(1) / tau_prime<A>(T, p);
  if constexpr (PACKED) {
    auto put2 = [&](auto I, float2 v) {
      constexpr int i = decltype(I)::value;
      store(ic<i>{}, v.x);
      store(ic<i + 1>{}, v.y);
    };
    collide_f2<L, DEV>(lw, T, inv_tau, get2, put2, (float)c_dev);
  } else {
    collide<L, A, DEV>(lw, T, inv_tau, get, store, c_dev);
  }
}

// Step-kernel variants for float arithmetic.  Every population is pulled once and all populations
// of a cell stay in registers.
//   bit 0: scalar arithmetic (0) or mirror pairs in float2 with paired FMA (1);
//   bit 1: registers as needed, 2 resident blocks of 128 threads per SM (0), or at most 168
//          registers for 3 resident blocks (1; the compiler spills a little).
// (Also measured slower and not built: keeping half-deviation populations as packed half2 pairs
// at 4 resident blocks (128 registers still spill); staging part of the populations in shared
// memory; a persistent interior kernel that prefetches each thread's next cell into shared memory
// with cp.async while it computes the current one; and two passes over the populations, moments
// then collision, at 64-80 registers and 6-8 resident blocks with L2 evict-last / evict-first
// hints, whose second pass executed about 50% more instructions and still missed L2 on a third
// of its reads.)
// Double arithmetic pulls each population twice (moments, then collision) and has one variant.
enum StepVariant : int { kRegScalar = 0, kRegPacked = 1, kReg3Scalar = 2, kReg3Packed = 3, kNumVariants = 4 };

template <class S, int VARIANT>
struct StepShape {
  static constexpr bool kKeep = std::is_same<typename S::A, float>::value;  // populations in registers
  static constexpr int kMinBlocks = (VARIANT & 2) ? 3 : 1;
};

// How a step kernel pulls: the row kernel's warps lie in rows with interior y and z and are told
// whether their x segment is interior too (constant offsets) or not (only x wraps); the shell row
// kernel's warps lie in boundary rows, whose y and z shifts are the same for the whole warp; the
// per-cell shell kernel (lattices shorter than the stencil reach) wraps every coordinate of every
// cell.
enum PullPath : int { kPathRow = 1, kPathEdge = 2, kPathShellRow = 3, kPathShellTab = 4 };

// One cell's time step (pull, moments, Landau matching, equilibrium, collision, store).  Invalid
// lanes (valid = false) carry a clamped in-range cell, compute and store nothing.
template <class L, class S, bool GENERAL, int VARIANT, int PATH, bool WALLS>
__device__ __forceinline__ void step_cell(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
                                          const StepParams& p, int* __restrict__ status, const Cell cl,
                                          const bool valid, const bool row_fast = false,
                                          const long long* __restrict__ roff = nullptr) {
  using A = typename S::A;
  using ST = typename S::T;
  constexpr bool PACKED = (VARIANT & 1) && std::is_same<A, float>::value;
  constexpr bool KEEP = StepShape<S, VARIANT>::kKeep;
  // Warp-uniform choice: a row warp whose segment is interior pulls with constant offsets; other
  // row warps wrap x only; shell cells resolve wrap / copy-out / bounce-back per population.
  static_assert(PATH == kPathRow || PATH == kPathEdge || PATH == kPathShellRow || PATH == kPathShellTab,
                "pull path");
  static_assert(PATH != kPathShellTab || !WALLS, "the shell-row table has no bounce-back walls");
  const bool fast = PATH == kPathRow && row_fast;
  const ST* __restrict__ base = src + cl.c;
  ST* __restrict__ out = dst + cl.c;
  // Half-deviation storage works in deviation space: the values in flight are d_i = f_i / w_i - c
  // as stored, and the moments and collision take the weights and c into their constants.
  constexpr bool DEV = std::is_same<S, StoreF16Dev>::value;
  auto ld = [&](auto I, const ST* ptr) -> A {
    constexpr int i = decltype(I)::value;
    if constexpr (DEV) return S::template load_dev<L, i>(ptr, p);
    else return S::template load<L, i>(ptr, p);
  };

  auto load = [&](auto I) -> A {
    constexpr int i = decltype(I)::value;
    if (fast) return ld(I, base + p.off[i]);
    if constexpr (PATH == kPathRow) return ld(I, base + x_row_offset<L, i, WALLS>(cl, p));
    else if constexpr (PATH == kPathShellRow) return ld(I, base + shell_row_offset<L, i, WALLS>(cl, p, row_fast));
    else if constexpr (PATH == kPathShellTab) {
      constexpr int vx = L::VX[i];
      long long o = roff[i];
      if constexpr (vx != 0) {
        if (!row_fast) o += src_coord<vx, false>(cl.x, p.nx, p.bc[0]) - (cl.x - vx);
      }
      return ld(I, base + o);
    }
    else return ld(I, src + pull_index<L, i, GENERAL, WALLS>(cl, p));
  };
  auto store = [&](auto I, A v) {
    constexpr int i = decltype(I)::value;
    if (valid) {
      if constexpr (DEV) S::template store_dev<L, i>(out + (long long)i * p.cells, v, p);
      else S::template store<L, i>(out + (long long)i * p.cells, v, p);
    }
  };

  A fk[KEEP ? L::Q : 1];
  if constexpr (KEEP) {
    // one warp-uniform branch around the whole pull, so the fast path is plain constant offsets
    if (fast) static_for<L::Q>([&](auto I) { fk[decltype(I)::value] = ld(I, base + p.off[decltype(I)::value]); });
    else static_for<L::Q>([&](auto I) { fk[decltype(I)::value] = load(I); });
  }
  auto get = [&](auto I) -> A {
    if constexpr (KEEP) return fk[decltype(I)::value];
    else return load(I);
  };
  relax_cell<L, S, PACKED>(get, store, p, status, valid);
}

// Cell of lane `lane` in row-kernel warp w (see k_step_interior).
__device__ __forceinline__ void row_cell(int w, int lane, const StepParams& p, Cell& cl, bool& valid, bool& fast) {
  const int seg = w % p.int_segs, row = w / p.int_segs;
  cl.y = p.iy0 + row % p.iyn;
  cl.z = p.iz0 + row / p.iyn;
  const int x0 = seg * 32, x = x0 + lane;
  valid = x < p.nx;
  cl.x = valid ? x : p.nx - 1;
  cl.c = (cl.z * p.ny + cl.y) * p.nx + cl.x;
  fast = x0 >= p.ix0 && min(x0 + 31, p.nx - 1) < p.ix0 + p.ixn;
}

// Interior rows (y and z inside the interior box, every x): warp w covers the 32-aligned x segment
// w % int_segs of row w / int_segs (the last segment may be partial).  A segment inside the
// interior x range pulls with constant offsets; the others wrap only x.  Whole rows in one kernel
// keep every sector of a row written by neighbouring warps.
template <class L, class S, int VARIANT, bool WALLS>
__global__ void __launch_bounds__(kStepThreads, StepShape<S, VARIANT>::kMinBlocks)
    k_step_interior(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
                    const __grid_constant__ StepParams p, int* __restrict__ status) {
  const int w = blockIdx.x * (kStepThreads / 32) + (threadIdx.x >> 5);
  if (w >= p.int_warps) return;  // whole warps only
  Cell cl;
  bool valid, fast;
  row_cell(w, threadIdx.x & 31, p, cl, valid, fast);
  step_cell<L, S, false, VARIANT, kPathRow, WALLS>(src, dst, p, status, cl, valid, fast);
}

// Row r of the shell: the rows of the z-boundary planes, then the y-boundary rows of the interior
// planes.
__device__ __forceinline__ void shell_row(int r, const StepParams& p, int& y, int& z) {
  const int A = (p.nz - p.izn) * p.ny;
  if (r < A) {
    const int zz = r / p.ny;
    y = r - zz * p.ny;
    z = zz < p.iz0 ? zz : zz + p.izn;
  } else {
    r -= A;
    const int wy = p.ny - p.iyn;
    const int zz = r / wy, yy = r - zz * wy;
    z = p.iz0 + zz;
    y = yy < p.iy0 ? yy : yy + p.iyn;
  }
}

// Shell rows for lattices whose periodic axes are all at least the stencil reach: warp w covers
// the 32-aligned x segment w % row_segs of shell row w / row_segs, so the y and z shifts of each
// population are the same for the whole warp and x wraps only in segments outside the interior x
// range.
// One warp per block, so that the row (and with it every population's y and z shift) derives from
// blockIdx alone, a value the compiler knows to be the same for the whole warp; as many blocks
// per SM as the four-warp kernels have warps.
template <class L, class S, int VARIANT, bool WALLS>
__global__ void __launch_bounds__(32, 4 * StepShape<S, VARIANT>::kMinBlocks)
    k_step_shell_rows(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
                      const __grid_constant__ StepParams p, int* __restrict__ status) {
  const int w = blockIdx.x;
  const int seg = w % p.row_segs, r = w / p.row_segs;
  Cell cl;
  shell_row(r, p, cl.y, cl.z);
  const int x0 = seg * 32, x = x0 + (threadIdx.x & 31);
  const bool valid = x < p.nx;
  cl.x = valid ? x : p.nx - 1;
  cl.c = (cl.z * p.ny + cl.y) * p.nx + cl.x;
  const bool xfast = x0 >= p.ix0 && min(x0 + 31, p.nx - 1) < p.ix0 + p.ixn;
  if constexpr (WALLS) {
    step_cell<L, S, false, VARIANT, kPathShellRow, WALLS>(src, dst, p, status, cl, valid, xfast);
  } else {
    __shared__ long long roff[L::Q];
    shell_row_table<L>(roff, cl, p);
    step_cell<L, S, false, VARIANT, kPathShellTab, false>(src, dst, p, status, cl, valid, xfast, roff);
  }
}

// Shell cells (rows whose y or z lies outside the interior box): z-boundary planes, then the
// y-boundary rows of the interior planes; wrapped / clamped pulls.
__device__ __forceinline__ Cell shell_cell(int s, const StepParams& p) {
  Cell cl;
  const int A = (p.nz - p.izn) * p.nxy;
  if (s < A) {
    const int zz = s / p.nxy, r = s - zz * p.nxy;
    cl.z = zz < p.iz0 ? zz : zz + p.izn;
    cl.y = r / p.nx;
    cl.x = r - cl.y * p.nx;
  } else {
    s -= A;
    const int rowy = (p.ny - p.iyn) * p.nx;
    const int zz = s / rowy, r = s - zz * rowy;
    cl.z = p.iz0 + zz;
    const int yy = r / p.nx;
    cl.y = yy < p.iy0 ? yy : yy + p.iyn;
    cl.x = r - yy * p.nx;
  }
  cl.c = (cl.z * p.ny + cl.y) * p.nx + cl.x;
  return cl;
}

template <class L, class S, bool GENERAL, int VARIANT, bool WALLS>
__global__ void __launch_bounds__(kStepThreads, StepShape<S, VARIANT>::kMinBlocks)
    k_step_shell(const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
                 const __grid_constant__ StepParams p, int* __restrict__ status) {
  const int s = blockIdx.x * kStepThreads + threadIdx.x;
  const bool valid = s < p.shell_cells;
  const Cell cl = shell_cell(valid ? s : p.shell_cells - 1, p);
  step_cell<L, S, GENERAL, VARIANT, kPathEdge, WALLS>(src, dst, p, status, cl, valid);
}

// ---------------------------------------------------------------------------------------------
// Batched step: many independent lattices (members) advance together.  Each time step is two
// persistent launches, one over the members' row tiles (four row-kernel warps each: constant
// offsets, or x wrapped only) and one over their shell tiles (four shell-row warps each, or
// kStepThreads shell cells each for members that need the modulo wrap): the decomposition of a
// solo step, so a member's populations are bitwise those
// of the same steps taken alone with the same variant, and each kernel carries one pull path.
// Blocks take tiles from the launch's queue (an atomic counter); a tile's member comes from a
// tile -> member table (row tiles first, then shell tiles), and a block copies a member's
// parameters to shared memory only when its member changes.  Members whose step count is reached
// are skipped.
// ---------------------------------------------------------------------------------------------
template <class L, class S, int VARIANT, bool WALLS, bool ROWS>
__global__ void __launch_bounds__(kStepThreads, StepShape<S, VARIANT>::kMinBlocks)
    k_step_batch(const BatchMember* __restrict__ members, const int* __restrict__ tile_member, int tile_begin,
                 int tile_end, int launch_index, int* __restrict__ counter) {
  using ST = typename S::T;
  __shared__ StepParams sp;
  __shared__ int s_tile, s_member;
  __shared__ long long s_roff[kStepThreads / 32][L::Q];  // shell tiles: each warp's row offsets
  int held = -1;  // member whose parameters sp holds (block-uniform)
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = tile_begin + atomicAdd(counter, 1);
      s_tile = t;
      s_member = t < tile_end ? __ldg(&tile_member[t]) : 0;
    }
    __syncthreads();
    const int tile = s_tile;
    const int mi = s_member;
    if (tile >= tile_end) return;
    const BatchMember& m = members[mi];
    const bool active = launch_index < m.steps_left;
    if (active && mi != held) {
      const int* srcw = reinterpret_cast<const int*>(&m.p);
      int* dstw = reinterpret_cast<int*>(&sp);
      for (int k = threadIdx.x; k < (int)(sizeof(StepParams) / sizeof(int)); k += kStepThreads) dstw[k] = srcw[k];
      held = mi;
    }
    __syncthreads();
    if (active) {
      const int par = (m.parity0 + launch_index) & 1;
      const ST* sb = static_cast<const ST*>(m.buf[par]);
      ST* db = static_cast<ST*>(m.buf[par ^ 1]);
      if constexpr (ROWS) {
        const int w = (tile - m.row_tile_begin) * (kStepThreads / 32) + (threadIdx.x >> 5);
        if (w < sp.int_warps) {  // whole warps only
          Cell cl;
          bool valid, fast;
          row_cell(w, threadIdx.x & 31, sp, cl, valid, fast);
          step_cell<L, S, false, VARIANT, kPathRow, WALLS>(sb, db, sp, m.status, cl, valid, fast);
        }
      } else if (sp.general) {
        // per cell, modulo wrap (a periodic axis shorter than the stencil reach)
        const int s = (tile - m.shell_tile_begin) * kStepThreads + threadIdx.x;
        const bool valid = s < sp.shell_cells;
        const Cell cl = shell_cell(valid ? s : sp.shell_cells - 1, sp);
        step_cell<L, S, true, VARIANT, kPathEdge, WALLS>(sb, db, sp, m.status, cl, valid);
      } else {
        // four shell-row warps, as in k_step_shell_rows
        const int w = (tile - m.shell_tile_begin) * (kStepThreads / 32) + (threadIdx.x >> 5);
        if (w < sp.shell_warps) {  // whole warps only
          const int seg = w % sp.row_segs, r = w / sp.row_segs;
          Cell cl;
          shell_row(r, sp, cl.y, cl.z);
          const int x0 = seg * 32, x = x0 + (threadIdx.x & 31);
          const bool valid = x < sp.nx;
          cl.x = valid ? x : sp.nx - 1;
          cl.c = (cl.z * sp.ny + cl.y) * sp.nx + cl.x;
          const bool xfast = x0 >= sp.ix0 && min(x0 + 31, sp.nx - 1) < sp.ix0 + sp.ixn;
          if (WALLS && sp.has_wall) {
            step_cell<L, S, false, VARIANT, kPathShellRow, WALLS>(sb, db, sp, m.status, cl, valid, xfast);
          } else {
            long long* roff = s_roff[threadIdx.x >> 5];
            shell_row_table<L>(roff, cl, sp);
            step_cell<L, S, false, VARIANT, kPathShellTab, false>(sb, db, sp, m.status, cl, valid, xfast, roff);
          }
        }
      }
    }
    __syncthreads();  // sp and s_tile are reused by the next tile
  }
}

// ---------------------------------------------------------------------------------------------
// float-float arithmetic: a value as the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2),
// built from the error-free transformations of Dekker and Knuth (two-sum; two-product by FMA).
// About 44 bits of significand, at float-pipe speed.
// ---------------------------------------------------------------------------------------------
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_from(double x) {
  const float hi = (float)x;
  return FF{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

// hi + lo of a + b exactly (Knuth's two-sum)
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return FF{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return FF{s, b - (s - a)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);  // exact error of the product
  return fast_two_sum(p, e + fmaf(a.hi, b.lo, a.lo * b.hi));
}

// a times a small integer k (|k| <= 6): exact in float-float
__device__ __forceinline__ FF ff_scale(FF a, float k) {
  const float p = a.hi * k;
  return fast_two_sum(p, fmaf(a.hi, k, -p) + a.lo * k);
}

// a + t (b + t (c + t d)) in float-float, rounded to float
__device__ __forceinline__ float ff_horner3(FF t, FF a, FF b, FF c, FF d) {
  FF r = ff_add(ff_mul(d, t), c);
  r = ff_add(ff_mul(r, t), b);
  r = ff_add(ff_mul(r, t), a);
  return r.hi + r.lo;
}

// The moments of float populations (deviations d_i for half storage, with the weights' own moments
// times c added) for the fields readout: per direction pair, the sums over energies for +v and -v
// are first combined into their sum P and difference D, and the moments accumulate c P (even
// moments) and c D (odd moments) in float.  The odd moments (the velocity) then cancel within each
// direction pair before they are summed over directions, which keeps T^{0a} near float rounding of
// the populations (about 1e-8 of T^00; summing +v and -v over all directions first and subtracting
// at the end loses an order of magnitude more).  Returned in double, with the weights' own moments
// and T^zz (trace identity) added in double.
template <class L, bool DEV, class GetF>
__device__ __forceinline__ Mom<double> moments_pd(GetF&& getf, double c) {
  float N0 = 0.f, Nx = 0.f, Ny = 0.f, Nz = 0.f, T00 = 0.f, T0x = 0.f, T0y = 0.f, T0z = 0.f, Txx = 0.f, Tyy = 0.f,
        Txy = 0.f, Txz = 0.f, Tyz = 0.f;
  static_for<L::NDP>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int first = L::DP_FIRST[k];
    constexpr int np = L::DP_NPAIR[k];
    float S1p = 0.f, S1m = 0.f, S2p = 0.f, S2m = 0.f;
    static_for<np>([&](auto J) {
      constexpr int ip = first + 2 * decltype(J)::value;
      constexpr double wk = DEV ? L::W[ip] : 1.0;  // mirror partners share the weight
      constexpr float p0 = (float)(wk * L::P0[L::LEV[ip]]);
      constexpr float p02 = (float)(wk * L::P0[L::LEV[ip]] * L::P0[L::LEV[ip]]);
      const float fa = getf(ic<ip>{}), fb = getf(ic<ip + 1>{});
      S1p = fmaf(p0, fa, S1p);
      S1m = fmaf(p0, fb, S1m);
      S2p = fmaf(p02, fa, S2p);
      S2m = fmaf(p02, fb, S2m);
    });
    constexpr int vx = L::VX[first], vy = L::VY[first], vz = L::VZ[first];
    constexpr double ir = L::INV_R, ir2 = L::INV_R2;
    const float P1 = S1p + S1m, D1 = S1p - S1m, P2 = S2p + S2m, D2 = S2p - S2m;
    N0 += P1;
    T00 += P2;
    if constexpr (vx != 0) {
      Nx = fmaf((float)(vx * ir), D1, Nx);
      T0x = fmaf((float)(vx * ir), D2, T0x);
      Txx = fmaf((float)(vx * vx * ir2), P2, Txx);
    }
    if constexpr (vy != 0) {
      Ny = fmaf((float)(vy * ir), D1, Ny);
      T0y = fmaf((float)(vy * ir), D2, T0y);
      Tyy = fmaf((float)(vy * vy * ir2), P2, Tyy);
    }
    if constexpr (vz != 0) {
      Nz = fmaf((float)(vz * ir), D1, Nz);
      T0z = fmaf((float)(vz * ir), D2, T0z);
    }
    if constexpr (vx != 0 && vy != 0) Txy = fmaf((float)(vx * vy * ir2), P2, Txy);
    if constexpr (vx != 0 && vz != 0) Txz = fmaf((float)(vx * vz * ir2), P2, Txz);
    if constexpr (vy != 0 && vz != 0) Tyz = fmaf((float)(vy * vz * ir2), P2, Tyz);
  });
  Mom<double> m{N0, Nx, Ny, Nz, T00, T0x, T0y, T0z, Txx, Tyy, 0.0, Txy, Txz, Tyz};
  if constexpr (DEV) add_rest_sums<L, double>(m, c);
  m.Tzz = m.T00 - m.Txx - m.Tyy;
  return m;
}

// ---------------------------------------------------------------------------------------------
// fields and conserved densities of one time level (double arithmetic; for float storages the
// Landau solve starts from the float solution and stops at 1e-12 U0)
//   PULL = true : the pre-collision populations pulled from the previous state (GENERAL: modulo
//                 wrap, for periodic axes shorter than the stencil reach)
//   PULL = false: the stored populations of each cell
// out.f[k][cell], k = n, eps, U0, U1, U2, U3; partial[block][5] = block sums of
// N^0, T^00, T^0x, T^0y, T^0z, reduced by warp shuffles in a fixed order.
// ---------------------------------------------------------------------------------------------
template <class L, class S, bool PULL, bool GENERAL>
__global__ void __launch_bounds__(kMomThreads) k_fields(const typename S::T* __restrict__ src,
                                                        const __grid_constant__ StepParams p,
                                                        const FieldOut out,
                                                        double* __restrict__ partial,
                                                        int* __restrict__ status, int block0) {
  // blocks [block0, block0 + gridDim.x) of the lattice's kMomThreads-cell blocks (a launch may cover
  // a chunk of the lattice; the partial sums land in the same slots either way)
  const int blk = block0 + blockIdx.x;
  const int gid = blk * kMomThreads + threadIdx.x;
  const bool valid = gid < p.cells;
  const Cell cl = make_cell(valid ? gid : p.cells - 1, p);
  auto index = [&](auto I) -> long long {
    constexpr int i = decltype(I)::value;
    return PULL ? pull_index<L, i, GENERAL, true>(cl, p) : (long long)i * p.cells + cl.c;
  };
  Mom<double> m;
  Landau<double> lw;
  if constexpr (std::is_same<typename S::A, double>::value) {
    m = moments<L, double>([&](auto I) -> double { return src[index(I)]; });
    lw = landau<double, 200>(m);
  } else {
    // float populations: the per-cell moments in float with each direction pair's difference taken
    // first (moments_pd; deviations for half storage); the cross-cell sums below in double
    constexpr bool DEV = std::is_same<S, StoreF16Dev>::value;
    auto getf = [&](auto I) -> float {
      constexpr int i = decltype(I)::value;
      if constexpr (DEV) return S::template load_dev<L, i>(src + index(I), p);
      else return (float)src[index(I)];
    };
    m = moments_pd<L, DEV>(getf, (double)p.half_nref);
    // the step's policy: float solve, double for cells above gamma_thr, for unconverged float
    // solves, or everywhere with landau_fp64; the result of a float solve is refined by one
    // double update (n and eps are the double Rayleigh quotients of the float U)
    const Mom<float> mf = convert<double, float>(m);
    const float NN = mf.N0 * mf.N0 - mf.Nx * mf.Nx - mf.Ny * mf.Ny - mf.Nz * mf.Nz;
    bool dbl = p.landau_fp64 || mf.N0 * mf.N0 > p.gamma_thr2 * NN;
    if (!dbl) {
      const Landau<float> lf = landau<float, 8>(mf);
      if (lf.ok && lf.conv)
        lw = landau_from<double, 1>(m, (double)lf.U0, (double)lf.Ux, (double)lf.Uy, (double)lf.Uz, 1e-10);
      dbl = !(lf.ok && lf.conv);
    }
    if (dbl) lw = landau<double, 200>(m);
  }
  if (valid) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    out.f[0][cl.c] = lw.ok ? lw.n : nan;
    out.f[1][cl.c] = lw.ok ? lw.eps : nan;
    out.f[2][cl.c] = lw.ok ? lw.U0 : nan;
    out.f[3][cl.c] = lw.ok ? lw.Ux : nan;
    out.f[4][cl.c] = lw.ok ? lw.Uy : nan;
    out.f[5][cl.c] = lw.ok ? lw.Uz : nan;
    // non-finite populations show as non-finite moments; any other cell without a frame is a
    // Landau failure
    const bool finite = isfinite(m.N0) && isfinite(m.Nx) && isfinite(m.Ny) && isfinite(m.Nz) && isfinite(m.T00) &&
                        isfinite(m.T0x) && isfinite(m.T0y) && isfinite(m.T0z) && isfinite(m.Txx) &&
                        isfinite(m.Tyy) && isfinite(m.Tzz) && isfinite(m.Txy) && isfinite(m.Txz) && isfinite(m.Tyz);
    if (!finite) atomicAdd(&status[kStatusNan], 1);
    else if (!lw.ok) atomicAdd(&status[kStatusNonconv], 1);
  }
  double d[5] = {valid ? m.N0 : 0.0, valid ? m.T00 : 0.0, valid ? m.T0x : 0.0, valid ? m.T0y : 0.0,
                 valid ? m.T0z : 0.0};
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d[k] += __shfl_down_sync(0xffffffffu, d[k], o);
  __shared__ double ws[kMomThreads / 32][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 5; ++k) ws[warp][k] = d[k];
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kMomThreads / 32; ++w) s += ws[w][threadIdx.x];
    partial[(long long)blk * 5 + threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------------------------
// initial state f_i = f_i^eq(n, T, u) (per-level form: coefficients in double, Horner steps in the
// storage's arithmetic), and population format conversion
// ---------------------------------------------------------------------------------------------
template <class L, class S>
__global__ void __launch_bounds__(128) k_init(const double* __restrict__ n, const double* __restrict__ Tf,
                                              const double* __restrict__ u, typename S::T* __restrict__ dst,
                                              const __grid_constant__ StepParams p, int* __restrict__ status,
                                              int c0, int c1) {
  // cells [c0, c1) (a launch may cover a chunk of the lattice)
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  const long long cells = p.cells;
  const double ux = u[c], uy = u[cells + c], uz = u[2 * cells + c];
  const double u2 = ux * ux + uy * uy + uz * uz;
  const double nn = n[c], T = Tf[c];
  if (!(u2 < 1.0) || !(T > 0.0) || !(nn > 0.0)) {
    atomicAdd(&status[kStatusBadInit], 1);
    return;
  }
  const double g = rsqrt(1.0 - u2);
  const double Ux = g * ux, Uy = g * uy, Uz = g * uz;
  // the equilibrium per energy level (see level_coef), coefficients in double
  const LevCoef<L, double> ed = level_coef<L, double>(eq_coef<L::ORDER, double>(nn, T, g));
  if constexpr (std::is_same<typename S::A, double>::value) {
    static_for<L::NDP>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr int first = L::DP_FIRST[k];
      constexpr int np = L::DP_NPAIR[k];
      constexpr int vx = L::VX[first], vy = L::VY[first], vz = L::VZ[first];
      const double t = (vx * Ux + vy * Uy + vz * Uz) * L::INV_R;
      static_for<np>([&](auto J) {
        constexpr int ip = first + 2 * decltype(J)::value;
        constexpr int l = L::LEV[ip];
        constexpr double w = L::W[ip];
        const double Ep = fma(t, fma(t, fma(t, ed.d[l], ed.c[l]), ed.b[l]), ed.a[l]);
        const double Em = fma(-t, fma(-t, fma(-t, ed.d[l], ed.c[l]), ed.b[l]), ed.a[l]);
        S::template store<L, ip>(dst + (long long)ip * cells + c, w * Ep, p);
        S::template store<L, ip + 1>(dst + (long long)(ip + 1) * cells + c, w * Em, p);
      });
    });
  } else {
    // Float storage rounds every population to float.  The cubic in t cancels strongly at the high
    // energy levels (terms up to ~200 times the value at p0 = 10.95, |u| = 0.6), so those levels
    // (p0 > 4) are evaluated in float-float arithmetic (a value as an unevaluated sum hi + lo of
    // two floats; error-free sums and products by FMA), the others in float: every population ends
    // within float rounding of the double evaluation, with no double arithmetic per population.
    LevCoef<L, FF> e;
    static_for<L::NLEV>([&](auto K) {
      constexpr int l = decltype(K)::value;
      e.a[l] = ff_from(ed.a[l]);
      e.b[l] = ff_from(ed.b[l]);
      e.c[l] = ff_from(ed.c[l]);
      e.d[l] = ff_from(ed.d[l]);
    });
    const FF Uxf = ff_from(Ux), Uyf = ff_from(Uy), Uzf = ff_from(Uz);
    static_for<L::NDP>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr int first = L::DP_FIRST[k];
      constexpr int np = L::DP_NPAIR[k];
      constexpr int vx = L::VX[first], vy = L::VY[first], vz = L::VZ[first];
      // t = v.U / R: exact small-integer multiples, float-float sum and scaling
      const FF t = ff_mul(ff_add(ff_add(ff_scale(Uxf, (float)vx), ff_scale(Uyf, (float)vy)), ff_scale(Uzf, (float)vz)),
                          ff_from(L::INV_R));
      static_for<np>([&](auto J) {
        constexpr int ip = first + 2 * decltype(J)::value;
        constexpr int l = L::LEV[ip];
        constexpr float w = (float)L::W[ip];
        float Ep, Em;
        if constexpr (L::P0[l] > 4.0) {
          const FF tm = ff_neg(t);
          Ep = ff_horner3(t, e.a[l], e.b[l], e.c[l], e.d[l]);
          Em = ff_horner3(tm, e.a[l], e.b[l], e.c[l], e.d[l]);
        } else {
          const float tf = t.hi + t.lo;
          Ep = fmaf(tf, fmaf(tf, fmaf(tf, e.d[l].hi, e.c[l].hi), e.b[l].hi), e.a[l].hi);
          Em = fmaf(-tf, fmaf(-tf, fmaf(-tf, e.d[l].hi, e.c[l].hi), e.b[l].hi), e.a[l].hi);
        }
        S::template store<L, ip>(dst + (long long)ip * cells + c, w * Ep, p);
        S::template store<L, ip + 1>(dst + (long long)(ip + 1) * cells + c, w * Em, p);
      });
    });
  }
}

// double[q][cells] <-> storage, for populations [i0, i1) (in-range cells only)
template <class L, class S, bool TO_F64>
__global__ void __launch_bounds__(128) k_convert(typename S::T* __restrict__ pop, double* __restrict__ dbl,
                                                 long long dbl_plane_offset, int i0, int i1,
                                                 const __grid_constant__ StepParams p) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.cells) return;
  const long long cells = p.cells;
  static_for<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (i < i0 || i >= i1) return;
    const long long di = (long long)(i - i0) * cells + c + dbl_plane_offset;
    if constexpr (TO_F64) dbl[di] = S::template to_f64<L, i>(pop[(long long)i * cells + c], p);
    else pop[(long long)i * cells + c] = S::template from_f64<L, i>(dbl[di], p);
  });
}

}  // namespace rlb
