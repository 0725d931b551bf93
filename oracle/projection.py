"""The discrete equilibrium as an explicit moment projection (Sec. II.B), independent of App. B.

Test infrastructure only.  The paper builds orthonormal polynomials J_k by Gram-Schmidt on the rest
weight w(p0) = exp(-p0)/(4 pi) with measure d^3p/p0 (Sec. II.B, Table I), projects the
Maxwell-Juttner distribution onto them, a_k = int f^eq J_k d^3p/p0 (Eq. (coeff)), and evaluates
f_i^eq = w_i sum_k a_k J_k(p_i) (Eq. (eq:disc1)).  This module does exactly that:

  * the space is spanned by the spatial monomials of degree <= order and p0 times the spatial
    monomials of degree <= order - 1 (on the light cone p0^2 = |p|^2 these span every polynomial
    of degree <= order);
  * the inner product of two monomials is a rest-frame moment of the weight,
    int w p0^k n_x^a n_y^b n_z^c d^3p/p0 = (k+1)! <n_x^a n_y^b n_z^c>_sphere, an exact rational,
    so Gram-Schmidt runs in exact rational arithmetic (orthogonal, not normalised, basis P_k);
  * the projections <f^eq, m> of f^eq on each monomial are Maxwell-Juttner moments in closed form:
    n/(2T) for degree 0 (the rest value of int f^eq d^3p/p0, a Lorentz scalar), N^mu = n U^mu,
    T^{mu nu} = -n T eta^{mu nu} + 4 n T U^mu U^nu and
    P^{mu nu l} = -4 n T^2 (eta^{mu nu} U^l + eta^{mu l} U^nu + eta^{nu l} U^mu) + 24 n T^2 U^mu U^nu U^l
    (Sec. II.C, after Eq. (moments:dis3)).
"""
import itertools
from fractions import Fraction
from functools import lru_cache
from math import factorial

import numpy as np

ETA = np.diag([1.0, -1.0, -1.0, -1.0])


def _dfact(n):
    return 1 if n <= 0 else n * _dfact(n - 2)


def sphere_mean(a, b, c):
    """<n_x^a n_y^b n_z^c> over the unit sphere, exact."""
    if a % 2 or b % 2 or c % 2:
        return Fraction(0)
    return Fraction(_dfact(a - 1) * _dfact(b - 1) * _dfact(c - 1), _dfact(a + b + c + 1))


def rest_moment(e, a, b, c):
    """int w(p0) p0^e px^a py^b pz^c d^3p/p0 with w = exp(-p0)/(4 pi), exact rational."""
    k = e + a + b + c
    return factorial(k + 1) * sphere_mean(a, b, c)


def monomials(order):
    """(p0 power, (a, b, c)) spanning polynomials of degree <= order on the light cone."""
    out = []
    for d in range(order + 1):
        out += [(0, e) for e in itertools.product(range(d + 1), repeat=3) if sum(e) == d]
    for d in range(order):
        out += [(1, e) for e in itertools.product(range(d + 1), repeat=3) if sum(e) == d]
    return out


@lru_cache(maxsize=None)
def orthogonal_basis(order):
    """Exact Gram-Schmidt: rows of the returned list are coefficient vectors (over ``monomials``) of
    mutually orthogonal polynomials P_k, together with <P_k, P_k>."""
    M = monomials(order)
    G = [[rest_moment(a0 + b0, *(x + y for x, y in zip(a, b))) for (b0, b) in M] for (a0, a) in M]
    basis, norms = [], []
    for j in range(len(M)):
        v = [Fraction(0)] * len(M)
        v[j] = Fraction(1)
        for P, nn in zip(basis, norms):
            proj = sum(P[r] * G[r][j] for r in range(len(M)) if P[r]) / nn  # <P, m_j> / <P, P>
            v = [vi - proj * pi for vi, pi in zip(v, P)]
        nn = sum(v[r] * v[s] * G[r][s] for r in range(len(M)) if v[r] for s in range(len(M)) if v[s])
        if nn == 0:
            raise ValueError("monomials are dependent on the light cone")
        basis.append(v)
        norms.append(nn)
    return M, basis, norms


def mj_moments(n, T, U):
    """Closed-form Maxwell-Juttner moments: scalar, N^mu, T^{mu nu}, P^{mu nu l}."""
    U = np.asarray(U, dtype=np.float64)
    N = n * U
    Tm = -n * T * ETA + 4 * n * T * np.outer(U, U)
    P = 24 * n * T ** 2 * np.einsum("a,b,c->abc", U, U, U) - 4 * n * T ** 2 * (
        np.einsum("ab,c->abc", ETA, U) + np.einsum("ac,b->abc", ETA, U) + np.einsum("bc,a->abc", ETA, U))
    return n / (2 * T), N, Tm, P


def _monomial_moment(mono, scalar, N, Tm, P):
    e0, (a, b, c) = mono
    idx = [0] * e0 + [1] * a + [2] * b + [3] * c
    if not idx:
        return scalar
    if len(idx) == 1:
        return N[idx[0]]
    if len(idx) == 2:
        return Tm[idx[0], idx[1]]
    return P[tuple(idx)]


def feq_over_w(order, n, T, U, p):
    """sum_k a_k J_k(p) for 4-momenta p (shape (m, 4)): the projection of f^eq / w."""
    M, basis, norms = orthogonal_basis(order)
    mom = mj_moments(n, T, U)
    b = np.array([_monomial_moment(m, *mom) for m in M])
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    vals = np.stack([p[:, 0] ** e0 * p[:, 1] ** a * p[:, 2] ** bb * p[:, 3] ** c for e0, (a, bb, c) in M], axis=1)
    out = np.zeros(len(p))
    for P, nn in zip(basis, norms):
        Pf = np.array([float(x) for x in P])
        a_k = float(Pf @ b) / float(nn)  # <f^eq, P_k> / <P_k, P_k>
        out += a_k * (vals @ Pf)
    return out


def equilibrium(lat, n, T, U):
    """f_i^eq = w_i sum_k a_k J_k(p_i) on the lattice ``lat`` (Eq. (eq:disc1))."""
    return lat.w * feq_over_w(lat.order, n, T, U, lat.momenta())
