"""Pins of the oracle's equilibrium and Landau matching (Sec. II.B-D, App. B)."""
import math

import numpy as np
import pytest

import oracle
from oracle import projection as pj


def random_state(rng, vmax=0.6):
    n = rng.uniform(0.1, 2.0)
    T = rng.uniform(0.5, 2.0)
    v = rng.normal(size=3)
    v *= rng.uniform(0, vmax) / np.linalg.norm(v)
    g = 1.0 / math.sqrt(1.0 - v @ v)
    return n, T, np.r_[g, g * v]


@pytest.mark.parametrize("order", [3, 2])
def test_rest_value(order):
    """At T = 1 and U = (1, 0, 0, 0) both appendix formulas reduce to f_i^eq = n w_i / 2, which is
    exp(-p0) n / (8 pi) divided by the weight exp(-p0) / (4 pi) (Sec. II.B with A = 1/(4 pi))."""
    lat = oracle.read_lattice(order)
    # projection route: round-off through basis values up to ~1e3 at p0 ~ 11
    assert np.allclose(oracle.equilibrium_cell(lat, 0.7, 1.0, [1.0, 0.0, 0.0, 0.0]), 0.35 * lat.w, rtol=1e-13, atol=0)
    assert np.allclose(oracle.equilibrium_appendix_cell(lat, 0.7, 1.0, [1.0, 0.0, 0.0, 0.0]), 0.35 * lat.w,
                       rtol=1e-14, atol=0)


@pytest.mark.parametrize("order", [3, 2])
def test_appendix_equals_gram_schmidt_projection(order):
    """The printed explicit equilibrium (Eq. (eq:equi3rd) / (eq:equi2nd)) equals the projection
    sum_k a_k J_k built independently by Gram-Schmidt (Eqs. (eq:expanded), (coeff)).  The explicit
    form, a polynomial in powers of p with terms up to ~1e4 times the result at T ~ 2, p0 ~ 11,
    carries rounding of order 1e-12 of the population scale."""
    lat = oracle.read_lattice(order)
    rng = np.random.default_rng(11 + order)
    for _ in range(20):
        n, T, U = random_state(rng, vmax=0.9)
        a = oracle.equilibrium_appendix_cell(lat, n, T, U)
        b = pj.equilibrium(lat, n, T, U)
        scale = np.maximum(np.abs(b), n * lat.w / 2)
        assert np.max(np.abs(a - b) / scale) < 1e-11


@pytest.mark.parametrize("order", [3, 2])
def test_oracle_projection_matches_exact_rational_route(order):
    """The C oracle's sum_k a_k J_k(p_i) (basis table from exact Gram-Schmidt, evaluated in long
    double) equals the numpy route over the same exact basis, and both sit within 1e-13 of the
    population scale of a 50-digit evaluation of the same projection."""
    import mpmath as mp
    lat = oracle.read_lattice(order)
    rng = np.random.default_rng(17 + order)
    M, basis, norms = pj.orthogonal_basis(order)
    mp.mp.dps = 50
    for _ in range(6):
        n, T, U = random_state(rng, vmax=0.8)
        a = oracle.equilibrium_cell(lat, n, T, U)
        b = pj.equilibrium(lat, n, T, U)
        scale = np.maximum(np.abs(b), n * lat.w / 2)
        assert np.max(np.abs(a - b) / scale) < 1e-13
        # 50-digit reference for a few populations
        s_, N_, T_, P_ = pj.mj_moments(n, T, U)
        bj = [mp.mpf(float(pj._monomial_moment(m, s_, N_, T_, P_))) for m in M]
        for i in (0, lat.q // 2, lat.q - 1, int(np.argmax(lat.p0))):
            p = [mp.mpf(float(lat.p0[i]))] + [mp.mpf(float(lat.p0[i])) * int(c) / mp.sqrt(lat.R2) for c in lat.v[i]]
            mv = [p[0] ** e0 * p[1] ** x * p[2] ** y * p[3] ** z for e0, (x, y, z) in M]
            val = 0
            for P, nn in zip(basis, norms):
                ak = sum(mp.mpf(c.numerator) / c.denominator * bj[j] for j, c in enumerate(P) if c) / (
                    mp.mpf(nn.numerator) / nn.denominator)
                val += ak * sum(mp.mpf(c.numerator) / c.denominator * mv[j] for j, c in enumerate(P) if c)
            exact = float(lat.w[i] * val)
            assert abs(a[i] - exact) < 1e-13 * scale[i]


def test_projection_off_lattice_momenta():
    """The two routes also agree away from the lattice momenta (any p on the light cone)."""
    rng = np.random.default_rng(5)
    lib = oracle.core._load()
    for order in (2, 3):
        for _ in range(10):
            n, T, U = random_state(rng)
            p0 = rng.uniform(0.2, 12.0, size=8)
            d = rng.normal(size=(8, 3))
            d /= np.linalg.norm(d, axis=1)[:, None]
            p = np.column_stack([p0, p0[:, None] * d])
            fn = lib.ora_feq3_over_w if order == 3 else lib.ora_feq2_over_w
            Uc = np.ascontiguousarray(U)
            a = np.array([fn(n, T, oracle.core._dp(Uc), *row) for row in p])
            b = pj.feq_over_w(order, n, T, U, p)
            assert np.max(np.abs(a - b) / np.maximum(np.abs(b), n / 2)) < 1e-10


@pytest.mark.parametrize("order", [3, 2])
def test_discrete_moments_match_maxwell_juttner(order):
    """Eqs. (moments:dis1)-(moments:dis3): the discrete f^eq reproduces N^mu = n U^mu and
    T^{mu nu} = -n T eta + 4 n T U U (both orders) and P^{mu nu l} (third order only)."""
    lat = oracle.read_lattice(order)
    p = lat.momenta()
    rng = np.random.default_rng(3)
    for _ in range(20):
        n, T, U = random_state(rng)
        f = oracle.equilibrium_cell(lat, n, T, U)
        _, N, Tm, P = pj.mj_moments(n, T, U)
        # Round-off of a 128-term sum: about 1e-13 of the largest component.
        assert np.allclose(f @ p, N, rtol=0, atol=1e-12 * np.abs(N).max())
        assert np.allclose(np.einsum("i,ia,ib->ab", f, p, p), Tm, rtol=0, atol=1e-12 * np.abs(Tm).max())
        Pd = np.einsum("i,ia,ib,ic->abc", f, p, p, p)
        if order == 3:
            assert np.allclose(Pd, P, rtol=0, atol=1e-12 * np.abs(P).max())
        elif np.linalg.norm(U[1:]) > 0.1:
            assert not np.allclose(Pd, P, rtol=1e-3, atol=1e-3 * n * T * T)


def test_mj_closed_forms_rest_frame():
    """The closed forms at rest equal direct radial integrals of n exp(-p/T)/(8 pi T^3):
    N^0 = n, T^00 = 3 n T (eps = 3 n T, Sec. II.B), T^xx = n T, P^000 = 12 n T^2, P^0xx = 4 n T^2."""
    n, T = 0.8, 1.3
    s, N, Tm, P = pj.mj_moments(n, T, [1, 0, 0, 0])
    c = n / (8 * math.pi * T ** 3)
    rad = lambda k: 4 * math.pi * c * math.factorial(k) * T ** (k + 1)  # int p^k e^{-p/T} dp * 4 pi
    assert s == pytest.approx(rad(1))
    assert N[0] == pytest.approx(rad(2))
    assert Tm[0, 0] == pytest.approx(rad(3))
    assert Tm[1, 1] == pytest.approx(rad(3) / 3)
    assert P[0, 0, 0] == pytest.approx(rad(4))
    assert P[0, 1, 1] == pytest.approx(rad(4) / 3)


def _eig_landau(N, Tm):
    """Timelike eigenvector of T^a_b from a dense eigen-solver, or None if there is none."""
    eta = np.diag([1.0, -1, -1, -1])
    vals, vecs = np.linalg.eig(Tm @ eta)
    for k in range(4):
        if abs(vals[k].imag) > 0:
            continue
        u = np.real(vecs[:, k])
        nrm = u @ eta @ u
        if nrm > 0:
            u = u / math.sqrt(nrm)
            u = u if u[0] > 0 else -u
            return u, float(np.real(vals[k])), float(u @ eta @ N)
    return None


@pytest.mark.parametrize("order", [3, 2])
def test_landau_recovers_equilibrium_fields(order):
    """From equilibrium populations Landau matching returns the input (n, eps = 3 n T, U)."""
    lat = oracle.read_lattice(order)
    rng = np.random.default_rng(7)
    for _ in range(20):
        n, T, U = random_state(rng, vmax=0.9)
        N, Tm = oracle.moments_cell(lat, oracle.equilibrium_cell(lat, n, T, U))
        st, U2, e, n2 = oracle.landau_cell(N, Tm)
        # The moments carry ~1e-13 relative round-off; the eigenproblem amplifies it by ~gamma^2.
        assert st == 0
        assert np.allclose(U2, U, rtol=0, atol=1e-11 * U[0])
        assert e == pytest.approx(3 * n * T, rel=1e-11)
        assert n2 == pytest.approx(n, rel=1e-11)


def test_landau_matches_eigendecomposition(lat3):
    """Off equilibrium the power iteration finds the timelike eigenvector that a dense eigen-solver
    of T^a_b finds (Eq. (eigenproblem))."""
    rng = np.random.default_rng(9)
    found = missing = 0
    for _ in range(100):
        n, T, U = random_state(rng, vmax=0.8)
        amp = rng.choice([0.02, 0.2, 1.0])
        f = oracle.equilibrium_cell(lat3, n, T, U) + amp * n * lat3.w * rng.normal(size=lat3.q)
        N, Tm = oracle.moments_cell(lat3, f)
        st, U2, e, n2 = oracle.landau_cell(N, Tm)
        ref = _eig_landau(N, Tm)
        if ref is None or ref[1] <= 0 or ref[2] <= 0:
            assert st == 4  # no Landau frame: reported as non-convergence
            missing += 1
            continue
        Ue, ee, ne = ref
        found += 1
        assert st == 0
        assert np.allclose(U2, Ue, rtol=0, atol=1e-11 * Ue[0])
        assert e == pytest.approx(ee, rel=1e-11)
        assert n2 == pytest.approx(ne, rel=1e-11)
    assert found >= 50


def test_landau_reports_nonconvergence():
    """A tensor with no timelike eigenvector of positive energy is rejected, not turned into NaN."""
    st, *_ = oracle.landau_cell(np.array([0.1, 1.0, 0.0, 0.0]), -np.eye(4))
    assert st == 4
