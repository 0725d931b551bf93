"""Pins of the committed quadratures against the paper (Sec. II.C, Eqs. (eq:dio), (eqs:eqs); App. A)."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import roots_genlaguerre

import oracle
from oracle.projection import rest_moment

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLDEN, "paper_values.json")))


def all_directions(R2):
    r = int(math.isqrt(R2)) + 1
    return {v for v in itertools.product(range(-r, r + 1), repeat=3) if sum(x * x for x in v) == R2}


def family_members(fams):
    out = set()
    for f in fams:
        for perm in itertools.permutations(f):
            for s in itertools.product((1, -1), repeat=3):
                out.add(tuple(a * b for a, b in zip(perm, s)))
    return out


@pytest.mark.parametrize("order,key", [(3, "third_order"), (2, "second_order")])
def test_counts_and_directions(order, key):
    lat = oracle.read_lattice(order)
    fam = PAPER["direction_families_" + key]
    dirs = {tuple(v) for v in lat.v}
    # Eq. (eq:dio): the printed families are exactly the integer solutions of |n|^2 = R^2.
    assert family_members(fam["families"]) == all_directions(fam["R2"])
    assert len(all_directions(fam["R2"])) == fam["count"]
    # Every direction is used (Sec. II.C: all velocity vectors are needed; App. A).
    assert dirs == all_directions(fam["R2"])
    assert lat.R2 == fam["R2"]
    counts = PAPER["population_counts"][key]
    assert lat.q == counts["kept"]
    assert len(set(lat.level)) * fam["count"] == counts["candidates"]
    # No population appears twice.
    assert len({(tuple(v), l) for v, l in zip(lat.v, lat.level)}) == lat.q


@pytest.mark.parametrize("order,key,deg", [(3, "third_order", 4), (2, "second_order", 3)])
def test_radial_nodes(order, key, deg):
    lat = oracle.read_lattice(order)
    nodes = np.array(sorted({float(p) for p in lat.p0}))
    printed = PAPER["radial_nodes_" + key]
    assert len(nodes) == deg
    assert np.all(np.abs(nodes - printed["values"]) <= printed["abs_tol"])
    # Zeros of the printed radial polynomial ...
    coeffs = PAPER["radial_polynomial_" + key]["coefficients_high_to_low"]
    scale = np.polyval(np.abs(coeffs), nodes)
    assert np.all(np.abs(np.polyval(coeffs, nodes)) <= 1e-13 * scale)
    # ... which are the Gauss nodes of the weight p e^{-p} (generalised Laguerre, alpha = 1),
    # the measure d^3p/p0 = p dp dOmega of Sec. II.A.
    x, _ = roots_genlaguerre(deg, 1.0)
    assert np.allclose(np.sort(x), nodes, rtol=1e-13, atol=0)


@pytest.mark.parametrize("order", [3, 2])
def test_weights_positive_mirror_symmetric(order):
    lat = oracle.read_lattice(order)
    assert np.all(lat.w > 0)
    idx = {(tuple(v), l): i for i, (v, l) in enumerate(zip(lat.v, lat.level))}
    for (v, l), i in idx.items():
        j = idx[(tuple(-x for x in v), l)]  # Eq. (eqs:eqs): w_i = w_j if p_i^k = -p_j^k
        assert lat.w[i] == lat.w[j]
        assert lat.p0[i] == lat.p0[j]
    assert math.fsum(lat.w) == pytest.approx(1.0, abs=1e-15)


def test_second_order_is_cubic_symmetric(lat2):
    idx = {(tuple(v), l): lat2.w[i] for i, (v, l) in enumerate(zip(lat2.v, lat2.level))}
    for (v, l), w in idx.items():
        for perm in itertools.permutations(v):
            for s in itertools.product((1, -1), repeat=3):
                assert idx[(tuple(a * b for a, b in zip(perm, s)), l)] == w


@pytest.mark.parametrize("order,kmax", [(3, 6), (2, 5)])
def test_rest_frame_moment_conditions(order, kmax):
    """Eq. (eqs:eqs): sum_i w_i p_i^mu ... p_i^lambda equals the rest-frame moment of
    w(p0) = exp(-p0)/(4 pi) over d^3p/p0 for every monomial up to degree kmax."""
    lat = oracle.read_lattice(order)
    p = lat.momenta()
    worst = 0.0
    for k in range(kmax + 1):
        for e in range(k + 1):
            for a, b, c in itertools.product(range(k - e + 1), repeat=3):
                if a + b + c != k - e:
                    continue
                terms = lat.w * p[:, 0] ** e * p[:, 1] ** a * p[:, 2] ** b * p[:, 3] ** c
                exact = float(rest_moment(e, a, b, c))
                scale = math.fsum(np.abs(terms)) + 1e-300
                worst = max(worst, abs(math.fsum(terms) - exact) / scale)
    assert worst < 1e-14


def test_third_order_conditions_fail_at_degree_7(lat3):
    """The quadrature is not exact beyond its design degree (so the previous test can fail)."""
    p = lat3.momenta()
    terms = lat3.w * p[:, 0] ** 1 * p[:, 3] ** 6
    assert abs(math.fsum(terms) - float(rest_moment(1, 0, 0, 6))) > 1e-6 * float(rest_moment(1, 0, 0, 6))


def _table1():
    out = {}
    for line in open(os.path.join(GOLDEN, "table1_polynomials.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, expr = line.rstrip("\n").split("\t")
        out[int(k)] = expr
    return out


def _eval_poly(expr, p):
    env = {"sqrt": np.sqrt, "p0": p[:, 0], "px": p[:, 1], "py": p[:, 2], "pz": p[:, 3]}
    return np.broadcast_to(eval(expr, env), (len(p),)).astype(float)


@pytest.mark.parametrize("order", [3, 2])
def test_table1_orthonormal_on_quadrature(order):
    """Eq. (ortho:qua): sum_i w_i J_l(p_i) J_k(p_i) = delta_lk for the printed J_k of Table I
    (orders 0-2 for the second-order lattice, 0-3 for the third-order one)."""
    lat = oracle.read_lattice(order)
    p = lat.momenta()
    J = {k: _eval_poly(e, p) for k, e in _table1().items() if k <= (29 if order == 3 else 13)}
    ks = sorted(J)
    G = np.array([[math.fsum(lat.w * J[a] * J[b]) for b in ks] for a in ks])
    assert np.abs(G - np.eye(len(ks))).max() < 1e-12
