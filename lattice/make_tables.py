"""Generate the discrete-velocity quadratures of the relativistic lattice Boltzmann model.

The paper (Sec. II.C, Eqs. (eq:dio), (eqs:eqs), (eq:mrecon2)) fixes how a quadrature is found but
prints neither weight table (both sit in its Supplementary Material).  This script rebuilds them:

  * directions  : every integer vector with |n|^2 = R^2 (Eq. (eq:dio)); R^2 = 41 (third order, 96
                  directions) or R^2 = 9 (second order, App. A, 30 directions);
  * energies    : the zeros of the radial polynomial R^(4) (Sec. II.C) or R^(3) (App. A), i.e. the
                  generalised Laguerre polynomials L_4^(1), L_3^(1);
  * candidates  : p_i = p0_l (1, n_m / R)  (Eq. (eq:mrecon2));
  * weights     : w_i >= 0, w(n) = w(-n), and  sum_i w_i M(p_i) = int w(p0) M(p) d^3p/p0  for every
                  monomial M of degree <= 6 (third order) or <= 5 (second order), with
                  w(p0) = exp(-p0)/(4 pi) so that the rest moment of p0^k n_x^a n_y^b n_z^c is
                  (k+1)! <n_x^a n_y^b n_z^c>_sphere (Eq. (eqs:eqs)).

Among the solutions the paper keeps the one with the most zero weights.  The third-order conditions
have rank 64 on the 192 mirror pairs, so every vertex of the feasible polytope has at most 128
populations; a mixed-integer program picks a 128-population vertex that still uses all 96 directions
(Sec. II.C: all directions are needed).  The second-order table is the unique cubic-symmetric vertex
(66 populations), the symmetric choice the paper asks for.  The support is then re-solved in 50-digit
arithmetic and written with 25 significant digits, so that every reader parses the same doubles.

Run once:  python lattice/make_tables.py   (writes lattice/d3q128.txt and lattice/d3q66.txt)
"""
import itertools
import os
from math import factorial

import mpmath as mp
import numpy as np
from scipy.optimize import Bounds, LinearConstraint, milp

HERE = os.path.dirname(os.path.abspath(__file__))
mp.mp.dps = 50


def _dfact(n):
    return 1 if n <= 0 else n * _dfact(n - 2)


def sphere_mean(a, b, c):
    """Average of n_x^a n_y^b n_z^c over the unit sphere (exact rational, as mpf)."""
    if a % 2 or b % 2 or c % 2:
        return mp.mpf(0)
    return mp.mpf(_dfact(a - 1) * _dfact(b - 1) * _dfact(c - 1)) / _dfact(a + b + c + 1)


def condition_rows(kmax):
    """Independent monomials p0^e px^a py^b pz^c (c <= 1) of degree <= kmax on the light cone.

    On the cone px^2 + py^2 + pz^2 = p0^2, so degree-j spatial monomials with c in {0, 1} span the
    degree-j part without redundancy.  Only even j survive mirror symmetry."""
    rows = []
    for k in range(kmax + 1):
        for j in range(0, k + 1, 2):
            for c in (0, 1):
                for a in range(j - c + 1):
                    rows.append((k - j, a, j - c - a, c))
    return rows


def build(R2, poly, kmax, symmetry):
    r = int(np.ceil(np.sqrt(R2)))
    dirs = [v for v in itertools.product(range(-r, r + 1), repeat=3) if sum(x * x for x in v) == R2]
    nodes = sorted(mp.polyroots([mp.mpf(c) for c in poly], maxsteps=200, extraprec=200))
    nodes = [mp.re(x) for x in nodes]
    R = mp.sqrt(R2)

    if symmetry == "cubic":
        def orbit(v):
            out = set()
            for perm in itertools.permutations(range(3)):
                for s in itertools.product((1, -1), repeat=3):
                    out.add(tuple(s[k] * v[perm[k]] for k in range(3)))
            return frozenset(out)
    else:  # inversion only (w(n) = w(-n), Eq. (eqs:eqs))
        def orbit(v):
            return frozenset({tuple(v), tuple(-x for x in v)})
    orbits = sorted({orbit(v) for v in dirs}, key=lambda o: max(o), reverse=True)
    rows = condition_rows(kmax)
    rhs = [factorial(e + a + b + c + 1) * sphere_mean(a, b, c) for (e, a, b, c) in rows]
    cols = [(o, l) for o in range(len(orbits)) for l in range(len(nodes))]

    def entry(row, col):
        e, a, b, c = row
        o, l = col
        p0 = nodes[l]
        return sum(p0 ** (e + a + b + c) * (mp.mpf(v[0]) / R) ** a * (mp.mpf(v[1]) / R) ** b
                   * (mp.mpf(v[2]) / R) ** c for v in orbits[o])

    A = mp.matrix(len(rows), len(cols))
    for i, row in enumerate(rows):
        for j, col in enumerate(cols):
            A[i, j] = entry(row, col)
    b = mp.matrix(rhs)

    # Support selection in float64: fewest populations, every direction used.
    Af = np.array(A.tolist(), dtype=float)
    bf = np.array([float(x) for x in rhs])
    U, S, Vt = np.linalg.svd(Af, full_matrices=False)
    rank = int((S > 1e-10 * S[0]).sum())
    Ar, br = S[:rank, None] * Vt[:rank], U[:, :rank].T @ bf
    n = len(cols)
    sizes = np.array([len(orbits[o]) for o, _ in cols], dtype=float)
    cover = np.zeros((len(orbits), 2 * n))
    for j, (o, _) in enumerate(cols):
        cover[o, n + j] = 1.0
    cons = [LinearConstraint(np.hstack([Ar, np.zeros((rank, n))]), br, br),
            LinearConstraint(np.hstack([np.eye(n), -np.eye(n)]), -np.inf, 0.0),
            LinearConstraint(cover, 1.0, np.inf)]
    res = milp(np.r_[np.zeros(n), sizes], constraints=cons,
               integrality=np.r_[np.zeros(n), np.ones(n)], bounds=Bounds(0.0, 1.0),
               options=dict(node_limit=2000, presolve=True))
    if res.x is None:
        raise RuntimeError("no quadrature found: " + res.message)
    support = [j for j in range(n) if res.x[j] > 1e-12]

    # Re-solve the equalities on the support in 50-digit arithmetic (least squares; the system is
    # consistent, the residual is checked below).
    As = mp.matrix(len(rows), len(support))
    for i in range(len(rows)):
        for k, j in enumerate(support):
            As[i, k] = A[i, j]
    ws, resid = mp.qr_solve(As, b)
    if resid > mp.mpf(10) ** -40 or min(ws) <= 0:
        raise RuntimeError("refinement failed: residual %s, min weight %s" % (resid, min(ws)))

    pops = []
    for k, j in enumerate(support):
        o, l = cols[j]
        wk = ws[k]  # each member of the orbit carries this weight
        for v in sorted(orbits[o], reverse=True):
            pops.append((v, l, nodes[l], wk))
    return dict(R2=R2, nodes=nodes, pops=pops, rank=rank, ndirs=len(dirs), nconds=len(rows))


def write(path, order, kmax, t):
    pops = t["pops"]
    # Order populations direction by direction (lexicographically descending), then by energy; a
    # direction and its mirror are listed next to each other.
    key = {}
    for v, l, p0, w in pops:
        rep = max(v, tuple(-x for x in v))
        key[(v, l)] = (tuple(-x for x in rep), l, v != rep)
    pops = sorted(pops, key=lambda p: key[(p[0], p[1])])
    with open(path, "w") as f:
        f.write("# Discrete-velocity quadrature of the order-%d relativistic lattice Boltzmann model.\n" % order)
        f.write("# p_i = p0_i (1, v_i / R), |v_i|^2 = R^2; weights w_i >= 0, w(v) = w(-v); the rest-frame\n")
        f.write("# moments of exp(-p0)/(4 pi) over d^3p/p0 are reproduced up to degree %d.\n" % kmax)
        f.write("# Generated by lattice/make_tables.py (%d independent conditions, rank %d, %d of %d\n"
                % (t["nconds"], t["rank"], len(pops), 2 * t["ndirs"] * len(t["nodes"]) // 2))
        f.write("# candidate populations).  Columns: vx vy vz level p0 w.\n")
        f.write("order %d\nR2 %d\nQ %d\nlevels %d\n" % (order, t["R2"], len(pops), len(t["nodes"])))
        for v, l, p0, w in pops:
            f.write("%d %d %d %d %s %s\n" % (v[0], v[1], v[2], l, mp.nstr(p0, 25, min_fixed=-1, max_fixed=1),
                                             mp.nstr(w, 25, min_fixed=-1, max_fixed=1)))


def main():
    t3 = build(41, [1, -20, 120, -240, 120], 6, "inversion")
    write(os.path.join(HERE, "d3q128.txt"), 3, 6, t3)
    t2 = build(9, [1, -12, 36, -24], 5, "cubic")
    write(os.path.join(HERE, "d3q66.txt"), 2, 5, t2)
    print("d3q128: Q=%d, d3q66: Q=%d" % (len(t3["pops"]), len(t2["pops"])))


if __name__ == "__main__":
    main()
