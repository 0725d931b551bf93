"""Build step: turn the committed quadrature files (lattice/d3q128.txt, lattice/d3q66.txt) into
compile-time C++ tables for the kernels (rlb_quadrature.h in the build directory).

The quadrature (directions v_i with |v_i|^2 = R^2, energies p0_l, weights w_i; Sec. II.C and App. A)
is data of the model.  The kernels need it as constant expressions so that zero velocity
components, mirror pairs and energy levels are resolved at compile time.

Populations in the files come in mirror pairs (2k, 2k+1) = (v, -v) at the same energy, grouped by
direction; the header records that grouping (direction pairs, their population pairs)."""
import math
import os
import sys


def read(path):
    hdr, rows = {}, []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        parts = line.split()
        if len(parts) == 2:
            hdr[parts[0]] = int(parts[1])
        else:
            rows.append(parts)
    return hdr, rows


def emit(name, path):
    hdr, rows = read(path)
    q = hdr["Q"]
    v = [(int(r[0]), int(r[1]), int(r[2])) for r in rows]
    lev = [int(r[3]) for r in rows]
    p0_txt = {}
    for r in rows:
        p0_txt.setdefault(int(r[3]), r[4])
    w_txt = [r[5] for r in rows]
    nlev = hdr["levels"]
    assert sorted(p0_txt) == list(range(nlev))
    # mirror pairs are adjacent and share energy and weight
    for k in range(0, q, 2):
        assert v[k + 1] == tuple(-x for x in v[k]) and lev[k] == lev[k + 1] and w_txt[k] == w_txt[k + 1], k
    # direction pairs: consecutive population pairs with the same "+" direction
    dp_first, dp_count, dp_v = [], [], []
    for k in range(0, q, 2):
        if not dp_v or dp_v[-1] != v[k]:
            dp_first.append(k)
            dp_count.append(0)
            dp_v.append(v[k])
        dp_count[-1] += 1
    assert len(set(dp_v)) == len(dp_v), "population pairs of one direction must be contiguous"
    vmax = [max(abs(x[a]) for x in v) for a in range(3)]

    def arr(xs):
        return "{" + ", ".join(str(x) for x in xs) + "}"

    out = []
    out.append("struct %s {" % name)
    out.append("  static constexpr int ORDER = %d, Q = %d, NLEV = %d, R2 = %d, NDP = %d;" %
               (hdr["order"], q, nlev, hdr["R2"], len(dp_v)))
    out.append("  static constexpr int VMAX_X = %d, VMAX_Y = %d, VMAX_Z = %d;" % tuple(vmax))
    R = math.sqrt(hdr["R2"])
    out.append("  static constexpr double R = %r, INV_R = %r, INV_R2 = %r;" % (R, 1.0 / R, 1.0 / hdr["R2"]))
    out.append("  static constexpr int VX[Q] = %s;" % arr(x[0] for x in v))
    out.append("  static constexpr int VY[Q] = %s;" % arr(x[1] for x in v))
    out.append("  static constexpr int VZ[Q] = %s;" % arr(x[2] for x in v))
    out.append("  static constexpr int LEV[Q] = %s;" % arr(lev))
    out.append("  static constexpr double P0[NLEV] = %s;" % arr(p0_txt[l] for l in range(nlev)))
    out.append("  static constexpr double W[Q] = %s;" % arr(w_txt))
    out.append("  static constexpr int DP_FIRST[NDP] = %s;" % arr(dp_first))
    out.append("  static constexpr int DP_NPAIR[NDP] = %s;" % arr(dp_count))
    out.append("};")
    return "\n".join(out)


def main(lattice_dir, out_path):
    body = ["// Generated at build time from the committed quadrature files; do not edit.",
            "#pragma once",
            emit("Quad3", os.path.join(lattice_dir, "d3q128.txt")),
            emit("Quad2", os.path.join(lattice_dir, "d3q66.txt")), ""]
    tmp = out_path + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(body))
    os.replace(tmp, out_path)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
