"""ctypes front end of the serial FP64 C oracle (rlb_oracle.c).  Test infrastructure only."""
import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rlb_oracle.c")
HDR = os.path.join(HERE, "gs_basis.h")
LIB = os.path.join(HERE, "_build", "librlb_oracle.so")
LATTICE_DIR = os.path.join(os.path.dirname(HERE), "lattice")
HBARC_GEV_FM = 0.1973269804

_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile rlb_oracle.c (plain gcc, strict ISO C so no FMA contraction)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                                                       os.path.getmtime(HDR)):
        tmp = LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
            lib.ora_feq3_over_w.argtypes = [d, d, dp, d, d, d, d]
            lib.ora_feq3_over_w.restype = d
            lib.ora_feq2_over_w.argtypes = [d, d, dp, d, d, d, d]
            lib.ora_feq2_over_w.restype = d
            lib.ora_equilibrium_cell.argtypes = [i, i, dp, dp, d, d, dp, dp]
            lib.ora_equilibrium_appendix_cell.argtypes = [i, i, ip, dp, dp, d, d, dp, dp]
            lib.ora_gs_table.argtypes = [i, i, ip, dp, dp]
            lib.ora_gs_table.restype = i
            lib.ora_moments_cell.argtypes = [i, i, ip, dp, dp, dp, dp]
            lib.ora_landau_cell.argtypes = [dp, dp, dp, dp, dp]
            lib.ora_landau_cell.restype = i
            lib.ora_tau_prime.argtypes = [d, d, d, d]
            lib.ora_tau_prime.restype = d
            lib.ora_step.argtypes = [i, i, ip, dp, dp, dp, i, i, i, ip, d, d, i, d, d, d, i, i, dp, dp, dp, dp]
            lib.ora_step.restype = l
            lib.ora_init_step_cells.argtypes = [i, i, ip, dp, dp, dp, i, i, i, ip, d, d, i, d, d, d, dp, dp, dp, l,
                                                ctypes.POINTER(ctypes.c_long), dp]
            lib.ora_init_step_cells.restype = l
            lib.ora_init.argtypes = [i, i, dp, dp, l, dp, dp, dp, dp]
            lib.ora_init.restype = i
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class Lattice:
    """A discrete-velocity quadrature: p_i = p0_i (1, v_i / R) with weights w_i (Eq. (eq:mrecon2))."""

    def __init__(self, order, R2, v, level, p0, w):
        self.order = int(order)
        self.R2 = int(R2)
        self.R = float(np.sqrt(R2))
        self.v = np.ascontiguousarray(v, dtype=np.int32)
        self.level = np.asarray(level, dtype=np.int32)
        self.p0 = np.ascontiguousarray(p0, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.q = len(self.w)
        self._gs = None

    @property
    def gs(self):
        """P_k(p_i) of the Gram-Schmidt basis for every population, shape (q, 30 or 14)."""
        if self._gs is None:
            nm = 30 if self.order == 3 else 14
            tab = np.empty((self.q, nm))
            _load().ora_gs_table(self.order, self.q, _ip(self.v), _dp(self.p0), _dp(tab))
            self._gs = tab
        return self._gs

    def momenta(self):
        """(q, 4) array of p_i^mu."""
        return np.column_stack([self.p0, self.p0[:, None] * self.v / self.R])


def lattice_path(order):
    return os.path.join(LATTICE_DIR, "d3q128.txt" if order == 3 else "d3q66.txt")


def read_lattice(order_or_path):
    path = lattice_path(order_or_path) if isinstance(order_or_path, int) else order_or_path
    hdr, rows = {}, []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if len(parts) == 2:
                hdr[parts[0]] = int(parts[1])
            else:
                rows.append(parts)
    v = [[int(r[0]), int(r[1]), int(r[2])] for r in rows]
    lat = Lattice(hdr["order"], hdr["R2"], v, [int(r[3]) for r in rows], [float(r[4]) for r in rows],
                  [float(r[5]) for r in rows])
    assert lat.q == hdr["Q"]
    return lat


def tau_prime(eta_over_s, R, T, dx_fm=0.008, T_unit_GeV=0.4):
    kappa = T_unit_GeV * dx_fm / HBARC_GEV_FM
    return _load().ora_tau_prime(float(eta_over_s), float(R), kappa, float(T))


def equilibrium_cell(lat, n, T, U):
    """f_i^eq = w_i sum_k a_k J_k(p_i) of one cell (Eqs. (coeff), (eq:disc1))."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty(lat.q)
    _load().ora_equilibrium_cell(lat.order, lat.q, _dp(lat.w), _dp(lat.gs), float(n), float(T), _dp(U), _dp(out))
    return out


def equilibrium_appendix_cell(lat, n, T, U):
    """f_i^eq of one cell from the explicit App. B formula (Eq. (eq:equi3rd) / (eq:equi2nd))."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty(lat.q)
    _load().ora_equilibrium_appendix_cell(lat.order, lat.q, _ip(lat.v), _dp(lat.p0), _dp(lat.w), float(n),
                                          float(T), _dp(U), _dp(out))
    return out


def moments_cell(lat, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    N = np.empty(4)
    Tm = np.empty(16)
    _load().ora_moments_cell(lat.order, lat.q, _ip(lat.v), _dp(lat.p0), _dp(f), _dp(N), _dp(Tm))
    return N, Tm.reshape(4, 4)


def landau_cell(N, Tm):
    """Returns (status, U, eps, n) of the Landau-frame solve."""
    N = np.ascontiguousarray(N, dtype=np.float64)
    Tm = np.ascontiguousarray(Tm, dtype=np.float64).reshape(16)
    U = np.empty(4)
    e = ctypes.c_double()
    n = ctypes.c_double()
    st = _load().ora_landau_cell(_dp(N), _dp(Tm), _dp(U), ctypes.byref(e), ctypes.byref(n))
    return st, U, e.value, n.value


class OracleRLB:
    """Serial FP64 reference simulation with the same state semantics as the GPU library.

    The stored state is post-collision.  ``moments()`` reports the Landau fields of the pre-collision
    populations of the current time level: the initial populations before any step, afterwards the
    pull of the previous state (what the last step collided)."""

    def __init__(self, lat, nx, ny, nz, bc=(0, 0, 0), eta_over_s=0.1, tau_prime=0.0, tau_local_T=1, T_ref=1.0,
                 dx_fm=0.008, T_unit_GeV=0.4):
        """bc per axis (x, y, z): 0 periodic, 1 copy-out, 2 bounce-back wall."""
        self.lat = lat
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.cells = nx * ny * nz
        self.bc = np.ascontiguousarray(bc, dtype=np.int32)
        self.eta_over_s, self.tau_prime, self.tau_local_T = float(eta_over_s), float(tau_prime), int(tau_local_T)
        self.T_ref, self.dx_fm, self.T_unit_GeV = float(T_ref), float(dx_fm), float(T_unit_GeV)
        self.f = np.zeros((lat.q,) + self.shape)
        self.prev = None
        self.steps = 0
        self.nonconv = 0

    def init(self, n, T, u):
        n = np.ascontiguousarray(np.broadcast_to(n, self.shape), dtype=np.float64)
        T = np.ascontiguousarray(np.broadcast_to(T, self.shape), dtype=np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (3,) + self.shape), dtype=np.float64)
        lat = self.lat
        st = _load().ora_init(lat.order, lat.q, _dp(lat.w), _dp(lat.gs), self.cells, _dp(n), _dp(T), _dp(u),
                              _dp(self.f))
        if st != 0:
            raise ValueError("invalid initial fields")
        self.prev, self.steps = None, 0

    def set_populations(self, f):
        self.f = np.array(f, dtype=np.float64, copy=True).reshape((self.lat.q,) + self.shape)
        self.prev, self.steps = None, 0

    def _call(self, fin, fout, pull, collide, fields=None, dens=None):
        lat = self.lat
        bad = _load().ora_step(lat.order, lat.q, _ip(lat.v), _dp(lat.p0), _dp(lat.w), _dp(lat.gs), self.nx,
                               self.ny, self.nz,
                               _ip(self.bc), self.eta_over_s, self.tau_prime, self.tau_local_T, self.T_ref,
                               self.dx_fm, self.T_unit_GeV, pull, collide, _dp(fin), _dp(fout), _dp(fields),
                               _dp(dens))
        if bad < 0:
            raise ValueError("bounce-back walls need a reversed partner for every population")
        return bad

    def step(self, k=1):
        for _ in range(k):
            out = np.empty_like(self.f)
            self.nonconv += self._call(self.f, out, 1, 1)
            self.prev, self.f = self.f, out
            self.steps += 1
        return self.nonconv

    def init_step_cells(self, n, T, u, sample):
        """Populations (len(sample), q) after one step from the equilibrium of (n, T, u), computed
        only at the listed cells (flat indices, x fastest)."""
        n = np.ascontiguousarray(np.broadcast_to(n, self.shape), dtype=np.float64)
        T = np.ascontiguousarray(np.broadcast_to(T, self.shape), dtype=np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (3,) + self.shape), dtype=np.float64)
        sample = np.ascontiguousarray(sample, dtype=np.int64)
        out = np.empty((len(sample), self.lat.q))
        lat = self.lat
        bad = _load().ora_init_step_cells(
            lat.order, lat.q, _ip(lat.v), _dp(lat.p0), _dp(lat.w), _dp(lat.gs), self.nx, self.ny, self.nz,
            _ip(self.bc),
            self.eta_over_s, self.tau_prime, self.tau_local_T, self.T_ref, self.dx_fm, self.T_unit_GeV, _dp(n),
            _dp(T), _dp(u), len(sample), sample.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out))
        if bad < 0:
            raise ValueError("invalid fields")
        return out

    def moments(self):
        """(n, eps, U[4], totals[5]) at the current time level; totals = sum N^0, T^00, T^0x, T^0y, T^0z."""
        fields = np.empty((6,) + self.shape)
        dens = np.empty((5,) + self.shape)
        if self.prev is None:
            self._call(self.f, self.f, 0, 0, fields, dens)
        else:
            self._call(self.prev, self.prev, 1, 0, fields, dens)
        totals = np.array([np.sum(dens[k], dtype=np.float64) for k in range(5)])
        return fields[0], fields[1], fields[2:6], totals
