"""Python binding of librlb (include/rlb.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module converts numpy arrays and
torch tensors to pointers and statuses to exceptions.  numpy arrays are passed as host buffers,
CUDA tensors as device buffers.  There is no CPU fallback: if the library cannot be loaded the
import fails.
"""
import ctypes
import os

import numpy as np

from . import builder as _build

RLB_OK, RLB_EINVAL, RLB_ENOMEM, RLB_ECUDA, RLB_ENONCONV, RLB_ENAN, RLB_ETIMEOUT, RLB_ESTATE = range(8)
STATUS_NAMES = ["RLB_OK", "RLB_EINVAL", "RLB_ENOMEM", "RLB_ECUDA", "RLB_ENONCONV", "RLB_ENAN", "RLB_ETIMEOUT",
                "RLB_ESTATE"]
STORAGE = {"f64": 0, "f32": 1, "f16dev": 2}
MAX_VARIANTS = 24
VARIANT_NAMES = ["registers/scalar", "registers/paired", "registers(168)/scalar", "registers(168)/paired",
                 "pipe tx128 8c8p", "pipe tx128 8c4p", "pipe tx64 8c8p", "pipe tx64 4c4p", "pipe tx128 8c6p",
                 "pipe tx64 8c4p", "pipe tx128 4c4p", "pipe tx64 2c4p", "rows tx128 8c4p", "rows tx128 8c8p",
                 "rows tx128 4c4p", "pipe tx128 12c4p 1w", "rows tx128 12c4p 1w", "pipe tx128 12c2p 1w",
                 "rows tx128 12c2p 1w", "rows tx96 12c4p 1w"]
BC = {"periodic": 0, "copyout": 1, "bounceback": 2}


class RLBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


class Params(ctypes.Structure):
    """Mirror of rlb_params (include/rlb.h); field order and types must match."""
    _fields_ = [
        ("order", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("eta_over_s", ctypes.c_double),
        ("tau_prime", ctypes.c_double),
        ("tau_local_T", ctypes.c_int),
        ("T_ref", ctypes.c_double),
        ("dx_fm", ctypes.c_double),
        ("T_unit_GeV", ctypes.c_double),
        ("storage", ctypes.c_int),
        ("landau_fp64", ctypes.c_int),
        ("gamma_thr", ctypes.c_double),
        ("n_ref", ctypes.c_double),
        ("step_variant", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("debug_flags", ctypes.c_int),
        ("q", ctypes.c_int),
        ("vel", ctypes.POINTER(ctypes.c_int)),
        ("level", ctypes.POINTER(ctypes.c_int)),
        ("p0", ctypes.POINTER(ctypes.c_double)),
        ("w", ctypes.POINTER(ctypes.c_double)),
    ]


_LIB = None
_LOAD_ERROR = None
DECLARED = ["rlb_default_params", "rlb_bytes_required", "rlb_create", "rlb_init", "rlb_step", "rlb_moments",
            "rlb_sync", "rlb_get_populations", "rlb_set_populations", "rlb_steps_done", "rlb_step_variant", "rlb_kernel_launches",
            "rlb_destroy", "rlb_last_error", "rlb_quadrature", "rlb_autotune", "rlb_totals_noalloc", "rlb_batch_create", "rlb_batch_add",
            "rlb_batch_remove", "rlb_batch_steps_left", "rlb_batch_run", "rlb_batch_autotune",
            "rlb_batch_set_variant", "rlb_batch_member_variant", "rlb_batch_kernel_launches", "rlb_batch_last_error",
            "rlb_batch_destroy"]


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load librlb.so (building it first if it is missing)."""
    global _LIB, _LOAD_ERROR
    if _LIB is not None:
        return _LIB
    if _LOAD_ERROR is not None:  # fail fast: a broken build is not retried in the same process
        raise _LOAD_ERROR
    try:
        path = _build.build() if build_if_missing else _build.LIB
    except Exception as e:
        _LOAD_ERROR = RuntimeError("librlb could not be built: %s" % e)
        raise _LOAD_ERROR
    lib = ctypes.CDLL(path)
    P, vp, dp, ip = ctypes.POINTER(Params), ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.rlb_default_params.argtypes = [P]
    lib.rlb_default_params.restype = None
    lib.rlb_bytes_required.argtypes = [P]
    lib.rlb_bytes_required.restype = ctypes.c_size_t
    lib.rlb_create.argtypes = [P, ctypes.POINTER(vp)]
    lib.rlb_create.restype = ip
    lib.rlb_init.argtypes = [vp, vp, vp, vp, ip]
    lib.rlb_init.restype = ip
    lib.rlb_step.argtypes = [vp, ctypes.c_long]
    lib.rlb_step.restype = ip
    lib.rlb_moments.argtypes = [vp, vp, vp, vp, dp, ip]
    lib.rlb_moments.restype = ip
    lib.rlb_sync.argtypes = [vp]
    lib.rlb_sync.restype = ip
    lib.rlb_get_populations.argtypes = [vp, vp, ip]
    lib.rlb_get_populations.restype = ip
    lib.rlb_set_populations.argtypes = [vp, vp, ip]
    lib.rlb_set_populations.restype = ip
    lib.rlb_steps_done.argtypes = [vp]
    lib.rlb_steps_done.restype = ctypes.c_long
    lib.rlb_step_variant.argtypes = [vp]
    lib.rlb_step_variant.restype = ip
    lib.rlb_kernel_launches.argtypes = [vp]
    lib.rlb_kernel_launches.restype = ctypes.c_long
    lib.rlb_destroy.argtypes = [vp]
    lib.rlb_destroy.restype = ip
    lib.rlb_last_error.argtypes = [vp]
    lib.rlb_last_error.restype = ctypes.c_char_p
    lib.rlb_quadrature.argtypes = [ip, ctypes.POINTER(ip), ctypes.POINTER(ctypes.POINTER(ctypes.c_int)),
                                   ctypes.POINTER(ctypes.POINTER(ctypes.c_int)), ctypes.POINTER(dp),
                                   ctypes.POINTER(dp)]
    lib.rlb_quadrature.restype = ip
    lib.rlb_autotune.argtypes = [vp, ip, ctypes.POINTER(ip), dp]
    lib.rlb_autotune.restype = ip
    lib.rlb_totals_noalloc.argtypes = [ip, ip, ip, ip, ip, ctypes.c_double, vp, dp, vp]
    lib.rlb_totals_noalloc.restype = ip
    lib.rlb_batch_create.argtypes = [ip, ip, vp, ctypes.POINTER(vp)]
    lib.rlb_batch_create.restype = ip
    lib.rlb_batch_add.argtypes = [vp, vp, ctypes.c_long, ctypes.POINTER(ip)]
    lib.rlb_batch_add.restype = ip
    lib.rlb_batch_remove.argtypes = [vp, ip]
    lib.rlb_batch_remove.restype = ip
    lib.rlb_batch_steps_left.argtypes = [vp, ip]
    lib.rlb_batch_steps_left.restype = ctypes.c_long
    lib.rlb_batch_run.argtypes = [vp, ctypes.c_long, ip, ctypes.POINTER(ip)]
    lib.rlb_batch_run.restype = ip
    lib.rlb_batch_autotune.argtypes = [vp, ip, ctypes.POINTER(ip), dp]
    lib.rlb_batch_autotune.restype = ip
    lib.rlb_batch_set_variant.argtypes = [vp, ip]
    lib.rlb_batch_set_variant.restype = ip
    lib.rlb_batch_member_variant.argtypes = [vp, ip]
    lib.rlb_batch_member_variant.restype = ip
    lib.rlb_batch_kernel_launches.argtypes = [vp]
    lib.rlb_batch_kernel_launches.restype = ctypes.c_long
    lib.rlb_batch_last_error.argtypes = [vp]
    lib.rlb_batch_last_error.restype = ctypes.c_char_p
    lib.rlb_batch_destroy.argtypes = [vp]
    lib.rlb_batch_destroy.restype = ip
    _LIB = lib
    return lib


def quadrature(order):
    """The library's built-in quadrature: dict(v[q,3], level[q], p0[q], w[q])."""
    lib = load()
    q = ctypes.c_int()
    v, lev = ctypes.POINTER(ctypes.c_int)(), ctypes.POINTER(ctypes.c_int)()
    p0, w = ctypes.POINTER(ctypes.c_double)(), ctypes.POINTER(ctypes.c_double)()
    st = lib.rlb_quadrature(order, ctypes.byref(q), ctypes.byref(v), ctypes.byref(lev), ctypes.byref(p0),
                            ctypes.byref(w))
    if st != RLB_OK:
        raise RLBError(st, "no built-in quadrature for order %r" % order)
    n = q.value
    return dict(v=np.ctypeslib.as_array(v, (n, 3)).copy(), level=np.ctypeslib.as_array(lev, (n,)).copy(),
                p0=np.ctypeslib.as_array(p0, (n,)).copy(), w=np.ctypeslib.as_array(w, (n,)).copy())


def totals_noalloc(f, order, storage, shape, n_ref=1.0, stream=None):
    """rlb_totals_noalloc: sum over cells of N^0, T^00, T^0x, T^0y, T^0z of the populations in the
    CUDA tensor ``f`` (storage layout [q][cells]), with no allocation inside the library."""
    lib = load()
    nz, ny, nx = shape
    st_code = STORAGE[storage] if isinstance(storage, str) else int(storage)
    if not _is_cuda_tensor(f) or not f.is_contiguous():
        raise ValueError("f must be a contiguous CUDA tensor")
    import torch
    want = {0: torch.float64, 1: torch.float32, 2: torch.float16}.get(st_code)
    q = {3: 128, 2: 66}.get(int(order))
    if want is None or q is None:
        raise ValueError("order must be 2 or 3 and storage one of %s" % sorted(STORAGE))
    # the library reads q * cells elements of the storage type: check the buffer holds exactly that
    if f.dtype != want or f.numel() != q * nx * ny * nz:
        raise ValueError("f must hold %d x %d elements of %s, got %d of %s" % (q, nx * ny * nz, want, f.numel(),
                                                                              f.dtype))
    tot = (ctypes.c_double * 5)()
    sp = None if stream is None else ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    st = lib.rlb_totals_noalloc(order, st_code, nx, ny, nz, n_ref, ctypes.c_void_p(f.data_ptr()), tot, sp)
    if st != RLB_OK:
        raise RLBError(st, lib.rlb_last_error(None).decode())
    return np.array(tot[:])


def read_quadrature_file(path):
    """Parse a committed quadrature file (lattice/*.txt): dict(order, R2, v, level, p0, w)."""
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
    return dict(order=hdr["order"], R2=hdr["R2"], v=np.array([[int(x) for x in r[:3]] for r in rows], np.int32),
                level=np.array([int(r[3]) for r in rows], np.int32), p0=np.array([float(r[4]) for r in rows]),
                w=np.array([float(r[5]) for r in rows]))


def _is_cuda_tensor(x):
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x, n_expected, name):
    """(pointer, on_device, keepalive) of a float64 array or tensor with n_expected elements."""
    if _is_cuda_tensor(x):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != n_expected:
            raise ValueError("%s must be a contiguous float64 CUDA tensor with %d elements" % (name, n_expected))
        return ctypes.c_void_p(x.data_ptr()), 1, x
    a = np.ascontiguousarray(x, dtype=np.float64)
    if a.size != n_expected:
        raise ValueError("%s must have %d elements, got %d" % (name, n_expected, a.size))
    return ctypes.c_void_p(a.ctypes.data), 0, a


class RLB:
    """One simulation context on the current CUDA device (rlb_create ... rlb_destroy).

    shape = (nz, ny, nx); arrays follow the library's layout (x fastest): scalar fields (nz, ny, nx),
    u (3, nz, ny, nx), U (4, nz, ny, nx), populations (q, nz, ny, nx)."""

    def __init__(self, shape, order=3, bc=("periodic", "periodic", "periodic"), eta_over_s=0.1, tau_prime=0.0,
                 tau_local_T=True, T_ref=1.0, dx_fm=0.008, T_unit_GeV=0.4, storage="f64", landau_fp64=False,
                 gamma_thr=2.0, n_ref=1.0, stream=None, quadrature=None, step_variant=-1, debug_flags=0):
        self._lib = load()
        nz, ny, nx = shape
        p = Params()
        self._lib.rlb_default_params(ctypes.byref(p))
        p.order, p.nx, p.ny, p.nz = order, nx, ny, nz
        for a, b in enumerate(bc):
            p.bc[a] = BC[b] if isinstance(b, str) else int(b)
        p.eta_over_s, p.tau_prime, p.tau_local_T = eta_over_s, tau_prime, int(bool(tau_local_T))
        p.T_ref, p.dx_fm, p.T_unit_GeV = T_ref, dx_fm, T_unit_GeV
        p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        p.landau_fp64, p.gamma_thr, p.n_ref = int(bool(landau_fp64)), gamma_thr, n_ref
        p.step_variant = int(step_variant)
        p.debug_flags = int(debug_flags)
        if stream is not None:
            p.stream = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        self._keep = []
        if quadrature is not None:
            v = np.ascontiguousarray(quadrature["v"], dtype=np.int32).reshape(-1)
            lev = np.ascontiguousarray(quadrature["level"], dtype=np.int32)
            p0 = np.ascontiguousarray(quadrature["p0"], dtype=np.float64)
            w = np.ascontiguousarray(quadrature["w"], dtype=np.float64)
            self._keep += [v, lev, p0, w]
            p.q = len(w)
            p.vel = v.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
            p.level = lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
            p.p0 = p0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            p.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.params = p
        h = ctypes.c_void_p()
        st = self._lib.rlb_create(ctypes.byref(p), ctypes.byref(h))
        if st != RLB_OK:
            raise RLBError(st, self._lib.rlb_last_error(None).decode())
        self._h = h
        self.shape = (nz, ny, nx)
        self.cells = nx * ny * nz
        self.order = order
        self.q = 128 if order == 3 else 66

    # -- helpers --------------------------------------------------------------------------------
    def _check(self, st):
        if st != RLB_OK:
            raise RLBError(st, self._lib.rlb_last_error(self._h).decode())

    @staticmethod
    def bytes_required(**kw):
        lib = load()
        p = Params()
        lib.rlb_default_params(ctypes.byref(p))
        for k, v in kw.items():
            if k == "bc":
                for a, b in enumerate(v):
                    p.bc[a] = BC[b] if isinstance(b, str) else int(b)
            elif k == "storage":
                p.storage = STORAGE[v] if isinstance(v, str) else int(v)
            else:
                setattr(p, k, v)
        return int(lib.rlb_bytes_required(ctypes.byref(p)))

    # -- the C ABI ------------------------------------------------------------------------------
    def init(self, n, T, u):
        """rlb_init: populations = discrete equilibrium of (n, T, u)."""
        pn, dn, kn = _ptr(n, self.cells, "n")
        pT, dT, kT = _ptr(T, self.cells, "T")
        pu, du, ku = _ptr(u, 3 * self.cells, "u")
        if not (dn == dT == du):
            raise ValueError("n, T, u must all be host arrays or all CUDA tensors")
        self._check(self._lib.rlb_init(self._h, pn, pT, pu, dn))

    def step(self, nsteps=1):
        self._check(self._lib.rlb_step(self._h, int(nsteps)))

    def sync(self):
        self._check(self._lib.rlb_sync(self._h))

    def moments(self, out=None):
        """rlb_moments: dict(n, eps, U, totals).  ``out`` = dict(n, eps, U) of float64 CUDA tensors
        (device outputs) or of C-contiguous float64 numpy arrays (host outputs, e.g. pinned)."""
        tot = (ctypes.c_double * 5)()
        if out is None:
            out = dict(n=np.empty(self.shape), eps=np.empty(self.shape), U=np.empty((4,) + self.shape))
        n, eps, U = out["n"], out["eps"], out["U"]
        ptrs = []
        for x, k, name in ((n, 1, "n"), (eps, 1, "eps"), (U, 4, "U")):
            if not _is_cuda_tensor(x) and not (isinstance(x, np.ndarray) and x.dtype == np.float64
                                                and x.flags.c_contiguous):
                raise ValueError("%s must be a float64 CUDA tensor or C-contiguous float64 array" % name)
            ptrs.append(_ptr(x, k * self.cells, name))
        devs = {d for _, d, _ in ptrs}
        if len(devs) != 1:
            raise ValueError("outputs must all be host arrays or all CUDA tensors")
        self._check(self._lib.rlb_moments(self._h, ptrs[0][0], ptrs[1][0], ptrs[2][0], tot, devs.pop()))
        return dict(n=n, eps=eps, U=U, totals=np.array(tot[:]))

    def populations(self, out=None):
        """rlb_get_populations: (q, nz, ny, nx) float64 (host array, or into a CUDA tensor ``out``)."""
        if out is None:
            f = np.empty((self.q,) + self.shape)
            self._check(self._lib.rlb_get_populations(self._h, ctypes.c_void_p(f.ctypes.data), 0))
            return f
        p, dev, _ = _ptr(out, self.q * self.cells, "out")
        self._check(self._lib.rlb_get_populations(self._h, p, dev))
        return out

    def set_populations(self, f):
        p, dev, keep = _ptr(f, self.q * self.cells, "f")
        self._check(self._lib.rlb_set_populations(self._h, p, dev))
        if dev:
            self.sync()

    def autotune(self, reps=5):
        """rlb_autotune: (chosen variant, ms per step of each variant)."""
        v = ctypes.c_int()
        ms = (ctypes.c_double * MAX_VARIANTS)()
        self._check(self._lib.rlb_autotune(self._h, int(reps), ctypes.byref(v), ms))
        n = max([i + 1 for i, x in enumerate(ms) if x > 0] or [1])
        return v.value, list(ms)[:n]

    @property
    def variant(self):
        """The step-kernel variant rlb_step uses."""
        return int(self._lib.rlb_step_variant(self._h))

    @property
    def steps_done(self):
        return int(self._lib.rlb_steps_done(self._h))

    @property
    def kernel_launches(self):
        return int(self._lib.rlb_kernel_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rlb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """rlb_batch_*: step many RLB contexts (same order and storage) together, each time step two
    persistent launches over shared tile queues (the members' interior rows, then their boundary
    cells), optionally replaying CUDA graphs of several steps."""

    def __init__(self, order=3, storage="f32", stream=None):
        self._lib = load()
        h = ctypes.c_void_p()
        st_code = STORAGE[storage] if isinstance(storage, str) else int(storage)
        sp = None if stream is None else ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        st = self._lib.rlb_batch_create(order, st_code, sp, ctypes.byref(h))
        if st != RLB_OK:
            raise RLBError(st, "rlb_batch_create failed")
        self._h = h
        self._members = {}

    def _check(self, st):
        if st != RLB_OK:
            raise RLBError(st, self._lib.rlb_batch_last_error(self._h).decode())

    def add(self, ctx, steps):
        slot = ctypes.c_int()
        self._check(self._lib.rlb_batch_add(self._h, ctx._h, int(steps), ctypes.byref(slot)))
        self._members[slot.value] = ctx
        return slot.value

    def remove(self, slot):
        self._check(self._lib.rlb_batch_remove(self._h, int(slot)))
        self._members.pop(slot, None)

    def steps_left(self, slot):
        return int(self._lib.rlb_batch_steps_left(self._h, int(slot)))

    def run(self, nsteps, graph=True):
        act = ctypes.c_int()
        self._check(self._lib.rlb_batch_run(self._h, int(nsteps), int(bool(graph)), ctypes.byref(act)))
        return act.value

    def autotune(self, reps=3):
        v = ctypes.c_int()
        ms = (ctypes.c_double * MAX_VARIANTS)()
        self._check(self._lib.rlb_batch_autotune(self._h, int(reps), ctypes.byref(v), ms))
        n = max([i + 1 for i, x in enumerate(ms) if x > 0] or [1])
        return v.value, list(ms)[:n]

    def set_variant(self, v):
        self._check(self._lib.rlb_batch_set_variant(self._h, int(v)))

    def member_variant(self, slot):
        """The step variant the batch runs the member in `slot` with (rlb_batch_member_variant)."""
        return int(self._lib.rlb_batch_member_variant(self._h, int(slot)))

    @property
    def kernel_launches(self):
        return int(self._lib.rlb_batch_kernel_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rlb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

