"""The C-ABI library builds, loads and exports what include/rlb.h declares (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1301_3423_gb300 import rlb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rlb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rlb_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = rlb.load()
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(rlb.DECLARED) == names


def test_params_layout_matches_c():
    """rlb_default_params fills the ctypes mirror field by field and writes nothing past it."""
    lib = rlb.load()
    buf = (ctypes.c_ubyte * (ctypes.sizeof(rlb.Params) + 64))()
    ctypes.memset(buf, 0xAB, len(buf))
    p = rlb.Params.from_buffer(buf)
    lib.rlb_default_params(ctypes.byref(p))
    assert all(b == 0xAB for b in bytes(buf)[ctypes.sizeof(rlb.Params):])
    assert (p.order, p.nx, p.ny, p.nz, list(p.bc)) == (3, 1, 1, 1, [0, 0, 0])
    assert (p.eta_over_s, p.tau_prime, p.tau_local_T, p.T_ref) == (0.1, 0.0, 1, 1.0)
    assert (p.dx_fm, p.T_unit_GeV, p.storage, p.landau_fp64) == (0.008, 0.4, 0, 0)
    assert (p.gamma_thr, p.n_ref, p.step_variant, p.stream, p.q) == (2.0, 1.0, -1, None, 0)
    assert p.debug_flags == 0


@pytest.mark.parametrize("order", [3, 2])
def test_builtin_quadrature_is_the_committed_table(order):
    """The kernels' compile-time table equals the committed quadrature bit for bit."""
    q = rlb.quadrature(order)
    lat = oracle.read_lattice(order)
    assert np.array_equal(q["v"], lat.v)
    assert np.array_equal(q["level"], lat.level)
    assert np.array_equal(q["p0"], lat.p0)
    assert np.array_equal(q["w"], lat.w)


def test_bytes_required():
    b = rlb.RLB.bytes_required(order=3, nx=256, ny=256, nz=256, storage="f32")
    cells = 256 ** 3
    assert b >= 2 * 128 * cells * 4 + 6 * cells * 8
    assert b < 2 * 128 * cells * 4 * 1.1
    assert rlb.RLB.bytes_required(order=5) == 0


@pytest.mark.parametrize("bad", [dict(order=4), dict(nx=0), dict(storage=7), dict(eta_over_s=-1.0),
                                 dict(gamma_thr=0.5), dict(bc=(0, 3, 0)), dict(step_variant=24)])
def test_create_rejects_invalid_parameters(bad):
    """Validation happens on the host before any device call."""
    kw = dict(shape=(4, 4, 4))
    kw.update({k: v for k, v in bad.items() if k not in ("nx",)})
    if "nx" in bad:
        kw["shape"] = (4, 4, bad["nx"])
    with pytest.raises(rlb.RLBError) as e:
        rlb.RLB(**kw)
    assert e.value.status == rlb.RLB_EINVAL
    assert "rlb_create" in str(e.value)


def test_create_rejects_a_different_quadrature():
    q = rlb.quadrature(3)
    q["w"] = q["w"].copy()
    q["w"][5] *= 1.0 + 1e-15
    with pytest.raises(rlb.RLBError) as e:
        rlb.RLB((4, 4, 4), quadrature=q)
    assert "population 5" in str(e.value)
