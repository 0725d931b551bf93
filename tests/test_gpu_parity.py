"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances:
  * double storage: per population |f_gpu - f_oracle| <= 1e-12 * max(|f_oracle|, w_i n_max / 2);
  * float / half-deviation storage: fields n, eps pointwise relative, u as
    max|du| / max(max|u_ref|, 0.01), against the FP64 oracle (1e-5 for float).
"""
import numpy as np
import pytest

import oracle
from paper_inputs import fields as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1301_3423_gb300 import RLB, RLBError  # noqa: E402
from paper_1301_3423_gb300 import rlb as rlbmod  # noqa: E402


def pop_scale(lat, f_ref, n_max):
    return np.maximum(np.abs(f_ref), (lat.w * n_max / 2).reshape((-1,) + (1,) * (f_ref.ndim - 1)))


def pop_err(lat, f_gpu, f_ref, n_max):
    return float(np.max(np.abs(f_gpu - f_ref) / pop_scale(lat, f_ref, n_max)))


def field_err(ref, got):
    """(n rel, eps rel, u) errors of the Landau fields."""
    en = np.max(np.abs(got["n"] - ref[0]) / np.abs(ref[0]))
    ee = np.max(np.abs(got["eps"] - ref[1]) / np.abs(ref[1]))
    u_ref = ref[2][1:] / ref[2][0]
    u_got = got["U"][1:] / got["U"][0]
    du = np.max(np.sqrt(((u_got - u_ref) ** 2).sum(axis=0)))
    eu = du / max(np.max(np.sqrt((u_ref ** 2).sum(axis=0))), 0.01)
    return float(en), float(ee), float(eu)


def near_equilibrium(lat, shape, seed, amp=0.02, vmax=0.4, bc=(0, 0, 0)):
    n, T, u = gen.smooth_random_fields(shape, seed=seed, vmax=vmax, sigma_lnT=0.15)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], bc=bc)
    o.init(n, T, u)
    rng = np.random.default_rng(seed + 7)
    return o.f + amp * (lat.w[:, None, None, None] * n[None] / 2) * rng.standard_normal(o.f.shape)


BCS = {"periodic": (0, 0, 0), "copyout_z": (0, 0, 1), "copyout_xy": (1, 1, 0), "walls_xz": (2, 0, 2),
       "box": (2, 2, 2)}


@pytest.mark.parametrize("order", [3, 2])
def test_init_matches_oracle(order):
    lat = oracle.read_lattice(order)
    shape = (11, 13, 17)
    n, T, u = gen.smooth_random_fields(shape, seed=21, vmax=0.6, sigma_lnT=0.2)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0])
    o.init(n, T, u)
    with RLB(shape, order=order) as g:
        g.init(n, T, u)
        f = g.populations()
        m = g.moments()
    err = pop_err(lat, f, o.f, n.max())
    print("init order %d: max population error %.2e" % (order, err))
    assert err < 1e-12
    # at t = 0 the reported fields are the initial fields
    assert np.allclose(m["n"], n, rtol=1e-12, atol=0)
    assert np.allclose(m["eps"], 3 * n * T, rtol=1e-12, atol=0)


@pytest.mark.parametrize("order", [3, 2])
def test_f32_init_matches_oracle_to_float_rounding(order):
    """Float storage: the equilibrium's coefficients in double, the per-population Horner steps in
    float; every stored population within a few float units of the oracle's (1e-6 of the scale)."""
    lat = oracle.read_lattice(order)
    shape = (11, 13, 17)
    n, T, u = gen.smooth_random_fields(shape, seed=21, vmax=0.6, sigma_lnT=0.2)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0])
    o.init(n, T, u)
    with RLB(shape, order=order, storage="f32") as g:
        g.init(n, T, u)
        f = g.populations()
    err = pop_err(lat, f, o.f, n.max())
    print("f32 init order %d: max population error %.2e" % (order, err))
    assert err < 1e-6


@pytest.mark.parametrize("order", [3, 2])
@pytest.mark.parametrize("bc", ["periodic", "copyout_z", "copyout_xy", "walls_xz", "box"])
def test_f64_steps_match_oracle(order, bc):
    """17 x 13 x 11 cells: 19 blocks of 128 threads with a ragged last block; interior warps take
    the constant-offset pull, boundary warps the wrapped / clamped one."""
    lat = oracle.read_lattice(order)
    shape = (11, 13, 17)
    f0 = near_equilibrium(lat, shape, seed=3 + order, bc=BCS[bc])
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], bc=BCS[bc], eta_over_s=0.1)
    o.set_populations(f0)
    o.step(8)
    with RLB(shape, order=order, bc=BCS[bc], eta_over_s=0.1) as g:
        g.set_populations(f0)
        g.step(8)
        f = g.populations()
        m = g.moments()
    assert pop_err(lat, f, o.f, 2.0) < 1e-12
    ref = o.moments()
    en, ee, eu = field_err(ref, m)
    assert max(en, ee, eu) < 1e-12
    assert np.allclose(m["totals"], ref[3], rtol=1e-13, atol=1e-13 * np.abs(ref[3]).max())


@pytest.mark.parametrize("order", [3, 2])
def test_f64_interior_warps_match_oracle(order):
    """80 x 16 x 14 cells: rows of 80 contain whole warps (x in [32, 64)) whose stencils stay
    inside the lattice, so the constant-offset pull runs for many steps next to the wrapped one."""
    lat = oracle.read_lattice(order)
    shape = (14, 16, 80)
    n, T, u = gen.smooth_random_fields(shape, seed=44, vmax=0.4, sigma_lnT=0.15, kmax=2)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], eta_over_s=0.1)
    o.init(n, T, u)
    o.step(6)
    with RLB(shape, order=order, eta_over_s=0.1) as g:
        g.init(n, T, u)
        g.step(6)
        f = g.populations()
    assert o.nonconv == 0
    assert pop_err(lat, f, o.f, n.max()) < 1e-12


@pytest.mark.parametrize("order", [3, 2])
@pytest.mark.parametrize("variant", [-1, 3])
@pytest.mark.parametrize("bc", ["periodic", "copyout_xy", "walls_xz"])
def test_interior_and_shell_kernels_match_oracle(order, variant, bc):
    """72 x 20 x 24 cells.  The row kernel takes the rows with interior y and z in x segments
    [0, 32) (x wraps), [32, 64) (constant offsets) and [64, 72) (partial warp, x wraps); the
    shell-row kernel takes the z-boundary planes and y-boundary rows, with per-population y and z
    shifts for the whole warp (wrapped, or x and y clamped for copy-out, or reversed populations at
    bounce-back walls).  Double storage per population; float storage (variant 3) on the fields."""
    lat = oracle.read_lattice(order)
    shape = (24, 20, 72)
    n, T, u = gen.smooth_random_fields(shape, seed=51, vmax=0.45, sigma_lnT=0.15, kmax=2)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], bc=BCS[bc], eta_over_s=0.1)
    o.init(n, T, u)
    o.step(6)
    storage = "f64" if variant < 0 else "f32"
    with RLB(shape, order=order, bc=BCS[bc], eta_over_s=0.1, storage=storage, step_variant=variant) as g:
        g.init(n, T, u)
        g.step(6)
        f = g.populations()
        m = g.moments()
    assert o.nonconv == 0
    if storage == "f64":
        assert pop_err(lat, f, o.f, n.max()) < 1e-12
    else:
        assert max(field_err(o.moments(), m)) < 1e-5


@pytest.mark.parametrize("order", [3, 2])
def test_small_periodic_dimensions(order):
    """Axes shorter than the stencil reach (|v| up to 6 > n): the general modulo path."""
    lat = oracle.read_lattice(order)
    shape = (5, 4, 3)
    f0 = near_equilibrium(lat, shape, seed=8)
    o = oracle.OracleRLB(lat, 3, 4, 5, tau_prime=0.9)
    o.set_populations(f0)
    o.step(6)
    with RLB(shape, order=order, tau_prime=0.9) as g:
        g.set_populations(f0)
        g.step(6)
        assert pop_err(lat, g.populations(), o.f, 2.0) < 1e-12


@pytest.mark.parametrize("order", [3, 2])
def test_riemann_tube_full_run(order):
    """Shock tube 1x1x800, copy-out ends, T = 1 | 0.5, n = T^3, eta/s = 0.1, 500 steps (Sec. III):
    every population after the full run within 1e-12 of the oracle."""
    lat = oracle.read_lattice(order)
    n, T, u = gen.riemann_tube(800)
    o = oracle.OracleRLB(lat, 1, 1, 800, bc=(0, 0, 1), eta_over_s=0.1)
    o.init(n, T, u)
    o.step(500)
    with RLB((800, 1, 1), order=order, bc=(0, 0, 1), eta_over_s=0.1) as g:
        g.init(n, T, u)
        g.step(500)
        f = g.populations()
        m = g.moments()
    assert pop_err(lat, f, o.f, 1.0) < 1e-12
    en, ee, eu = field_err(o.moments(), m)
    assert max(en, ee, eu) < 1e-12


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("order", [3, 2])
def test_f32_fields_within_1e5(order, variant):
    """Float storage and arithmetic: Landau fields within 1e-5 of the FP64 oracle after 40 steps of
    the random-field case (|v| <= 0.6, sigma_lnT = 0.2, eta/s = 0.1), for every step-kernel variant
    (2 or 3 resident blocks, scalar or paired arithmetic)."""
    lat = oracle.read_lattice(order)
    shape = (11, 13, 17)
    n, T, u = gen.smooth_random_fields(shape, seed=31, vmax=0.6, sigma_lnT=0.2)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], eta_over_s=0.1)
    o.init(n, T, u)
    o.step(40)
    with RLB(shape, order=order, storage="f32", eta_over_s=0.1, step_variant=variant) as g:
        g.init(n, T, u)
        g.step(40)
        m = g.moments()
    en, ee, eu = field_err(o.moments(), m)
    print("f32 order %d variant %d: n %.2e eps %.2e u %.2e" % (order, variant, en, ee, eu))
    assert max(en, ee, eu) < 1e-5


def test_f16dev_fields_error_is_bounded():
    lat = oracle.read_lattice(3)
    shape = (11, 13, 17)
    n, T, u = gen.smooth_random_fields(shape, seed=31, vmax=0.3, sigma_lnT=0.1)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], eta_over_s=0.1)
    o.init(n, T, u)
    o.step(20)
    with RLB(shape, order=3, storage="f16dev", eta_over_s=0.1) as g:
        g.init(n, T, u)
        g.step(20)
        m = g.moments()
    en, ee, eu = field_err(o.moments(), m)
    print("f16dev: n %.2e eps %.2e u %.2e" % (en, ee, eu))
    assert max(en, ee, eu) < 1e-2


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_conservation_on_gpu(storage, tol):
    """Periodic lattice: sum N^0 and sum T^{0 nu} stay constant (Eqs. (eq:conser1), (eq:conser2))."""
    shape = (24, 20, 28)
    n, T, u = gen.smooth_random_fields(shape, seed=5, vmax=0.5, sigma_lnT=0.2)
    with RLB(shape, order=3, storage=storage, eta_over_s=0.1) as g:
        g.init(n, T, u)
        t0 = g.moments()["totals"]
        g.step(60)
        t1 = g.moments()["totals"]
    assert np.max(np.abs(t1 - t0)) <= tol * np.abs(t0).max()


def test_autotune_keeps_the_state_and_picks_a_variant():
    shape = (20, 24, 64)
    n, T, u = gen.smooth_random_fields(shape, seed=3, vmax=0.4)
    with RLB(shape, storage="f32") as a, RLB(shape, storage="f32") as b:
        a.init(n, T, u)
        b.init(n, T, u)
        v, ms = a.autotune(reps=2)
        # register variants 0..3 and the pipelined shapes that fit this lattice
        assert 0 <= v < len(ms) and len(ms) >= 5 and ms[v] > 0 and all(t > 0 for t in ms[:5])
        assert np.array_equal(a.populations(), b.populations())  # autotuning changed nothing
        a.step(1)
        with pytest.raises(RLBError) as e:
            a.autotune()
        assert e.value.status == rlbmod.RLB_ESTATE


def test_checkpoint_resume_is_bitwise():
    shape = (8, 9, 10)
    n, T, u = gen.smooth_random_fields(shape, seed=9, vmax=0.4)
    with RLB(shape, storage="f32") as a, RLB(shape, storage="f32") as b:
        a.init(n, T, u)
        a.step(5)
        b.set_populations(a.populations())
        a.step(7)
        b.step(7)
        assert np.array_equal(a.populations(), b.populations())


def test_device_and_host_inputs_agree():
    shape = (6, 7, 9)
    n, T, u = gen.smooth_random_fields(shape, seed=4, vmax=0.4)
    with RLB(shape) as a, RLB(shape) as b:
        a.init(n, T, u)
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        b.init(dev(n), dev(T), dev(u))
        assert np.array_equal(a.populations(), b.populations())
        out = dict(n=torch.empty(shape, dtype=torch.float64, device="cuda"),
                   eps=torch.empty(shape, dtype=torch.float64, device="cuda"),
                   U=torch.empty((4,) + shape, dtype=torch.float64, device="cuda"))
        b.moments(out=out)
        assert np.array_equal(out["n"].cpu().numpy(), a.moments()["n"])


def test_landau_failure_is_reported_not_hidden():
    """A cell whose tensor has no timelike eigenvector raises RLB_ENONCONV at the next
    synchronising call; the other cells are unaffected."""
    lat = oracle.read_lattice(3)
    shape = (4, 5, 6)
    f0 = near_equilibrium(lat, shape, seed=2)
    bad = f0.copy()
    bad[:, 2, 3, 4] = 0.0
    bad[0, 2, 3, 4] = 1.0  # a single population: N null-like, no Landau frame
    with RLB(shape, tau_prime=1.0) as g:
        g.set_populations(bad)
        with pytest.raises(RLBError) as e:
            g.moments()
        assert e.value.status == rlbmod.RLB_ENONCONV
        assert "1 cell" in str(e.value)
    # every cell holding one population: after the pull each cell holds one population again,
    # so every collision of the step fails and the step reports it
    single = np.zeros_like(f0)
    single[0] = 1.0
    with RLB(shape, tau_prime=1.0) as g:
        g.set_populations(single)
        g.step(1)
        with pytest.raises(RLBError) as e:
            g.sync()
        assert e.value.status == rlbmod.RLB_ENONCONV
        assert np.array_equal(g.populations()[0], single[0])  # streamed, not collided


@pytest.mark.parametrize("storage,tol,variant,bc", [("f64", 1e-12, -1, "periodic")] +
                         [("f32", 2e-5, v, "periodic") for v in range(4)] +
                         [("f16dev", 2e-2, v, "periodic") for v in (0, 3)] +
                         [("f64", 1e-12, -1, "box"), ("f32", 2e-5, 3, "box")] +
                         [("f32", 2e-5, v, "periodic") for v in (4, 5, 6, 7)] +
                         [("f64", 1e-12, 11, "periodic"), ("f16dev", 2e-2, 4, "periodic"), ("f32", 2e-5, 4, "box")])
def test_full_size_sampled_cells(storage, tol, variant, bc):
    """256^3 random-field case in the benchmark's launch configuration: one step from the seeded
    equilibrium, 96 cells (corners, faces, interior, random) against the oracle cell by cell; also
    with bounce-back walls on every face."""
    lat = oracle.read_lattice(3)
    N = 256
    shape = (N, N, N)
    n, T, u = gen.smooth_random_fields(shape, seed=1, vmax=0.6, sigma_lnT=0.2)
    rng = np.random.default_rng(0)
    pts = [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N // 2, 5), (N - 1, 3, N - 2), (7, 7, 7), (N // 2, N // 2, N // 2)]
    flat = [x + N * (y + N * z) for z, y, x in pts] + list(rng.integers(0, N ** 3, size=90))
    sample = np.array(flat, dtype=np.int64)
    o = oracle.OracleRLB(lat, N, N, N, bc=BCS[bc], eta_over_s=0.1)
    ref = o.init_step_cells(n, T, u, sample)
    with RLB(shape, order=3, bc=BCS[bc], storage=storage, eta_over_s=0.1, step_variant=variant) as g:
        assert variant < 0 or g.variant == variant
        g.init(n, T, u)
        g.step(1)
        dev = torch.empty((lat.q, N ** 3), dtype=torch.float64, device="cuda")
        g.populations(out=dev)
        got = dev[:, torch.from_numpy(sample).cuda()].T.cpu().numpy()
        del dev
    scale = np.maximum(np.abs(ref), lat.w[None, :] * n.max() / 2)
    err = float(np.max(np.abs(got - ref) / scale))
    print("full-size %s variant %d %s sampled error %.2e" % (storage, variant, bc, err))
    assert err < tol


def test_non_finite_populations_are_reported_as_enan():
    """A NaN population makes the cell's moments non-finite: rlb_moments reports RLB_ENAN (not a
    Landau failure), and the context stays usable."""
    lat = oracle.read_lattice(3)
    shape = (4, 5, 6)
    f0 = near_equilibrium(lat, shape, seed=2)
    bad = f0.copy()
    bad[7, 1, 2, 3] = np.nan
    with RLB(shape, tau_prime=1.0) as g:
        g.set_populations(bad)
        with pytest.raises(RLBError) as e:
            g.moments()
        assert e.value.status == rlbmod.RLB_ENAN
        assert "1 cells with non-finite" in str(e.value)
        g.set_populations(f0)
        g.step(2)
        g.moments()  # clean again


@pytest.mark.parametrize("order", [3, 2])
@pytest.mark.parametrize("T_ref", [1.0, 2.5])
def test_reference_temperature_relaxation_time_matches_oracle(order, T_ref):
    """tau_local_T = 0: tau' from the reference temperature T_ref (Sec. III) instead of each
    cell's Landau temperature, on the shock tube whose local T differs from T_ref; double storage
    per population at 1e-12 against the oracle after 30 steps."""
    lat = oracle.read_lattice(order)
    n, T, u = gen.riemann_tube(96)
    o = oracle.OracleRLB(lat, 1, 1, 96, bc=(0, 0, 1), eta_over_s=0.1, tau_local_T=0, T_ref=T_ref)
    o.init(n, T, u)
    o.step(30)
    with RLB((96, 1, 1), order=order, bc=(0, 0, 1), eta_over_s=0.1, tau_local_T=False, T_ref=T_ref) as g:
        g.init(n, T, u)
        g.step(30)
        f = g.populations()
    assert pop_err(lat, f, o.f, 1.0) < 1e-12


def test_context_larger_than_the_device_is_enomem():
    """rlb_create maps a refused cudaMalloc to RLB_ENOMEM (nothing is launched): 1200^3 float cells
    need 1.8 TB of populations."""
    with pytest.raises(RLBError) as e:
        RLB((1200, 1200, 1200), order=3, storage="f32")
    assert e.value.status == rlbmod.RLB_ENOMEM
    with RLB((4, 4, 8), order=3, storage="f32") as g:  # the device is still usable
        n, T, u = gen.smooth_random_fields((4, 4, 8), seed=1, vmax=0.2, sigma_lnT=0.1)
        g.init(n, T, u)
        g.step(1)
        g.sync()
