"""GPU parity of the pipelined step kernel (step variants 4 and up: bulk copies of each tile's
pulled population rows into shared memory, consumer warps relaxing the cells from there) against
the FP64 oracle.  Same tolerances as test_gpu_parity: double storage per population at 1e-12 of
max(|f|, w_i n_max / 2); float storage on the Landau fields at 1e-5."""
import numpy as np
import pytest

import oracle
from paper_inputs import fields as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1301_3423_gb300 import RLB  # noqa: E402
from paper_1301_3423_gb300 import rlb as rlbmod  # noqa: E402

from test_gpu_parity import BCS, field_err, near_equilibrium, pop_err  # noqa: E402

PIPE = list(range(4, len(rlbmod.VARIANT_NAMES)))


@pytest.mark.parametrize("order", [3, 2])
@pytest.mark.parametrize("bc", ["periodic", "copyout_z", "copyout_xy", "walls_xz", "box"])
@pytest.mark.parametrize("variant", [11, 7, 10, 15])
def test_f64_pipe_matches_oracle(order, bc, variant):
    """Double storage, 72 x 13 x 11 cells, with 64-cell tiles and 2 consumer warps (the shape whose
    stages fit double rows of both orders), 64-cell tiles with 4 consumer warps and 128-cell tiles
    (second order only): a ragged last tile per row; periodic x split into copies at the lattice ends, copy-out and
    bounce-back x patched by the consumers, y and z resolved per row by the producer (walls
    patched)."""
    lat = oracle.read_lattice(order)
    shape = (11, 13, 72)
    f0 = near_equilibrium(lat, shape, seed=13 + order, bc=BCS[bc])
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], bc=BCS[bc], eta_over_s=0.1)
    o.set_populations(f0)
    o.step(6)
    with RLB(shape, order=order, bc=BCS[bc], eta_over_s=0.1, step_variant=variant) as g:
        if g.variant != variant:
            pytest.skip("variant %d has no stage layout for double rows of order %d" % (variant, order))
        g.set_populations(f0)
        launches0 = g.kernel_launches
        g.step(6)
        steps_launches = g.kernel_launches - launches0
        f = g.populations()
        m = g.moments()
    err = pop_err(lat, f, o.f, 2.0)
    print("pipe f64 order %d %s variant %d: %.2e" % (order, bc, variant, err))
    assert steps_launches == 6  # one launch per step: the pipelined kernel ran
    assert err < 1e-12
    en, ee, eu = field_err(o.moments(), m)
    assert max(en, ee, eu) < 1e-12


@pytest.mark.parametrize("order", [3, 2])
@pytest.mark.parametrize("shape", [(5, 4, 8), (7, 3, 16), (9, 8, 36)])
def test_f64_pipe_small_and_ragged_lattices(order, shape):
    """Axes shorter than the stencil reach (modulo wrap of y and z in the producer, x split into
    several periods), rows narrower than a tile, a row of 36 cells (a 4-cell second tile)."""
    lat = oracle.read_lattice(order)
    f0 = near_equilibrium(lat, shape, seed=8)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], tau_prime=0.9)
    o.set_populations(f0)
    o.step(5)
    for variant in (11,):
        with RLB(shape, order=order, tau_prime=0.9, step_variant=variant) as g:
            assert g.variant == variant
            g.set_populations(f0)
            l0 = g.kernel_launches
            g.step(5)
            assert g.kernel_launches - l0 == 5
            assert pop_err(lat, g.populations(), o.f, 2.0) < 1e-12, variant


@pytest.mark.parametrize("order", [3, 2])
@pytest.mark.parametrize("variant", PIPE)
def test_f32_pipe_fields_within_1e5(order, variant):
    """Float storage on every pipelined shape: Landau fields within 1e-5 of the FP64 oracle after
    40 steps of the random-field case (|v| <= 0.6, sigma_lnT = 0.2, eta/s = 0.1)."""
    lat = oracle.read_lattice(order)
    shape = (11, 13, 40)
    n, T, u = gen.smooth_random_fields(shape, seed=31, vmax=0.6, sigma_lnT=0.2)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], eta_over_s=0.1)
    o.init(n, T, u)
    o.step(40)
    with RLB(shape, order=order, storage="f32", eta_over_s=0.1, step_variant=variant) as g:
        if g.variant != variant:
            pytest.skip("variant %d has no stage layout for float rows of order %d" % (variant, order))
        g.init(n, T, u)
        l0 = g.kernel_launches
        g.step(40)
        assert g.kernel_launches - l0 == 40
        m = g.moments()
    en, ee, eu = field_err(o.moments(), m)
    print("pipe f32 order %d variant %d: n %.2e eps %.2e u %.2e" % (order, variant, en, ee, eu))
    assert max(en, ee, eu) < 1e-5


@pytest.mark.parametrize("bc", ["copyout_xy", "walls_xz", "box"])
def test_f32_pipe_boundaries_equal_register_kernel(bc):
    """Float storage with patched boundaries: the pipelined kernel (variant 4) and the register
    kernel with the same paired arithmetic (variant 3) evaluate the same operations on the same
    pulled values, so their populations agree to float rounding after 10 steps."""
    shape = (12, 10, 40)
    n, T, u = gen.smooth_random_fields(shape, seed=17, vmax=0.5, sigma_lnT=0.2)
    out = {}
    for v in (3, 4):
        with RLB(shape, order=3, bc=BCS[bc], storage="f32", eta_over_s=0.1, step_variant=v) as g:
            assert g.variant == v
            g.init(n, T, u)
            g.step(10)
            out[v] = g.populations()
    lat = oracle.read_lattice(3)
    assert pop_err(lat, out[4], out[3], n.max()) < 1e-5


def test_f16dev_pipe_matches_register_kernel():
    """Half-deviation storage: the pipelined kernel against the register kernel after 20 steps."""
    shape = (11, 13, 40)
    n, T, u = gen.smooth_random_fields(shape, seed=31, vmax=0.3, sigma_lnT=0.1)
    lat = oracle.read_lattice(3)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], eta_over_s=0.1)
    o.init(n, T, u)
    o.step(20)
    ref = o.moments()
    for v in (3, 4, 7):
        with RLB(shape, order=3, storage="f16dev", eta_over_s=0.1, step_variant=v) as g:
            assert g.variant == v
            g.init(n, T, u)
            g.step(20)
            m = g.moments()
        en, ee, eu = field_err(ref, m)
        print("f16dev variant %d: n %.2e eps %.2e u %.2e" % (v, en, ee, eu))
        assert max(en, ee, eu) < 1e-2


def test_conservation_pipe():
    """Periodic lattice, pipelined float step: sum N^0, sum T^{0 nu} constant to float rounding."""
    shape = (24, 20, 32)
    n, T, u = gen.smooth_random_fields(shape, seed=5, vmax=0.5, sigma_lnT=0.2)
    with RLB(shape, order=3, storage="f32", eta_over_s=0.1, step_variant=4) as g:
        assert g.variant == 4
        g.init(n, T, u)
        t0 = g.moments()["totals"]
        g.step(60)
        t1 = g.moments()["totals"]
    assert np.max(np.abs(t1 - t0)) <= 2e-6 * np.abs(t0).max()


@pytest.mark.parametrize("storage,variant", [("f64", 11), ("f32", 4), ("f32", 6), ("f32", 12), ("f32", 15),
                                             ("f32", 16)])
def test_landau_failure_in_pipe_is_reported(storage, variant):
    """Every cell holding a single population: the pipelined step streams without collision and
    reports RLB_ENONCONV once per cell (float arithmetic: the two warps of a cell stream their own
    halves, one of them counts)."""
    lat = oracle.read_lattice(3)
    shape = (4, 5, 8)
    single = np.zeros((lat.q,) + shape)
    single[0] = 1.0
    with RLB(shape, tau_prime=1.0, storage=storage, step_variant=variant) as g:
        assert g.variant == variant
        g.set_populations(single)
        g.step(1)
        with pytest.raises(rlbmod.RLBError) as e:
            g.sync()
        assert e.value.status == rlbmod.RLB_ENONCONV
        assert "%d cell updates" % (4 * 5 * 8) in str(e.value)
        assert np.array_equal(g.populations(), single)


@pytest.mark.parametrize("storage,pipe,reg,tol", [("f64", 11, 0, 1e-12), ("f32", 4, 3, 1e-5), ("f32", 5, 3, 1e-5),
                                                  ("f32", 6, 3, 1e-5), ("f16dev", 8, 3, 5e-3), ("f32", 12, 3, 1e-5),
                                                  ("f16dev", 13, 3, 5e-3), ("f32", 15, 3, 1e-5), ("f32", 16, 3, 1e-5),
                                                  ("f32", 17, 3, 1e-5), ("f16dev", 16, 3, 5e-3)])
def test_pipe_equals_register_kernel_with_many_tiles_per_block(storage, pipe, reg, tol):
    """128 x 64 x 64 cells, 6 steps: every block runs dozens of tiles through its stage ring, so
    every stage is reused many times (the register kernels are checked against the oracle in
    test_gpu_parity).  Double storage per population at 1e-12, float at 1e-5; half deviations
    within a few half-precision units (the two kernels may round a float result differently
    before the half store)."""
    shape = (64, 64, 128)
    n, T, u = gen.smooth_random_fields(shape, seed=23, vmax=0.5, sigma_lnT=0.2)
    out = {}
    for v in (pipe, reg):
        with RLB(shape, order=3, storage=storage, eta_over_s=0.1, step_variant=v) as g:
            assert g.variant == v
            g.init(n, T, u)
            g.step(6)
            g.sync()
            out[v] = g.populations()
    lat = oracle.read_lattice(3)
    err = pop_err(lat, out[pipe], out[reg], n.max())
    print("%s pipe %d vs register %d: %.2e" % (storage, pipe, reg, err))
    assert err < tol


@pytest.mark.parametrize("variant", [5, 12, 15])
def test_expired_waits_are_reported_and_the_context_stays_usable(variant):
    """Testing flag: the pipelined step's producers withhold every tile, so each consumer's bounded
    wait (2 s) runs out; the kernel returns, the next synchronising call reports RLB_ETIMEOUT, and
    the context keeps working (no GPU fault, no hang).  Row segments (5), row tiles (12), three
    consumer groups with one stage each (15)."""
    shape = (8, 8, 128)
    n, T, u = gen.smooth_random_fields(shape, seed=3, vmax=0.3, sigma_lnT=0.1)
    with RLB(shape, order=3, storage="f32", eta_over_s=0.1, step_variant=variant, debug_flags=1) as g:
        assert g.variant == variant
        g.init(n, T, u)
        f0 = g.populations()
        g.step(1)
        with pytest.raises(rlbmod.RLBError) as e:
            g.sync()
        assert e.value.status == rlbmod.RLB_ETIMEOUT
        g.sync()  # the status was reported once and cleared
        # the step's result is not a valid state (nothing was written); the context still works and
        # a state can be restored
        g.populations()
        g.set_populations(f0)
        assert np.array_equal(g.populations(), f0)
        g.moments()


# ---- row tiles (variants 12..14): a tile is 128 / nx whole rows of an x-periodic lattice --------

# (shape (nz, ny, nx), bc): rows of 8 to 128 cells, G = 16 .. 1 rows per tile, row counts that leave
# the last tile short, y and z axes whose wrap splits a tile's source rows into two runs, copy-out
# and bounce-back y / z
ROW_CASES = [((7, 13, 128), (0, 0, 0)), ((5, 11, 64), (0, 0, 0)), ((6, 9, 40), (0, 1, 0)),
             ((9, 7, 32), (0, 0, 1)), ((6, 10, 48), (0, 2, 2)), ((5, 6, 96), (0, 1, 2)), ((4, 5, 8), (0, 0, 0))]


@pytest.mark.parametrize("storage,rows,seg", [("f32", 12, 5), ("f32", 13, 4), ("f32", 16, 15), ("f32", 18, 17),
                                              ("f16dev", 12, 5), ("f16dev", 14, 10), ("f16dev", 16, 15),
                                              ("f32", 19, 16), ("f16dev", 19, 16)])
@pytest.mark.parametrize("case", range(len(ROW_CASES)))
def test_row_tiles_equal_row_segments_bitwise(storage, rows, seg, case):
    """Row tiles pull every cell's populations from the same source cells as row segments of the
    same block layout and evaluate the same arithmetic on them, so after 7 steps the populations
    are bitwise equal (the segment kernel's x wrap is split copies; the row tiles' is a per-lane
    offset into one copy of the whole rows).  96-cell row tiles (19) against 128-cell ones (16)."""
    shape, bc = ROW_CASES[case]
    n, T, u = gen.smooth_random_fields(shape, seed=40 + case, vmax=0.5, sigma_lnT=0.2)
    out = {}
    for v in (rows, seg):
        with RLB(shape, order=3, bc=bc, storage=storage, eta_over_s=0.1, step_variant=v) as g:
            if g.variant != v:
                pytest.skip("variant %d does not exist for %s on %s" % (v, storage, shape))
            g.init(n, T, u)
            l0 = g.kernel_launches
            g.step(7)
            assert g.kernel_launches - l0 == 7
            out[v] = g.populations()
    assert np.array_equal(out[rows], out[seg])


@pytest.mark.parametrize("case", range(len(ROW_CASES)))
def test_row_tiles_f64_match_oracle(case):
    """Second order, double storage (the row-tile shape whose stages fit double rows: 4 consumer
    warps, variant 14): populations within 1e-12 of the FP64 oracle after 6 steps, and the fields."""
    shape, bc = ROW_CASES[case]
    lat = oracle.read_lattice(2)
    f0 = near_equilibrium(lat, shape, seed=50 + case, bc=bc)
    o = oracle.OracleRLB(lat, shape[2], shape[1], shape[0], bc=bc, eta_over_s=0.1)
    o.set_populations(f0)
    o.step(6)
    with RLB(shape, order=2, bc=bc, eta_over_s=0.1, step_variant=14) as g:
        assert g.variant == 14
        g.set_populations(f0)
        l0 = g.kernel_launches
        g.step(6)
        assert g.kernel_launches - l0 == 6
        f = g.populations()
        m = g.moments()
    err = pop_err(lat, f, o.f, 2.0)
    print("rows f64 order 2 %s %s: %.2e" % (shape, bc, err))
    assert err < 1e-12
    assert max(field_err(o.moments(), m)) < 1e-12


def test_row_tiles_many_tiles_per_block_equal_register_kernel():
    """64- and 32-cell rows (two and four rows per tile) on lattices with hundreds of tiles per
    block: float fields of the row tiles against the register kernel with the same float
    arithmetic (variant 3) after 6 steps, at float rounding."""
    lat = oracle.read_lattice(3)
    for shape in ((48, 40, 64), (40, 60, 32)):
        n, T, u = gen.smooth_random_fields(shape, seed=61, vmax=0.5, sigma_lnT=0.2)
        out = {}
        for v in (12, 3):
            with RLB(shape, order=3, storage="f32", eta_over_s=0.1, step_variant=v) as g:
                assert g.variant == v
                g.init(n, T, u)
                g.step(6)
                out[v] = g.populations()
        err = pop_err(lat, out[12], out[3], n.max())
        print("rows %s vs register: %.2e" % (shape, err))
        assert err < 1e-5


def test_row_tiles_default_and_availability():
    """Row tiles exist only for an x-periodic lattice with nx <= 128 on 16-byte boundaries (and at
    least the stencil's x reach); the library picks them by default where their tiles are at least
    3/4 used, and row segments for wider rows."""
    for shape, bc, storage, expect in [((8, 8, 64), (0, 0, 0), "f32", True), ((8, 8, 64), (1, 0, 0), "f32", False),
                                       ((8, 8, 256), (0, 0, 0), "f32", False), ((8, 8, 36), (0, 0, 0), "f32", True),
                                       ((8, 8, 36), (0, 0, 0), "f16dev", False)]:
        with RLB(shape, order=3, bc=bc, storage=storage, step_variant=12) as g:
            assert (g.variant == 12) == expect, (shape, bc, storage, g.variant)
    with RLB((8, 8, 64), order=3, storage="f32") as g:
        assert g.variant == 16  # one warp per cell, row tiles
    with RLB((8, 8, 256), order=3, storage="f32") as g:
        assert g.variant == 15  # one warp per cell, row segments
    with RLB((8, 8, 96), order=3, storage="f32") as g:
        assert g.variant == 19  # 96-cell row tiles
