"""Batched stepping: uneven instances in persistent kernels over shared tile queues, with CUDA-graph step
loops; each member's result equals its solo run."""
import numpy as np
import pytest

from paper_inputs import fields as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1301_3423_gb300 import RLB, Batch, RLBError  # noqa: E402
from paper_1301_3423_gb300 import rlb as rlbmod  # noqa: E402

# (shape, bc, eta/s, steps, field kind)
MEMBERS = [
    ((400, 1, 1), (0, 0, 1), 0.1, 23, "tube"),
    ((32, 32, 32), (0, 0, 0), 0.01, 37, "shear"),
    ((20, 24, 40), (0, 0, 0), 0.5, 11, "random"),
    ((3, 5, 7), (0, 0, 0), 0.1, 29, "random"),
    ((900, 1, 1), (0, 0, 1), 0.5, 41, "tube"),
    ((16, 40, 72), (1, 0, 0), 0.1, 17, "random"),
    ((24, 16, 48), (2, 0, 2), 0.1, 13, "random"),
    ((600, 1, 1), (0, 0, 2), 0.1, 19, "tube"),
    # rows that fill 64- and 128-cell tiles: the batched pipelined kernel's members
    ((6, 5, 128), (0, 0, 0), 0.1, 9, "random"),
    ((5, 4, 192), (1, 0, 0), 0.1, 7, "random"),
    ((4, 6, 128), (2, 0, 2), 0.1, 5, "random"),
    # rows that fill 96-cell row tiles exactly (with a 128-cell row-tile variant they take the
    # 96-cell companion)
    ((6, 5, 96), (0, 0, 0), 0.1, 9, "random"),
    ((5, 6, 48), (0, 2, 2), 0.1, 6, "random"),
]


def fields_for(shape, kind, seed):
    if kind == "tube":
        return gen.riemann_tube(shape[0])
    if kind == "shear":
        return gen.shear_wave(shape[2], amp=0.05, ny=shape[1], nz=shape[0])
    return gen.smooth_random_fields(shape, seed=seed, vmax=0.4, sigma_lnT=0.15, kmax=2)


def make(order, storage, variant, k, stream=None):
    shape, bc, eta, steps, kind = MEMBERS[k]
    ctx = RLB(shape, order=order, bc=bc, eta_over_s=eta, storage=storage, step_variant=variant,
              landau_fp64=(storage != "f64"), stream=stream)
    ctx.init(*fields_for(shape, kind, seed=10 + k))
    return ctx, steps


@pytest.mark.parametrize("order,storage,variant", [(3, "f32", 0), (3, "f32", 3), (3, "f64", -1), (2, "f32", 1),
                                                   (3, "f16dev", 0), (3, "f16dev", 3),
                                                   (3, "f32", 5), (3, "f32", 4), (2, "f32", 5), (3, "f16dev", 4),
                                                   (3, "f64", 11), (3, "f32", 12), (3, "f32", 13), (2, "f32", 12),
                                                   (3, "f16dev", 13), (2, "f64", 14), (3, "f32", 15), (3, "f32", 16),
                                                   (3, "f16dev", 16), (2, "f32", 18), (3, "f32", 19)])
@pytest.mark.parametrize("graph", [True, False])
def test_batched_members_equal_solo_runs(order, storage, variant, graph):
    """Variants 0-3: every member on the register kernels.  Variants 4 to 11: members whose rows
    fill the pipelined tiles (the 128-cell rows here) on the batched pipelined kernel, the others
    (1 x 1 x N tubes, rows of 7 to 192 cells) on the register kernel a context of that storage runs
    alone.  Row-tile variants: the x-periodic members with rows of 32 and 40 cells (and 128 unless
    a float cell takes two warps) on the row-tile kernel, the other 128-cell rows on the
    row-segment kernel of the same layout, the rest on the register kernel.  Each member equals its
    solo run with the variant the batch reports."""
    ctxs = [make(order, storage, variant, k) for k in range(len(MEMBERS))]
    with Batch(order, storage) as b:
        if variant >= 0:
            b.set_variant(variant)
        slots = [b.add(c, s) for c, s in ctxs]
        used = [b.member_variant(s) for s in slots]  # the variant each member runs with in the batch
        if variant >= 4:
            assert any(v == variant for v in used) and any(v != variant for v in used)
        if rlbmod.VARIANT_NAMES[max(variant, 0)].startswith("rows tx128"):
            # a row-segment member beside the row-tile ones
            assert any(v >= 4 and rlbmod.VARIANT_NAMES[v].startswith("pipe") for v in used)
        if variant == 16:
            assert 19 in used  # the 96-cell companion
        solo = []
        for k in range(len(MEMBERS)):
            ctx, steps = make(order, storage, used[k] if variant >= 0 else variant, k)
            if variant >= 0:
                assert ctx.variant == used[k]
            ctx.step(steps)
            solo.append(ctx.populations())
            ctx.close()
        active = len(ctxs)
        while active:
            active = b.run(8, graph=graph)  # members stop at their own step counts
        assert all(b.steps_left(s) == 0 for s in slots)
    for k, (c, steps) in enumerate(ctxs):
        assert c.steps_done == steps
        assert np.array_equal(c.populations(), solo[k]), "member %d differs from its solo run" % k
        c.close()


def test_batch_autotune_changes_nothing_and_members_can_leave():
    ctxs = [make(3, "f32", -1, k) for k in range(len(MEMBERS))]
    before = [c.populations() for c, _ in ctxs]
    with Batch(3, "f32") as b:
        slots = [b.add(c, s) for c, s in ctxs]
        v, ms = b.autotune(reps=2)
        # the register variants and the pipelined shapes that exist for float storage
        assert 0 <= v < len(ms) and ms[v] > 0 and all(t > 0 for t in ms[:6])
        for (c, _), f0 in zip(ctxs, before):
            assert np.array_equal(c.populations(), f0)
        b.run(5)
        b.remove(slots[2])
        with pytest.raises(RLBError):
            b.autotune()
        left = b.run(1000)
        assert left == 0
        assert ctxs[2][0].steps_done == 5
    for c, _ in ctxs:
        c.close()


def test_batch_rejects_mismatched_members():
    ctx = RLB((4, 4, 4), order=3, storage="f64")
    with Batch(3, "f32") as b:
        with pytest.raises(RLBError) as e:
            b.add(ctx, 3)
        assert e.value.status == rlbmod.RLB_EINVAL
    ctx.close()
