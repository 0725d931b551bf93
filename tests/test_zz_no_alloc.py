"""rlb_totals_noalloc: conserved totals for callers that cannot allocate device memory.

Such a caller passes its own population buffer and a host array for the result; the library keeps
its scratch in a fixed device array and allocates nothing.  Its result must equal what the
allocating path (rlb_moments before the first step) reports for the same populations.  This file is
collected last so that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_inputs import fields as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1301_3423_gb300 import RLB, RLBError  # noqa: E402
from paper_1301_3423_gb300 import rlb as rlbmod  # noqa: E402

DTYPE = {"f64": torch.float64, "f32": torch.float32, "f16dev": torch.float16}


def stored_buffer(g, storage, n_ref):
    """The caller's own copy of the context's stored populations, in the storage precision: double
    and float values come back exactly from rlb_get_populations; half deviations are recovered as
    d_i = f_i / w_i - n_ref / 2, which rounds back to the stored half value."""
    f64 = torch.empty((g.q, g.cells), dtype=torch.float64, device="cuda")
    g.populations(out=f64)
    if storage == "f16dev":
        w = torch.from_numpy(rlbmod.quadrature(g.order)["w"]).cuda()[:, None]
        return (f64 / w - n_ref / 2).to(torch.float16).contiguous()
    return f64.to(DTYPE[storage]).contiguous()


@pytest.mark.parametrize("order,storage", [(3, "f64"), (3, "f32"), (3, "f16dev"), (2, "f64"), (2, "f32"),
                                           (2, "f16dev")])
def test_totals_without_allocation_match_rlb_moments(order, storage):
    shape = (12, 10, 9)
    n_ref = 1.3
    n, T, u = gen.smooth_random_fields(shape, seed=6, vmax=0.4, sigma_lnT=0.15)
    with RLB(shape, order=order, storage=storage, eta_over_s=0.1, n_ref=n_ref) as g:
        g.init(n, T, u)
        ref = g.moments()["totals"]
        f = stored_buffer(g, storage, n_ref)
    torch.cuda.synchronize()
    for _ in range(2):  # two calls in a row share the scratch array
        got = rlbmod.totals_noalloc(f, order, storage, shape, n_ref=n_ref)
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_binding_rejects_a_buffer_of_the_wrong_size_or_type():
    """The binding checks the buffer against q * cells elements of the storage type before the
    library reads it."""
    f = torch.zeros(128 * 4 * 4 * 4 - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        rlbmod.totals_noalloc(f, 3, "f64", (4, 4, 4))
    f = torch.zeros(128 * 4 * 4 * 4, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        rlbmod.totals_noalloc(f, 3, "f64", (4, 4, 4))


def test_rejects_lattices_beyond_the_scratch_limit():
    """A correctly sized buffer for 256 x 256 x 129 cells (above the 8,388,608-cell limit): the
    library refuses it with RLB_EINVAL before launching anything."""
    shape = (129, 256, 256)
    f = torch.zeros(128 * 129 * 256 * 256, dtype=torch.float16, device="cuda")
    with pytest.raises(RLBError) as e:
        rlbmod.totals_noalloc(f, 3, "f16dev", shape)
    assert e.value.status == rlbmod.RLB_EINVAL
    assert "exceed the fixed scratch limit" in str(e.value)
    del f
