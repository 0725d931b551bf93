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

DTYPE = {"f64": torch.float64, "f32": torch.float32}


@pytest.mark.parametrize("order,storage", [(3, "f64"), (3, "f32"), (2, "f64"), (2, "f32")])
def test_totals_without_allocation_match_rlb_moments(order, storage):
    shape = (12, 10, 9)
    n, T, u = gen.smooth_random_fields(shape, seed=6, vmax=0.4, sigma_lnT=0.15)
    with RLB(shape, order=order, storage=storage, eta_over_s=0.1) as g:
        g.init(n, T, u)
        ref = g.moments()["totals"]
        q = g.q
        f64 = torch.empty((q, g.cells), dtype=torch.float64, device="cuda")
        g.populations(out=f64)
    # the caller's own buffer, in the storage precision (exact: the stored values are float32 or
    # float64 already)
    f = f64.to(DTYPE[storage]).contiguous()
    torch.cuda.synchronize()
    for _ in range(2):  # two calls in a row share the scratch array
        got = rlbmod.totals_noalloc(f, order, storage, shape)
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_rejects_lattices_beyond_the_scratch_limit():
    f = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(RLBError) as e:
        rlbmod.totals_noalloc(f, 3, "f64", (256, 256, 256))
    assert e.value.status == rlbmod.RLB_EINVAL
    assert "exceed the fixed scratch limit" in str(e.value)
