"""Host field transfers of rlb_init / rlb_moments: page-locked host arrays are read and written in
place by the kernels (over the CPU-GPU link), pageable ones go through device staging copies, device
tensors stay on the device; all three give the same populations and fields bitwise."""
import numpy as np
import pytest

from paper_inputs import fields as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1301_3423_gb300 import RLB  # noqa: E402


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16dev"])
def test_pinned_pageable_and_device_fields_agree(storage):
    shape = (9, 20, 64)
    n, T, u = gen.smooth_random_fields(shape, seed=71, vmax=0.5, sigma_lnT=0.2)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pops, fields = {}, {}
    # (n, T, u) as pageable, page-locked, mixed (one pageable array: staged) and device inputs
    for how, args in [("pageable", (n, T, u)), ("pinned", (pinned(n), pinned(T), pinned(u))),
                      ("mixed", (pinned(n), T, pinned(u))), ("device", (dev(n), dev(T), dev(u)))]:
        with RLB(shape, order=3, storage=storage, eta_over_s=0.1) as g:
            g.init(*args)
            pops[how] = g.populations()
            g.step(4)
            g.sync()
            outs = {"pageable": None,
                    "pinned": dict(n=pinned(np.zeros(shape)), eps=pinned(np.zeros(shape)),
                                   U=pinned(np.zeros((4,) + shape))),
                    "mixed": dict(n=pinned(np.zeros(shape)), eps=np.zeros(shape), U=pinned(np.zeros((4,) + shape))),
                    "device": dict(n=torch.zeros(shape, dtype=torch.float64, device="cuda"),
                                   eps=torch.zeros(shape, dtype=torch.float64, device="cuda"),
                                   U=torch.zeros((4,) + shape, dtype=torch.float64, device="cuda"))}[how]
            m = g.moments(out=outs)
            fields[how] = {k: (v.cpu().numpy() if torch.is_tensor(v) else np.array(v)) for k, v in m.items()}
    for how in ("pinned", "mixed", "device"):
        assert np.array_equal(pops[how], pops["pageable"]), how
        for k in ("n", "eps", "U", "totals"):
            assert np.array_equal(fields[how][k], fields["pageable"][k]), (how, k)


def test_views_into_a_pinned_allocation():
    """Arrays that start inside a larger page-locked allocation (the device address follows the
    host offset)."""
    shape = (5, 8, 32)
    cells = 5 * 8 * 32
    n, T, u = gen.smooth_random_fields(shape, seed=72, vmax=0.4, sigma_lnT=0.1)
    big = torch.zeros(5 * cells + 1000, dtype=torch.float64).pin_memory().numpy()
    off = 123
    hn = big[off:off + cells].reshape(shape)
    hT = big[off + cells:off + 2 * cells].reshape(shape)
    hu = big[off + 2 * cells:off + 5 * cells].reshape((3,) + shape)
    hn[...] = n
    hT[...] = T
    hu[...] = u
    out = torch.zeros(6 * cells + 77, dtype=torch.float64).pin_memory().numpy()
    o = dict(n=out[7:7 + cells].reshape(shape), eps=out[7 + cells:7 + 2 * cells].reshape(shape),
             U=out[7 + 2 * cells:7 + 6 * cells].reshape((4,) + shape))
    with RLB(shape, order=3, storage="f32", eta_over_s=0.1) as g:
        g.init(hn, hT, hu)
        f_view = g.populations()
        g.step(3)
        m_view = g.moments(out=o)
        m_view = {k: np.array(v) for k, v in m_view.items()}
    with RLB(shape, order=3, storage="f32", eta_over_s=0.1) as g:
        g.init(n, T, u)
        f_ref = g.populations()
        g.step(3)
        m_ref = g.moments()
    assert np.array_equal(f_view, f_ref)
    for k in ("n", "eps", "U", "totals"):
        assert np.array_equal(m_view[k], m_ref[k]), k
