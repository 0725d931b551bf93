"""Serving: continuous batching under an HBM budget; every result equals its solo run; a float
simulation that breaks down is rerun in double storage."""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1301_3423_gb300 import RLB  # noqa: E402
from paper_1301_3423_gb300 import serve  # noqa: E402


def solo(req, landau_fp64):
    """The request run alone with the kernels the server's batches use (the register step kernel,
    variant 0, which the batched kernel reproduces bitwise)."""
    with RLB(req.shape, order=3, bc=req.bc, eta_over_s=req.eta_over_s, storage=req.storage,
             landau_fp64=landau_fp64, step_variant=0) as c:
        c.init(*serve.initial_fields(req))
        c.step(req.steps)
        return c.moments()


@pytest.mark.parametrize("landau_fp64", [False, True])
def test_served_results_equal_solo_runs_and_admission_respects_the_budget(landau_fp64):
    reqs = serve.poisson_requests(12, rate=200.0, seed=3, sizes=(16, 24, 32), step_scale=0.02, f16_fraction=0.3)
    # a budget below the total forces waiting and re-admission
    sizes = [serve.Server.bytes_of(r) for r in reqs]
    budget = max(sizes) + 0.3 * (sum(sizes) - max(sizes))
    srv = serve.Server(hbm_budget=budget, chunk=7, landau_fp64=landau_fp64)
    try:
        st = srv.run(reqs, realtime=False)
    finally:
        srv.close()
    assert st["requests"] == len(reqs)
    assert srv.peak_in_use <= budget
    assert srv.peak_active < len(reqs)  # not everything fitted at once
    by_id = {r.rid: r for r in srv.results}
    for req in reqs:
        ref = solo(req, landau_fp64)
        got = by_id[req.rid]
        assert got.steps == req.steps
        for key in ("n", "eps", "U", "totals"):
            assert np.array_equal(getattr(got, key), ref[key]), (req, key)


def test_realtime_stream_reports_latency_percentiles():
    reqs = serve.poisson_requests(10, rate=50.0, seed=9, sizes=(16, 32), step_scale=0.02)
    srv = serve.Server(hbm_budget=20e9, chunk=10)
    try:
        st = srv.run(reqs, realtime=True, max_wall=120)
    finally:
        srv.close()
    assert st["requests"] == 10
    assert 0 < st["p50_tts_s"] <= st["p99_tts_s"]
    assert st["aggregate_mlups"] > 0


def test_breakdown_in_float_is_rerun_in_double():
    """Request 16 of the benchmark's serving stream, a 964-cell shock tube at eta/s = 0.01 in float
    storage, loses Landau frames.  With escalation the server reruns it in double storage; the
    double run loses them too (from step 490 the FP64 oracle finds cells without a Landau frame: the
    model breaks down, not the precision), so the result is a failure that says it was rerun."""
    req = dataclasses.replace(serve.poisson_requests(40, rate=20.0, seed=5, f16_fraction=0.3)[16], arrival=0.0)
    assert (req.kind, req.shape, req.eta_over_s, req.storage) == ("tube", (964, 1, 1), 0.01, "f32")
    lat = oracle.read_lattice(3)
    o = oracle.OracleRLB(lat, req.shape[2], req.shape[1], req.shape[0], bc=req.bc, eta_over_s=req.eta_over_s)
    o.init(*serve.initial_fields(req))
    o.step(req.steps)
    assert o.nonconv > 0  # the FP64 oracle's own step loses Landau frames
    srv = serve.Server(hbm_budget=20e9, chunk=25, escalate=True)
    try:
        st = srv.run([req], realtime=False)
    finally:
        srv.close()
    r = srv.results[0]
    assert st["escalated_to_f64"] == 1
    assert r.status == "failed" and r.storage == "f64"
    assert "rerun in f64 after the f32 run broke down" in r.detail and "RLB_ENONCONV" in r.detail
