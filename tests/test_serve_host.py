"""Host-side logic of the continuous-batching server (serve.py) with fake simulations: admission
against the budget, first-come-first-served waiting, rejection of requests above the budget,
failures at creation (RLB_ENOMEM) reported as results, cancellation of waiting and running
requests, large lattices stepped on their own, and numerical breakdowns rerun in double storage.
No GPU is involved."""
import numpy as np
import pytest

from paper_1301_3423_gb300 import serve
from paper_1301_3423_gb300.rlb import RLB_ECUDA, RLB_ENOMEM, RLB_ENONCONV, RLBError


class FakeCtx:
    def __init__(self, req, log):
        self.req, self.log, self.taken, self.kernel_launches, self.closed = req, log, 0, 0, False

    def init(self, n, T, u):
        self.log.append(("init", self.req.rid))

    def step(self, k):
        self.taken += k
        self.kernel_launches += k

    def moments(self):
        z = np.full(self.req.shape, float(self.taken))
        return dict(n=z, eps=z, U=np.stack([z] * 4), totals=np.full(5, float(self.req.rid)))

    def close(self):
        self.closed = True
        self.log.append(("close", self.req.rid))


class FakeBatch:
    def __init__(self):
        self.members, self.kernel_launches = {}, 0

    def add(self, ctx, steps):
        slot = max(self.members, default=-1) + 1
        self.members[slot] = [ctx, steps]
        return slot

    def remove(self, slot):
        del self.members[slot]

    def steps_left(self, slot):
        return self.members[slot][1]

    def run(self, n, graph=True):
        for m in self.members.values():
            k = min(n, m[1])
            m[0].taken += k
            m[1] -= k
        self.kernel_launches += 2 * n

    def close(self):
        pass


def make_server(budget, sizes, fail=(), solo_cells=10 ** 9, chunk=10):
    log = []

    def context(req):
        if req.rid in fail:
            raise RLBError(RLB_ENOMEM, "rlb_create: out of memory")
        return FakeCtx(req, log)

    srv = serve.Server(hbm_budget=budget, chunk=chunk, context=context, batch=lambda storage: FakeBatch(),
                       bytes_of=lambda req: sizes[req.rid], solo_cells=solo_cells)
    return srv, log


def req(rid, steps=25, shape=(4, 4, 4), arrival=0.0, storage="f32"):
    return serve.Request(rid, "random", shape, 0.1, steps, storage, rid, arrival)


def test_admission_waits_for_memory_and_keeps_arrival_order(monkeypatch):
    monkeypatch.setattr(serve, "initial_fields", lambda r: (None, None, None))
    sizes = {0: 60.0, 1: 60.0, 2: 30.0}
    srv, log = make_server(100.0, sizes)
    st = srv.run([req(0), req(1), req(2, steps=5)], realtime=False)
    assert st["completed"] == 3 and st["queued_while_full"] == 1
    assert srv.peak_in_use <= 100.0
    by = {r.rid: r for r in srv.results}
    # request 1 does not fit next to request 0: admitted only once 0 has finished; request 2 is
    # behind it in the queue although it would have fitted (first come, first served)
    assert by[1].admitted >= by[0].finished and by[2].admitted >= by[0].finished
    assert all(r.steps == s for r, s in ((by[0], 25), (by[1], 25), (by[2], 5)))
    assert all(np.all(by[i].n == by[i].steps) for i in by)  # each took exactly its own steps
    assert [e for e in log if e[0] == "close"] == [("close", 0), ("close", 2), ("close", 1)]


def test_request_above_the_budget_is_rejected_not_raised(monkeypatch):
    monkeypatch.setattr(serve, "initial_fields", lambda r: (None, None, None))
    srv, _ = make_server(100.0, {0: 150.0, 1: 10.0})
    st = srv.run([req(0), req(1)], realtime=False)
    assert st["rejected"] == 1 and st["completed"] == 1
    r0 = [r for r in srv.results if r.rid == 0][0]
    assert r0.status == "rejected" and "more than the whole budget" in r0.detail


def test_creation_failure_is_a_failed_result(monkeypatch):
    monkeypatch.setattr(serve, "initial_fields", lambda r: (None, None, None))
    srv, _ = make_server(100.0, {0: 10.0, 1: 10.0}, fail={0})
    st = srv.run([req(0), req(1)], realtime=False)
    assert st["failed"] == 1 and st["completed"] == 1
    r0 = [r for r in srv.results if r.rid == 0][0]
    assert r0.status == "failed" and "RLB_ENOMEM" in r0.detail
    assert srv.in_use == 0.0


def test_cancel_waiting_and_running_requests_frees_their_memory(monkeypatch):
    monkeypatch.setattr(serve, "initial_fields", lambda r: (None, None, None))
    sizes = {0: 60.0, 1: 60.0, 2: 60.0}
    srv, log = make_server(100.0, sizes)
    calls = []

    def on_round(s):
        if not calls:
            calls.append(1)
            assert s.cancel(2)        # waiting: leaves the queue at once
            assert s.cancel(0)        # running: released at the end of the next round
            assert not s.cancel(99)

    st = srv.run([req(0, steps=100), req(1), req(2)], realtime=False, on_round=on_round)
    by = {r.rid: r for r in srv.results}
    assert by[0].status == "cancelled" and by[2].status == "cancelled" and by[1].status == "ok"
    assert st["cancelled"] == 2 and srv.in_use == 0.0
    # request 1 was admitted once request 0's memory was released, before 0 would have finished
    assert by[1].admitted >= by[0].finished
    assert ("close", 0) in log


def test_large_lattices_step_on_their_own(monkeypatch):
    monkeypatch.setattr(serve, "initial_fields", lambda r: (None, None, None))
    srv, _ = make_server(1000.0, {0: 10.0, 1: 10.0}, solo_cells=1000, chunk=7)
    st = srv.run([req(0, steps=30, shape=(10, 10, 10)), req(1, steps=30)], realtime=False)
    assert st["completed"] == 2
    by = {r.rid: r for r in srv.results}
    assert np.all(by[0].n == 30) and np.all(by[1].n == 30)  # both took exactly 30 steps
    assert "f32" in srv.batches and len(srv.batches["f32"].members) == 0


class BreakingCtx(FakeCtx):
    """Request 1 loses Landau frames unless it runs in double storage; request 2 hits a device
    error, which is not a numerical breakdown."""

    def moments(self):
        if self.req.rid == 1 and self.req.storage != "f64":
            raise RLBError(RLB_ENONCONV, "12 cell updates without a Landau frame")
        if self.req.rid == 2:
            raise RLBError(RLB_ECUDA, "device error")
        return super().moments()


@pytest.mark.parametrize("escalate", [True, False])
def test_numerical_breakdown_is_rerun_in_double_storage(monkeypatch, escalate):
    monkeypatch.setattr(serve, "initial_fields", lambda r: (None, None, None))
    log = []
    created = []

    def context(r):
        created.append((r.rid, r.storage))
        return BreakingCtx(r, log)

    srv = serve.Server(hbm_budget=100.0, chunk=10, context=context, batch=lambda storage: FakeBatch(),
                       bytes_of=lambda r: 20.0 if r.storage == "f64" else 10.0, escalate=escalate)
    st = srv.run([req(0), req(1), req(2)], realtime=False)
    r1 = [r for r in srv.results if r.rid == 1][0]
    r2 = [r for r in srv.results if r.rid == 2][0]
    assert r2.status == "failed" and "device error" in r2.detail  # never escalated
    if escalate:
        assert st["completed"] == 2 and st["failed"] == 1 and st["escalated_to_f64"] == 1
        assert r1.status == "ok" and r1.storage == "f64" and r1.steps == 25
        assert "rerun in f64 after the f32 run broke down" in r1.detail
        assert created.count((1, "f32")) == 1 and created.count((1, "f64")) == 1
        assert r1.arrival == 0.0 and r1.finished >= r1.admitted
    else:
        assert st["completed"] == 1 and st["failed"] == 2 and st["escalated_to_f64"] == 0
        assert r1.status == "failed" and "Landau" in r1.detail and r1.storage == "f32"
    assert srv.in_use == 0.0
