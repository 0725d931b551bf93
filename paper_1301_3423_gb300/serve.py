"""Continuous-batching request loop for relativistic lattice Boltzmann simulations.

Requests (shock tubes, shear waves, random-field boxes of different sizes, eta/s and storage
precision) arrive over time.  The server keeps every admitted simulation resident on the device,
admits waiting requests first-come-first-served while their memory fits the HBM budget, and
advances all admitted simulations together in rounds of ``chunk`` steps: small lattices in one
batch per storage precision, stepped by the persistent tile-queue kernel (optionally a replayed
CUDA graph); lattices of at least ``solo_cells`` cells by their own step launches (the pipelined
kernel), which fill the GPU on their own.  A simulation that reaches its step count is finished
(its Landau fields and conserved totals are read back), its memory is released and waiting
requests are admitted in the next round.

Failures are results, not exceptions: a request larger than the whole budget is rejected, one whose
context cannot be created (e.g. RLB_ENOMEM) or whose read-back fails is marked failed, and
cancel(rid) removes a waiting or running request between rounds, releasing its memory.  With
``escalate`` a float or half-storage simulation that breaks down numerically (cells without a
Landau frame, non-finite populations) is run again from its initial state in double storage; its
result says so and keeps the original arrival time, so the rerun counts in its time to solution.

Everything numerical runs in librlb; this module only schedules.
"""
import dataclasses
import time

import numpy as np

from paper_inputs import fields as gen

from .rlb import RLB, RLB_ENAN, RLB_ENONCONV, Batch, RLBError


@dataclasses.dataclass
class Request:
    rid: int
    kind: str            # "tube", "shear" or "random"
    shape: tuple          # (nz, ny, nx)
    eta_over_s: float
    steps: int
    storage: str          # "f32", "f16dev" (or "f64")
    seed: int
    arrival: float        # seconds after the stream starts
    bc: tuple = (0, 0, 0)
    escalated_from: str = ""  # the storage of a run that broke down, when this is its rerun


@dataclasses.dataclass
class Result:
    rid: int
    n: np.ndarray
    eps: np.ndarray
    U: np.ndarray
    totals: np.ndarray
    admitted: float
    finished: float
    arrival: float
    cells: int
    steps: int              # steps taken
    status: str = "ok"      # "ok", "rejected", "failed" or "cancelled"
    detail: str = ""
    storage: str = ""       # the storage precision the result was computed in

    @property
    def tts(self):
        return self.finished - self.arrival


def initial_fields(req):
    """Seeded initial fields of a request (see paper_inputs.fields)."""
    if req.kind == "tube":
        return gen.riemann_tube(req.shape[0])
    if req.kind == "shear":
        nz, ny, nx = req.shape
        return gen.shear_wave(nx, amp=0.05, ny=ny, nz=nz)
    return gen.smooth_random_fields(req.shape, seed=req.seed, vmax=0.4, sigma_lnT=0.15, kmax=2, density="uniform")


def poisson_requests(n, rate=20.0, seed=0, sizes=(32, 48, 64, 96, 128, 192, 256, 384), step_scale=1.0,
                     f16_fraction=0.3, max_side=384):
    """A seeded request stream: exponential inter-arrival times (mean 1/rate); kind uniform over
    tube / shear / random; box side L drawn with probability proportional to 1/L^3; tubes of
    400..4000 cells; eta/s in {0.01, 0.1, 0.5}; steps 500 (tube), 2000 (shear), 1000 (random)
    times step_scale; float storage, or half deviation storage with probability f16_fraction."""
    rng = np.random.default_rng(seed)
    sizes = [L for L in sizes if L <= max_side]
    p = np.array([1.0 / L ** 3 for L in sizes])
    p /= p.sum()
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        kind = str(rng.choice(["tube", "shear", "random"]))
        eta = float(rng.choice([0.01, 0.1, 0.5]))
        storage = "f16dev" if rng.random() < f16_fraction else "f32"
        if kind == "tube":
            N = int(rng.integers(400, 4001))
            shape, bc, steps = (N, 1, 1), (0, 0, 1), 500
        else:
            L = int(rng.choice(sizes, p=p))
            shape, bc, steps = (L, L, L), (0, 0, 0), (2000 if kind == "shear" else 1000)
        out.append(Request(rid, kind, shape, eta, max(1, int(round(steps * step_scale))), storage,
                           int(rng.integers(1 << 30)), t, bc))
    return out


class Server:
    """Admission against an HBM budget plus continuous batching (see the module docstring).

    ``context`` and ``batch`` build the simulations and batches (the library's RLB and Batch by
    default; the host-side tests pass fakes), ``bytes_of`` gives a request's device bytes."""

    def __init__(self, order=3, hbm_budget=150e9, chunk=50, use_graph=True, stream=None, autotune=False,
                 landau_fp64=False, solo_cells=128 ** 3, context=None, batch=None, bytes_of=None, escalate=False):
        """landau_fp64: solve Landau matching in double for every cell (default: in float, in double
        for cells above gamma_thr).  escalate: rerun numerical breakdowns of reduced-precision
        simulations in double storage (see the module docstring)."""
        self.order = order
        self.escalate = bool(escalate)
        self.escalated = 0  # reruns in double storage
        self.landau_fp64 = bool(landau_fp64)
        self.budget = float(hbm_budget)
        self.chunk = int(chunk)
        self.use_graph = use_graph
        self.stream = stream
        self.autotune = autotune
        self.solo_cells = int(solo_cells)
        self._context = context or (lambda req: RLB(req.shape, order=self.order, bc=req.bc,
                                                    eta_over_s=req.eta_over_s, storage=req.storage,
                                                    landau_fp64=self.landau_fp64, stream=self.stream))
        self._batch_factory = batch or (lambda storage: Batch(self.order, storage, stream=self.stream))
        self._bytes_of = bytes_of or (lambda req: self.bytes_of(req, self.order))
        self.batches = {}
        self.active = {}        # key -> (request, context, admitted time, bytes); key (storage, slot) or ("solo", rid)
        self.solo_left = {}     # rid -> steps still to take, for solo simulations
        self.waiting = []
        self.cancelled = set()
        self.in_use = 0.0
        self.peak_in_use = 0.0
        self.peak_active = 0
        self.queued_while_full = 0  # requests that had to wait for memory
        self._waited = set()
        self.results = []
        self.t0 = None
        self.kernel_launches = 0

    def now(self):
        return time.perf_counter() - self.t0 if self.t0 is not None else 0.0

    def _batch(self, storage):
        if storage not in self.batches:
            self.batches[storage] = self._batch_factory(storage)
        return self.batches[storage]

    @staticmethod
    def bytes_of(req, order=3):
        nz, ny, nx = req.shape
        return RLB.bytes_required(order=order, nx=nx, ny=ny, nz=nz, storage=req.storage, bc=req.bc)

    def _finish(self, req, status, detail="", m=None, admitted=None, steps=0):
        nz, ny, nx = req.shape
        empty = np.zeros(0)
        if req.escalated_from:
            detail = ("rerun in f64 after the %s run broke down" % req.escalated_from) + ("; " + detail if detail else "")
        self.results.append(Result(req.rid, m["n"] if m else empty, m["eps"] if m else empty, m["U"] if m else empty,
                                   m["totals"] if m else empty, admitted if admitted is not None else self.now(),
                                   self.now(), req.arrival, nx * ny * nz, steps, status, detail, req.storage))

    def cancel(self, rid):
        """Cancel request rid: a waiting one leaves the queue now, a running one at the end of the
        current round (its memory is released then).  Returns False if rid is unknown or done."""
        for i, req in enumerate(self.waiting):
            if req.rid == rid:
                del self.waiting[i]
                self._finish(req, "cancelled")
                return True
        if any(v[0].rid == rid for v in self.active.values()):
            self.cancelled.add(rid)
            return True
        return False

    def _release(self, key):
        req, ctx, t_adm, need = self.active.pop(key)
        if key[0] != "solo":
            self.batches[key[0]].remove(key[1])
        else:
            self.solo_left.pop(req.rid, None)
        self.kernel_launches += ctx.kernel_launches
        ctx.close()
        self.in_use -= need
        return req, ctx, t_adm

    def _admit(self):
        admitted = 0
        while self.waiting:
            req = self.waiting[0]
            need = self._bytes_of(req)
            if need > self.budget:
                self.waiting.pop(0)
                self._finish(req, "rejected", "needs %.1f GB, more than the whole budget of %.1f GB" %
                             (need / 1e9, self.budget / 1e9))
                continue
            if self.in_use + need > self.budget:
                if req.rid not in self._waited:
                    self._waited.add(req.rid)
                    self.queued_while_full += 1
                break  # first come, first served: wait for memory
            self.waiting.pop(0)
            try:
                ctx = self._context(req)
            except RLBError as e:  # e.g. RLB_ENOMEM: the device has less free memory than the budget says
                self._finish(req, "failed", str(e))
                continue
            try:
                ctx.init(*initial_fields(req))
            except RLBError as e:
                ctx.close()
                self._finish(req, "failed", str(e))
                continue
            nz, ny, nx = req.shape
            if nx * ny * nz >= self.solo_cells:
                key = ("solo", req.rid)
                self.solo_left[req.rid] = req.steps
            else:
                key = (req.storage, self._batch(req.storage).add(ctx, req.steps))
            self.active[key] = (req, ctx, self.now(), need)
            self.in_use += need
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            self.peak_active = max(self.peak_active, len(self.active))
            admitted += 1
        return admitted

    def _steps_left(self, key):
        if key[0] == "solo":
            return self.solo_left[self.active[key][0].rid]
        return self.batches[key[0]].steps_left(key[1])

    def _round(self):
        for storage, b in self.batches.items():
            if any(k[0] == storage for k in self.active):
                b.run(self.chunk, graph=self.use_graph)
        for key, (req, ctx, _, _) in list(self.active.items()):
            if key[0] == "solo":
                k = min(self.chunk, self.solo_left[req.rid])
                ctx.step(k)
                self.solo_left[req.rid] -= k
        for key in [k for k, v in self.active.items() if v[0].rid in self.cancelled]:
            req, ctx, t_adm = self._release(key)
            self.cancelled.discard(req.rid)
            self._finish(req, "cancelled", admitted=t_adm)
        done = [k for k in self.active if self._steps_left(k) == 0]
        for key in done:
            req, ctx, t_adm, need = self.active[key]
            try:
                m = ctx.moments()
                status, detail = "ok", ""
            except RLBError as e:  # a simulation that broke down (no Landau frame, NaN) is reported
                m, status, detail = None, "failed", str(e)
                if (self.escalate and e.status in (RLB_ENONCONV, RLB_ENAN) and req.storage != "f64"
                        and req.rid not in self.cancelled):
                    # rerun from the initial state in double storage, ahead of the waiting queue
                    self._release(key)
                    self.escalated += 1
                    self.waiting.insert(0, dataclasses.replace(req, storage="f64", escalated_from=req.storage))
                    continue
            self._release(key)
            self._finish(req, status, detail, m, t_adm, req.steps)

    def run(self, requests, realtime=True, max_wall=None, on_round=None):
        """Serve a request stream.  With realtime=True a request is only visible after its arrival
        time (wall clock since the start); otherwise all are queued at once.  on_round(server), if
        given, is called after every round (e.g. to cancel requests)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self.t0 = time.perf_counter()
        k = 0
        while k < len(pending) or self.waiting or self.active:
            t = self.now()
            while k < len(pending) and (not realtime or pending[k].arrival <= t):
                self.waiting.append(pending[k])
                k += 1
            self._admit()
            if self.active:
                self._round()
            elif k < len(pending) and realtime:
                time.sleep(max(0.0, min(0.01, pending[k].arrival - self.now())))
            if on_round is not None:
                on_round(self)
            if max_wall is not None and self.now() > max_wall:
                raise TimeoutError("serving did not finish within %.0f s" % max_wall)
        makespan = self.now()
        for b in self.batches.values():
            self.kernel_launches += b.kernel_launches
        return self.stats(makespan)

    def stats(self, makespan):
        ok = [r for r in self.results if r.status == "ok"]
        tts = np.array([r.tts for r in ok])
        upd = float(sum(r.cells * r.steps for r in ok))
        count = {s: sum(r.status == s for r in self.results) for s in ("ok", "rejected", "failed", "cancelled")}
        return {"requests": len(self.results), "completed": count["ok"], "rejected": count["rejected"],
                "failed": count["failed"], "cancelled": count["cancelled"], "makespan_s": makespan,
                "p50_tts_s": float(np.percentile(tts, 50)) if len(tts) else None,
                "p99_tts_s": float(np.percentile(tts, 99)) if len(tts) else None,
                "aggregate_mlups": upd / makespan / 1e6 if makespan > 0 else None,
                "cell_updates": upd, "peak_hbm_gb": self.peak_in_use / 1e9, "peak_active": self.peak_active,
                "queued_while_full": self.queued_while_full, "budget_gb": self.budget / 1e9,
                "escalated_to_f64": self.escalated}

    def close(self):
        for _, ctx, _, _ in self.active.values():
            ctx.close()
        self.active.clear()
        for b in self.batches.values():
            b.close()
        self.batches.clear()
