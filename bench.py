"""Throughput benchmark of the relativistic lattice Boltzmann step on GB300.

Workload (one "step" = one time step of the whole lattice through the fused pull-collide kernel):
the 256^3 periodic random-field case of the third-order model (Q = 128) with float storage:
velocity from Fourier modes |k| <= 4 rescaled to max |v| = 0.6, log-normal temperature
(sigma 0.2, mean 1), uniform density n = 1 (the n = T^3 variant of this case loses its Landau
frames in 3D; see the design notes), eta/s = 0.1 with the local-temperature relaxation time.

Prints one JSON line:
  value      MLUPS (million lattice-cell updates per second) with the state resident in HBM;
  e2e        the same metric for a whole job through the C ABI from pinned host buffers
             (rlb_init from host fields, K steps, rlb_moments back to host);
  roofline   the step kernel's algorithmic bytes (Q x 2 x 4 bytes per cell update) per launch over
             its CUDA-event duration, against the measured HBM copy bandwidth;
  batched    64 uneven instances at their full step counts in persistent batched launches,
             against the same instances one at a time and against double storage (solves/s and
             the float-vs-double field error per instance of a subset);
  serving    a Poisson request stream plus three 384^3 requests under a 150 GB budget (p50/p99
             time to solution, peak device bytes, requests that waited for memory);
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample of the same workload;
  fp64_plain the same lattice with double storage and arithmetic (MLUPS).

--impl reference times the oracle alone (the reference arm of this comparison).
Multi-GPU (torchrun): every rank steps its own independent lattice (replicas; no collective on the
data path); value = all ranks' cell updates / the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_inputs import fields as gen  # noqa: E402

METRIC = "MLUPS"
BASELINE_METRIC = "MLUPS & HBM-roofline %, FP32 batched vs FP64 plain at <=1e-5 rel err; p50/p99"
N_LATTICE = 256
ORDER = 3
Q = 128
ETA_S = 0.1
DENSITY = "uniform"
SIGMA_LNT = 0.2
WORKLOAD = ("random-field %d^3 periodic, third-order RLB (Q=128, R^2=41), FP32 storage, eta/s=0.1, "
            "max|v|=0.6, log-normal T (sigma 0.2, mean 1), uniform n")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# Sources that decide the step kernels' memory traffic: a DRAM-traffic record taken with ncu is
# used only while these are byte-for-byte the ones it was taken on.
TRAFFIC_SOURCES = ("rlb_kernels.cuh", "rlb_pipe.cuh", "rlb_common.h", "rlb_inst_variant.cu", "rlb_inst_pipe.cu")


def kernel_sources_digest():
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1301_3423_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "step_f32_traffic.json")


def recorded_traffic(n_side, variant, density, path=None):
    """DRAM bytes (read + write) of one step from profiles/step_f32_traffic.json, or None when the
    record is missing or was taken on other kernel sources, another variant or lattice."""
    path = path or TRAFFIC_RECORD
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if (rec.get("sources_sha256") != kernel_sources_digest() or rec.get("variant") != variant
            or rec.get("lattice") != n_side or rec.get("density") != density):
        return None
    return rec.get("dram_bytes_per_step")


def step_kernel_name(variant):
    """The kernels one time step of float storage launches with this variant."""
    from paper_1301_3423_gb300.rlb import VARIANT_NAMES
    name = VARIANT_NAMES[variant] if 0 <= variant < len(VARIANT_NAMES) else str(variant)
    if variant >= 4:
        return "k_step_pipe<Quad3, StoreF32> (%s; one launch per step)" % name
    return "k_step_interior + k_step_shell_rows <Quad3, StoreF32, variant %d> (%s)" % (variant, name)


def dist_env():
    """(world, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_setup(backend=None):
    """One process per GPU: join the process group when world > 1 (NCCL when CUDA is present,
    else gloo, or `backend`).  The replicas exchange only timings, never simulation data."""
    world, rank, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The maximum of x over all ranks (the slowest replica's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, cells, steps, ms_max):
    """Whole-job cell updates per second (MLUPS) of `world` replicas that each took `steps` steps
    of `cells` cells, over the slowest replica's time."""
    return world * cells * steps / (ms_max * 1e-3) / 1e6


def cpu_baseline(n, T, u, budget_s=12.0, planes=2):
    """The FP64 oracle, as it stands, on one host core, timed on a bounded sample of the workload:
    the first ``planes`` z-planes of the same initial fields as a periodic slab, stepped until
    about budget_s seconds are spent."""
    import oracle
    lat = oracle.read_lattice(ORDER)
    ns, Ts, us = n[:planes].copy(), T[:planes].copy(), u[:, :planes].copy()
    nz, ny, nx = ns.shape
    o = oracle.OracleRLB(lat, nx, ny, nz, eta_over_s=ETA_S)
    o.init(ns, Ts, us)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    cells = nx * ny * nz
    return {"value": cells * steps / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "host_cores": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": "%d steps of the first %d z-planes of the %dx%dx%d workload as a periodic %dx%dx%d slab "
                      "(%d cells; serial FP64 C oracle, %.1f s)" % (steps, planes, nx, ny, nx, nx, ny, nz, cells, dt)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def field_errors(ref, got):
    """n, eps pointwise relative; u as max|du| / max(max|u_ref|, 0.01)."""
    en = float(np.max(np.abs(got["n"] - ref["n"]) / np.abs(ref["n"])))
    ee = float(np.max(np.abs(got["eps"] - ref["eps"]) / np.abs(ref["eps"])))
    ur = ref["U"][1:] / ref["U"][0]
    ug = got["U"][1:] / got["U"][0]
    du = float(np.max(np.sqrt(((ug - ur) ** 2).sum(axis=0))))
    return {"n_rel": en, "eps_rel": ee, "u_rel": du / max(float(np.max(np.sqrt((ur ** 2).sum(axis=0)))), 0.01)}


def batched_instances(scale, seed=4, count=64):
    """The batched workload: `count` instances drawn by seed from shock tubes 1x1xN (N in 400..4000,
    copy-out ends, 500 steps) and 32^3..128^3 periodic shear (2000 steps) or random-field (1000
    steps) boxes, eta/s in {0.01, 0.1, 0.5}; step counts times `scale`."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        kind = str(rng.choice(["tube", "shear", "random"]))
        eta = float(rng.choice([0.01, 0.1, 0.5]))
        if kind == "tube":
            N = int(rng.integers(400, 4001))
            shape, bc, steps = (N, 1, 1), (0, 0, 1), 500
        else:
            L = int(rng.choice([32, 48, 64, 96, 128]))
            shape, bc, steps = (L, L, L), (0, 0, 0), (2000 if kind == "shear" else 1000)
        out.append((kind, shape, bc, eta, max(1, int(round(steps * scale))), int(rng.integers(1 << 30))))
    return out


def make_instance(spec, storage, variant=-1, stream=None, landau_fp64=False):
    """One instance of the batched workload.  Float storage solves Landau matching in float with a
    double solve for cells above gamma_thr; landau_fp64=True solves every cell in double."""
    from paper_1301_3423_gb300 import RLB
    kind, shape, bc, eta, steps, seed = spec
    c = RLB(shape, order=ORDER, bc=bc, eta_over_s=eta, storage=storage, landau_fp64=landau_fp64,
            step_variant=variant, stream=stream)
    if kind == "tube":
        f = gen.riemann_tube(shape[0])
    elif kind == "shear":
        f = gen.shear_wave(shape[2], amp=0.05, ny=shape[1], nz=shape[0])
    else:
        f = gen.smooth_random_fields(shape, seed=seed, vmax=0.4, sigma_lnT=0.15, kmax=2, density="uniform")
    c.init(*f)
    return c


def run_batched(args, stream):
    """64 uneven instances stepped together (persistent tile-queue kernels, CUDA-graph step loops),
    against the same instances stepped one at a time in float and in double.  Double storage is
    timed on a subset of 8 instances spread over the mix (it runs at ~0.2 G updates/s), which also
    gives the float-vs-double field error of each of those instances."""
    import torch

    from paper_1301_3423_gb300 import Batch
    specs = batched_instances(args.batch_scale)
    updates = float(sum(np.prod(sp[1]) * sp[4] for sp in specs))
    order = sorted(range(len(specs)), key=lambda k: np.prod(specs[k][1]) * specs[k][4])
    sub = [order[int(round(j * (len(order) // 2 - 1) / 7))] for j in range(8)]  # smaller half of the mix

    def batched_run(landau_fp64, variant=None, keep=()):
        ctxs = [make_instance(sp, "f32", stream=stream, landau_fp64=landau_fp64) for sp in specs]
        b = Batch(ORDER, "f32", stream=stream)
        for c, sp in zip(ctxs, specs):
            b.add(c, sp[4])
        if variant is None:
            variant, _ = b.autotune(reps=2)
        else:
            b.set_variant(variant)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        active = len(ctxs)
        while active:
            active = b.run(25, graph=True)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        kept = {}
        for k, c in enumerate(ctxs):
            if k in keep:
                kept[k] = c.moments()
            c.sync()
            c.close()
        launches = b.kernel_launches
        b.close()
        return t, variant, launches, kept

    t_batch, variant, launches, fields32 = batched_run(False, keep=set(sub))
    t_batch_d, _, _, fields32d = batched_run(True, variant, keep=set(sub))
    t_seq = 0.0  # only the stepping counts, as for the batch
    for sp in specs:
        c = make_instance(sp, "f32", stream=stream)
        c.sync()
        t1 = time.perf_counter()
        c.step(sp[4])
        c.sync()
        t_seq += time.perf_counter() - t1
        c.close()
    u64 = float(sum(np.prod(specs[k][1]) * specs[k][4] for k in sub))
    t64 = 0.0
    errs = []
    for k in sub:
        c = make_instance(specs[k], "f64", stream=stream)
        c.sync()
        t1 = time.perf_counter()
        c.step(specs[k][4])
        c.sync()
        t64 += time.perf_counter() - t1
        m64 = c.moments()
        e = field_errors(m64, fields32[k])
        ed = field_errors(m64, fields32d[k])
        errs.append(dict(kind=specs[k][0], shape=list(specs[k][1]), steps=specs[k][4], eta_over_s=specs[k][3], **e,
                         with_fp64_landau=ed))
        c.close()
    worst = max(max(e["n_rel"], e["eps_rel"], e["u_rel"]) for e in errs)
    worst_d = max(max(e["with_fp64_landau"].values()) for e in errs)
    return {"instances": len(specs), "cell_updates": updates, "step_scale": args.batch_scale,
            "value": updates / t_batch / 1e6, "unit": "MLUPS", "seconds": t_batch, "solves_per_s": len(specs) / t_batch,
            "hbm_frac": updates * Q * 2 * 4 / t_batch / 1e9 / measured_peaks()[0]["hbm_gbs"],
            "variant": variant, "kernel_launches": launches, "graph_steps": 25,
            "landau": "float, double above gamma_thr = 2",
            "fp64_landau_every_cell": {"value": updates / t_batch_d / 1e6, "seconds": t_batch_d,
                                       "solves_per_s": len(specs) / t_batch_d},
            "sequential_f32": {"value": updates / t_seq / 1e6, "seconds": t_seq, "solves_per_s": len(specs) / t_seq},
            "fp64_plain": {"value": u64 / t64 / 1e6, "instances": len(sub), "seconds": t64,
                           "solves_per_s_est": len(specs) / (t64 * updates / u64),
                           "estimate": "the subset's double-storage rate applied to the whole mix"},
            "f32_batched_vs_f64_plain": {"max_rel_err": worst, "max_rel_err_fp64_landau": worst_d, "bar": 1e-5,
                                         "per_instance": errs}}


def run_serving(args, stream):
    """Poisson request stream (mean 20 / s, 40 requests, sides up to 384 drawn with probability
    proportional to 1/L^3, full step counts) plus three 384^3 float shear-wave requests (2000 steps)
    early in the stream, through the continuous-batching server under a 150 GB budget: two 384^3
    lattices fit (58 GB each), the third waits for memory.  Reduced-precision simulations that
    break down numerically are rerun in double storage (listed under "escalated")."""
    from paper_1301_3423_gb300 import serve
    reqs = serve.poisson_requests(40, rate=20.0, seed=5, step_scale=args.batch_scale, f16_fraction=0.3)
    for j, t in enumerate((0.0, 0.02, 0.04)):
        reqs.append(serve.Request(1000 + j, "shear", (384, 384, 384), 0.1, max(1, int(round(2000 * args.batch_scale))),
                                  "f32", 77 + j, t))
    srv = serve.Server(hbm_budget=150e9, chunk=25, stream=stream, escalate=True)
    try:
        st = srv.run(reqs, realtime=True, max_wall=900)
    finally:
        srv.close()
    big = [r.tts for r in srv.results if r.rid >= 1000 and r.status == "ok"]
    by_id = {r.rid: r for r in reqs}
    st["not_ok"] = [{"rid": r.rid, "status": r.status, "detail": r.detail[:200], "kind": by_id[r.rid].kind,
                     "shape": list(by_id[r.rid].shape), "eta_over_s": by_id[r.rid].eta_over_s,
                     "storage": by_id[r.rid].storage} for r in srv.results if r.status != "ok"]
    st["escalated"] = [{"rid": r.rid, "detail": r.detail[:200], "kind": by_id[r.rid].kind,
                        "shape": list(by_id[r.rid].shape), "eta_over_s": by_id[r.rid].eta_over_s,
                        "from": by_id[r.rid].storage, "status": r.status}
                       for r in srv.results if r.storage == "f64" and by_id[r.rid].storage != "f64"]
    st.update({"rate_per_s": 20.0, "step_scale": args.batch_scale,
               "largest_side": max(max(r.shape) if r.kind != "tube" else 0 for r in reqs),
               "f16dev_requests": sum(r.storage == "f16dev" for r in reqs),
               "tts_384_s": big, "solo_cells": srv.solo_cells})
    return st


def workload_config(args, world):
    """The benchmark workload's config (the same for this arm and the reference arm)."""
    N = args.n
    return {"workload": WORKLOAD % N, "lattice": [N, N, N], "order": ORDER, "q": Q, "storage": "f32",
            "eta_over_s": ETA_S, "max_v": 0.6, "sigma_lnT": args.sigma, "density": args.density,
            "boundary": "periodic", "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2: two population buffers of %.1f GB" % (N ** 3 * Q * 4 / 1e9),
            "baseline_metric": BASELINE_METRIC}


def run_reference(args, world, rank):
    if rank != 0:
        return
    N = args.n
    n, T, u = gen.smooth_random_fields((N, N, N), seed=1, vmax=0.6, sigma_lnT=args.sigma, density=args.density)
    budget = args.cpu_budget if args.cpu_budget > 0 else max(10.0, min(60.0, 0.1 * args.steps))
    cb = cpu_baseline(n, T, u, budget_s=budget)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args, world),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", "--lattice", dest="n", type=int, default=N_LATTICE, help="lattice edge (default 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--variant", type=int, default=-1, help="force a step-kernel variant instead of autotuning")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="fraction of the batched / served step counts (500 / 2000 / 1000) to run")
    ap.add_argument("--density", default=DENSITY, choices=["uniform", "cube"],
                    help="initial density: uniform n = 1, or n = T^3")
    ap.add_argument("--sigma", type=float, default=SIGMA_LNT, help="std of ln T")
    ap.add_argument("--cpu-budget", type=float, default=0.0,
                    help="seconds of oracle work for the CPU baseline / reference arm (0: default)")
    args = ap.parse_args()
    if args.impl == "reference":
        # rank 0 alone times the oracle; the other ranks exit without work (no process group)
        world, rank, _ = dist_env()
        run_reference(args, world, rank)
        return
    world, rank, local = dist_setup()

    import torch

    from paper_1301_3423_gb300 import RLB
    from paper_1301_3423_gb300.rlb import VARIANT_NAMES
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    N = args.n
    shape = (N, N, N)
    cells = N ** 3
    n, T, u = gen.smooth_random_fields(shape, seed=1 + rank, vmax=0.6, sigma_lnT=args.sigma, density=args.density)


    # ---- device-resident throughput (the headline value) ------------------------------------
    g = RLB(shape, order=ORDER, storage="f32", eta_over_s=ETA_S, stream=stream, step_variant=args.variant)
    g.init(n, T, u)
    if args.variant < 0:
        variant, variant_ms = g.autotune(reps=3)
    else:
        variant, variant_ms = args.variant, []
    g.step(args.warmup)
    g.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = g.kernel_launches
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_wall = time.perf_counter()
        e0.record(stream)
        g.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    barrier(world)
    launches = g.kernel_launches - launches0
    ms_total = e0.elapsed_time(e1)
    ms_total_max = max_over_ranks(ms_total, world)
    g.sync()  # raises if any cell lost its Landau frame: a broken simulation is not a measurement
    value = job_value(world, cells, args.steps, ms_total_max)
    # A step is one launch of the interior kernel plus one of the shell kernel (disjoint cells):
    # the roofline takes the algorithmic bytes of the whole step over the step's device time.
    per_step_s = ms_total * 1e-3 / args.steps
    algo_bytes = cells * Q * 2 * 4
    peaks, peak_src = measured_peaks()
    achieved = algo_bytes / per_step_s / 1e9
    traffic = recorded_traffic(N, variant, args.density)
    g.close()

    # ---- FP64 plain path on the same lattice ------------------------------------------------
    fp64 = None
    if not args.no_fp64:
        k64 = max(3, args.steps // 30)
        g64 = RLB(shape, order=ORDER, storage="f64", eta_over_s=ETA_S, stream=stream)
        g64.init(n, T, u)
        g64.step(2)
        g64.sync()
        e0.record(stream)
        g64.step(k64)
        e1.record(stream)
        e1.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1), world)
        g64.sync()
        g64.close()
        fp64 = {"value": world * cells * k64 / (ms64 * 1e-3) / 1e6, "unit": "MLUPS", "steps": k64,
                "ms_per_step": ms64 / k64, "bound": "fp64 alu"}

    # ---- float against double fields after the same steps -------------------------------------
    accuracy = None
    if not args.no_accuracy:
        ka = 30
        res, rates = {}, {}
        for st_name in ("f32", "f64", "f16dev"):
            ga = RLB(shape, order=ORDER, storage=st_name, eta_over_s=ETA_S, stream=stream,
                     step_variant=(variant if st_name == "f32" else -1))
            ga.init(n, T, u)
            ga.sync()
            e0.record(stream)
            ga.step(ka)
            e1.record(stream)
            e1.synchronize()
            rates[st_name] = cells * ka / (e0.elapsed_time(e1) * 1e-3) / 1e6
            res[st_name] = ga.moments()
            ga.close()
        accuracy = dict(steps=ka, **field_errors(res["f64"], res["f32"]))
        e16 = field_errors(res["f64"], res["f16dev"])
        accuracy["f16dev"] = dict(e16, mlups=rates["f16dev"], bar=1e-5,
                                  meets_bar=max(e16.values()) <= 1e-5,
                                  note="half-precision store of f_i / w_i - n_ref / 2: about 11 significant bits "
                                       "per population, below the 1e-5 field bar")
        del res

    # ---- end to end through the C ABI from pinned host buffers -------------------------------
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hn, hT, hu = pin(n), pin(T), pin(u)
        on, oe, oU = (torch.empty(shape, dtype=torch.float64).pin_memory(),
                      torch.empty(shape, dtype=torch.float64).pin_memory(),
                      torch.empty((4,) + shape, dtype=torch.float64).pin_memory())
        ge = RLB(shape, order=ORDER, storage="f32", eta_over_s=ETA_S, stream=stream, step_variant=variant)
        ptr = lambda t: t.numpy()
        outs = dict(n=on.numpy(), eps=oe.numpy(), U=oU.numpy())
        ge.init(ptr(hn), ptr(hT), ptr(hu))
        ge.step(args.warmup)
        ge.moments(out=outs)
        ge.sync()
        jobs = []
        for _ in range(5):  # the whole job five times; the median is reported, all five are kept
            barrier(world)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            t0 = time.perf_counter()
            ev[0].record(stream)
            ge.init(ptr(hn), ptr(hT), ptr(hu))
            ev[1].record(stream)
            ge.step(args.steps)
            ev[2].record(stream)
            ge.moments(out=outs)
            ev[3].record(stream)
            t_job = max_over_ranks(time.perf_counter() - t0, world)
            jobs.append({"s": t_job, "init_ms": ev[0].elapsed_time(ev[1]), "steps_ms": ev[1].elapsed_time(ev[2]),
                         "moments_ms": ev[2].elapsed_time(ev[3])})
        ge.close()
        t_e2e = statistics.median(j["s"] for j in jobs)
        h2d = 5 * cells * 8
        d2h = 6 * cells * 8 + 5 * 8
        e2e = {"value": world * cells * args.steps / t_e2e / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "job": "rlb_init from pinned host fields + %d steps + rlb_moments to host; median of 5 jobs"
                      % args.steps, "jobs": jobs}

    batched = None if args.no_batch else run_batched(args, stream)
    serving = None if args.no_serve else run_serving(args, stream)
    if rank != 0:
        return
    cb = None if args.no_cpu_baseline else cpu_baseline(n, T, u)
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": peak_src, "algorithmic_bytes_per_step": algo_bytes,
                     "kernel": step_kernel_name(variant),
                     "step_ms": per_step_s * 1e3, "launches_per_step": launches / args.steps},
        "cpu_baseline": cb,
        "e2e": e2e,
        "fp64_plain": fp64,
        "accuracy_f32_vs_f64": accuracy,
        "batched": batched,
        "serving": serving,
        "gpu_launches": launches,
        "autotune": {"variant": variant, "ms_per_step": variant_ms,
                     "variants": VARIANT_NAMES[:len(variant_ms)]},
        "clocks": clk.summary(),
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
