"""The N > 1 path of bench.py on the CPU: one process per rank over gloo.  The benchmark's replicas
share no simulation data; the ranks only agree on the slowest replica's time, from which rank 0
reports the whole-job value, and the reference arm runs on rank 0 alone."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    bench = load_bench()
    w, r, _ = bench.dist_setup("gloo")
    bench.barrier(w)
    ms = 100.0 + 7.0 * r  # each replica's own time
    ms_max = bench.max_over_ranks(ms, w)
    value = bench.job_value(w, 256 ** 3, 300, ms_max)
    bench.barrier(w)
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump({"world": w, "rank": r, "ms_max": ms_max, "value": value}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == world for x in res)
    assert all(x["ms_max"] == 107.0 for x in res)  # the slower replica's time on every rank
    expect = world * 256 ** 3 * 300 / (107.0e-3) / 1e6
    assert all(abs(x["value"] - expect) <= 1e-9 * expect for x in res)


def test_single_process_needs_no_process_group():
    bench = load_bench()
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(1, 10, 4, 2.0) == 10 * 4 / 2e-3 / 1e6


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """bench.py --impl reference launched as two ranks: rank 0 times the oracle and prints one JSON
    line, rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "1", "--lattice", "16", "--cpu-budget", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_traffic_record_is_used_only_for_the_kernel_sources_it_was_taken_on(tmp_path, monkeypatch):
    """roofline.traffic comes from the step traffic record only while the step kernels' sources
    hash to the recorded digest and the variant, lattice and density match."""
    bench = load_bench()
    rec = {"lattice": 256, "variant": 4, "density": "uniform", "dram_bytes_per_step": 1.75e10,
           "algorithmic_bytes_per_step": 17179869184, "sources_sha256": bench.kernel_sources_digest()}
    path = str(tmp_path / "traffic.json")
    json.dump(rec, open(path, "w"))
    assert bench.recorded_traffic(256, 4, "uniform", path) == rec["dram_bytes_per_step"]
    assert bench.recorded_traffic(256, 5, "uniform", path) is None
    assert bench.recorded_traffic(128, 4, "uniform", path) is None
    assert bench.recorded_traffic(256, 4, "cube", path) is None
    assert bench.recorded_traffic(256, 4, "uniform", str(tmp_path / "missing.json")) is None
    monkeypatch.setattr(bench, "kernel_sources_digest", lambda: "0" * 64)  # the kernels changed
    assert bench.recorded_traffic(256, 4, "uniform", path) is None
    # the committed record, if it matches the current sources, is at least the algorithmic bytes
    committed = json.load(open(bench.TRAFFIC_RECORD))
    assert committed["dram_bytes_per_step"] >= committed["algorithmic_bytes_per_step"] * 0.99
