"""bench.py without a GPU: the reference arm's JSON line (the CPU oracle on a
bounded sample), its behaviour on ranks other than 0, and the max-over-ranks
timing of the multi-GPU replicas, run as two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def run_bench(args, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=600)


def test_reference_arm_prints_the_contract_line():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * bench.interior(bench.LEVEL) / d["value"]) < 1e-6
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOAD


def test_reference_arm_other_ranks_exit_without_work():
    r = run_bench(["--impl", "reference", "--gpus", "2"], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_whole_job_rate():
    assert bench.whole_job_rate(1, 1000, 10, 1000.0) == 10000.0
    assert bench.whole_job_rate(4, 1000, 10, 1000.0) == 40000.0
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 17.25][rank]
    m = bench.max_over_ranks(ms, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
        f.write(repr(m))


def test_max_over_ranks_with_two_gloo_ranks(tmp_path):
    """Each replica times its own steps; the line reports the slowest rank's
    time, which every rank receives."""
    mp = pytest.importorskip("torch.multiprocessing")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [float(open(tmp_path / f"r{r}.txt").read()) for r in range(2)]
    assert got == [17.25, 17.25]
