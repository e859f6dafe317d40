"""The multi-rank path of bench.py on CPU: two gloo ranks, each a replica with its own
time; the job is timed by the slowest rank and its throughput counts both replicas."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    total = bench.max_over_ranks(100.0 + 25.0 * rank, dist, "cpu")
    dist.barrier()
    q.put((rank, total, bench.job_throughput(1000, 4, world, total)))
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's 125 ms; 2 replicas x 1000 pairs x 4 steps / 0.125 s
    assert [t for _, t, _ in out] == [125.0, 125.0]
    assert all(v == pytest.approx(2 * 1000 * 4 / 0.125) for _, _, v in out)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(10, 2, 1, 1000.0) == pytest.approx(20.0)


def test_reference_arm_json_line():
    """`bench.py --impl reference` prints one JSON line with the keys the benchmark
    contract asks of the reference arm (on the 8-orbital FCI workload, a few seconds)."""
    import json
    import subprocess
    import sys

    ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "fci_8o", "--steps", "2", "--warmup", "1", "--ref-rows", "200"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
