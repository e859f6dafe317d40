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
