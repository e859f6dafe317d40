"""Row partition of sigma on CPU (paper Sec. 3.1: static data replicated, results merged):
the cost-balanced ranges, and the all-gather of row slices over two and three gloo ranks,
with each rank's rows computed by the oracle (the GPU computes them in the -m gpu tests)."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2501_18185_gb300 import partition as PT
from paper_2501_18185_gb300 import workloads as W


def _check_ranges(r, M, parts):
    assert len(r) == parts and r[0][0] == 0 and r[-1][1] == M
    for (b0, e0), (b1, e1) in zip(r, r[1:]):
        assert b0 <= e0 == b1 <= e1


@pytest.mark.parametrize("parts", [1, 2, 3, 7, 16])
def test_balanced_ranges_cover_and_balance(parts):
    rng = np.random.default_rng(parts)
    w = rng.exponential(size=1001) * 100
    w[rng.random(1001) < 0.1] = 0.0
    r = PT.balanced_ranges(w, parts)
    _check_ranges(r, len(w), parts)
    target = w.sum() / parts
    for b, e in r:
        assert w[b:e].sum() <= target + w.max() + 1e-9


def test_balanced_ranges_edge_cases():
    _check_ranges(PT.balanced_ranges(np.zeros(0), 3), 0, 3)                 # no rows
    r = PT.balanced_ranges(np.ones(2), 5)                                     # more parts than rows
    _check_ranges(r, 2, 5)
    assert sum(e - b for b, e in r) == 2
    r = PT.balanced_ranges(np.zeros(10), 4)                                   # all weights zero: by rows
    _check_ranges(r, 10, 4)
    assert [e - b for b, e in r] == [2, 3, 2, 3]
    r = PT.balanced_ranges(np.array([0, 0, 10.0, 0, 0]), 2)                   # one heavy row
    _check_ranges(r, 5, 2)
    with pytest.raises(ValueError):
        PT.balanced_ranges(np.array([1.0, -1.0]), 2)
    with pytest.raises(ValueError):
        PT.balanced_ranges(np.ones(3), 0)


def test_rebalance_evens_out_a_cost_the_weights_miss():
    """True row time = weight x a factor that grows along the list (as the staging of
    touched buckets does): after one measured round, the re-cut ranges are more even."""
    rng = np.random.default_rng(11)
    w = rng.uniform(50, 150, size=20000)
    true = w * np.linspace(1.0, 2.0, w.size)
    for parts in (2, 4, 8):
        r0 = PT.balanced_ranges(w, parts)
        t0 = np.array([true[b:e].sum() for b, e in r0])
        r1 = PT.rebalance(w, r0, t0)
        _check_ranges(r1, w.size, parts)
        t1 = np.array([true[b:e].sum() for b, e in r1])
        assert t1.max() / t1.mean() < t0.max() / t0.mean()
        assert t1.max() / t1.mean() - 1 < 0.15 * (t0.max() / t0.mean() - 1)    # one round
        r2 = PT.rebalance(w, r1, t1)
        t2 = np.array([true[b:e].sum() for b, e in r2])
        assert t2.max() / t2.mean() < 1.005                                     # two rounds
    with pytest.raises(ValueError):
        PT.rebalance(w, PT.balanced_ranges(w, 2), [1.0])


def test_row_weights():
    assert np.array_equal(PT.row_weights([0, 5, 2], 3), [3.0, 8.0, 5.0])


def _rank_main(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import Oracle

        mode, n, na, nb, frac, nvec, forced = case
        w = W.random_small(401 + n, mode, n, na, nb, naux=4, frac=frac, nvec=nvec)
        o = Oracle.from_workload(w)
        cost = np.array([len(o.connections(r)[0]) for r in range(w.M)])
        if forced == "empty_first":   # an empty range, then an uneven split
            ranges = [(0, 0), (0, w.M - 7), (w.M - 7, w.M)]
        else:
            ranges = PT.balanced_ranges(PT.row_weights(cost, 1.0), world)
        b, e = ranges[rank]
        dt = torch.complex128 if mode == "spinors" else torch.float64
        S = torch.full((w.M, nvec), float("nan"), dtype=dt)
        if e > b:
            S[b:e] = torch.from_numpy(o.sigma_rows(np.arange(b, e), w.c))
        PT.gather_rows(S, ranges)
        ref = o.sigma(w.c)
        q.put((rank, bool(np.array_equal(S.numpy(), ref)), ranges))
    except Exception as ex:  # reported to the parent
        q.put((rank, repr(ex), None))
    finally:
        dist.destroy_process_group()


CASES = [
    ("spin_orbitals", 6, 3, 2, 1.0, 1, None),
    ("spinors", 7, 3, 0, 0.6, 2, None),
    ("spin_orbitals", 5, 2, 2, 1.0, 3, "empty_first"),
]


@pytest.mark.parametrize("world,case", [(2, CASES[0]), (2, CASES[1]), (3, CASES[2])])
def test_gather_rows_on_gloo_ranks(world, case):
    """Each rank fills only its range (NaN elsewhere); after the all-gather every rank
    holds the oracle's whole sigma, element for element (the rows are the same oracle
    rows, so the merge must be exact)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 400) + 17 * world + len(case[0])
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for rank, ok, ranges in out:
        assert ok is True, (rank, ok)
    assert len({tuple(map(tuple, r)) for _, _, r in out}) == 1
