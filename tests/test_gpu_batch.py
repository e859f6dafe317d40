"""Batched sigma over 64 heterogeneous full-CI instances in one persistent launch.

Every instance's slice of the batched result is checked against the oracle (all rows of
the small instances, sampled rows of the large ones) under each schedule, and against
the instance's own sci_sigma.  The graph-captured launch replays to the same result.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11
_cache = {}


def batch_case(torch):
    if "b" not in _cache:
        ws = W.batch_instances()
        hams = [sci.Hamiltonian.from_workload(w) for w in ws]
        C = torch.from_numpy(np.concatenate([w.c[:, 0] for w in ws])).cuda()
        refs = []
        for w in ws:
            o = Oracle.from_workload(w)
            rows = np.arange(w.M) if w.M <= 3000 else np.unique(np.concatenate(
                [np.random.default_rng(w.M).choice(w.M, 1500, replace=False), [0, w.M - 1]]))
            refs.append((rows, o.sigma_rows(rows, w.c)[:, 0]))
        _cache["b"] = (ws, hams, C, refs)
    return _cache["b"]


def check_all(ws, S, offsets, refs):
    S = S.cpu().numpy()
    for w, off, (rows, ref) in zip(ws, offsets, refs):
        got = S[off + rows]
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err < TOL, (w.name, err)


@pytest.mark.parametrize("schedule", [sci.SCI_SCHED_TILE, sci.SCI_SCHED_WARP, sci.SCI_SCHED_AUTO])
def test_batch_matches_oracle(gpu, schedule):
    torch = gpu
    ws, hams, C, refs = batch_case(torch)
    B = sci.Batch(hams)
    assert B.M == sum(w.M for w in ws)
    B.plan(schedule, C, torch.empty_like(C))
    S = B.sigma(C)
    check_all(ws, S, B.offsets, refs)
    scheds = {B.info(i)["schedule"] for i in range(len(ws))}
    if schedule == sci.SCI_SCHED_AUTO:
        assert scheds <= {"tile", "warp"}
        assert all(B.info(i)["ms_tile"] > 0 and B.info(i)["ms_warp"] > 0 for i in range(len(ws)))
    it = B.items()
    assert it["M"] == B.M and it["pairs"] == sum(H.count_pairs() for H in hams) and it["ctas"] > 0


def test_batch_graph_replay_and_instance_sigma(gpu):
    torch = gpu
    ws, hams, C, refs = batch_case(torch)
    B = sci.Batch(hams)
    B.plan(sci.SCI_SCHED_AUTO, C, torch.empty_like(C))
    S = torch.full_like(C, np.nan)
    B.capture(C, S)
    B.replay()
    torch.cuda.synchronize()
    check_all(ws, S, B.offsets, refs)
    first = S.clone()
    B.replay()
    B.replay()
    torch.cuda.synchronize()
    assert float((S - first).abs().max()) <= 1e-13 * float(first.abs().max())
    # each slice equals the instance's own sigma
    for H, w, off in zip(hams, ws, B.offsets):
        own = H.sigma(C[off:off + w.M]).cpu().numpy()
        sl = S[off:off + w.M].cpu().numpy()
        assert np.linalg.norm(sl - own) <= 1e-13 * max(np.linalg.norm(own), 1e-300)


def test_batch_mixed_selected_instance(gpu):
    """A selected (non-FCI) instance: WARP is refused, AUTO and TILE take the bucket walk."""
    torch = gpu
    ws = [W.random_small(81, "spin_orbitals", 9, 3, 3, frac=0.6), W.random_small(82, "spin_orbitals", 8, 3, 2)]
    hams = [sci.Hamiltonian.from_workload(w) for w in ws]
    C = torch.from_numpy(np.concatenate([w.c[:, 0] for w in ws])).cuda()
    B = sci.Batch(hams)
    with pytest.raises(sci.SciError) as e:
        B.plan(sci.SCI_SCHED_WARP)
    assert e.value.code == sci.SCI_ERR_ARG
    B.plan(sci.SCI_SCHED_AUTO, C, torch.empty_like(C))
    assert B.info(0)["schedule"] == "tile" and B.info(0)["ms_warp"] < 0
    S = B.sigma(C).cpu().numpy()
    for w, off in zip(ws, B.offsets):
        ref = Oracle.from_workload(w).sigma(w.c)[:, 0]
        assert np.linalg.norm(S[off:off + w.M] - ref) / np.linalg.norm(ref) < TOL


def test_batch_errors(gpu):
    torch = gpu
    w = W.random_small(83, "spinors", 8, 3, 0)
    H = sci.Hamiltonian.from_workload(w)
    b = sci.sci_batch_create(0)
    try:
        with pytest.raises(sci.SciError):
            sci.sci_batch_add(b, H.ctx)             # complex instances are not batched
        with pytest.raises(sci.SciError):
            sci.sci_batch_sigma(b, None, None)      # before a plan
        with pytest.raises(sci.SciError):
            sci.sci_batch_replay(b)                 # nothing captured
    finally:
        sci.sci_batch_destroy(b)
