"""Row-partitioned sigma on one GPU (paper Sec. 3.1: static data replicated, each process
computing its share of the results, merged at the end).

Each range's sigma comes from a context restricted to that range (sci_set_row_range, its
range tables and RANGED kernels); the ranges together must give the whole sigma: against
the full launch to 1e-12 (the same per-bucket sums, only the order of the FP64 atomic adds
into S differs) and against the oracle to 1e-11, with the rows outside a range left
untouched.  The per-row costs that balance the ranges are checked exactly against the
oracle's connection counts.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import partition as PT
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _workload(name):
    if name == "fci_8o":
        return W.fci_small_8o()
    if name == "spinor_10":
        return W.random_small(5, "spinors", 10, 4, 0, frac=0.5, nvec=3)
    if name == "sel_30o_60k":
        return W.selected_30o(M=60000, nvec=3)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["fci_8o", "spinor_10", "sel_30o_60k"])
def test_row_costs_match_oracle_connection_counts(gpu, name):
    w = _workload(name)
    H = sci.Hamiltonian.from_workload(w)
    cost = H.row_costs().cpu().numpy()
    o = Oracle.from_workload(w)
    rows = np.arange(w.M) if w.M <= 5000 else np.unique(np.r_[0, w.M - 1, np.random.default_rng(3).choice(w.M, 2000)])
    for r in rows:
        assert cost[r] == len(o.connections(int(r))[0]), r
    assert int(cost.sum()) == H.count_pairs()


@pytest.mark.parametrize("name,K", [("fci_8o", 3), ("spinor_10", 2), ("sel_30o_60k", 2), ("sel_30o_60k", 5),
                                    ("sel_30o_60k", 16)])
def test_row_ranges_concatenate_to_sigma(gpu, name, K):
    torch = gpu
    w = _workload(name)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    cost = H.row_costs().cpu().numpy()
    ranges = PT.balanced_ranges(PT.row_weights(cost, 1.0), K)
    total_pairs = H.count_pairs()
    precs = [sci.SCI_PREC_F64, sci.SCI_PREC_F64_DS] + ([] if w.ints.complex_ else [sci.SCI_PREC_F32_STORE_F64_ACC])
    for prec in precs:
        Cp = C.float() if prec == sci.SCI_PREC_F32_STORE_F64_ACC else C
        full = H.sigma(Cp, prec=prec).cpu().numpy()
        merged = np.full_like(full, np.nan)
        pairs = 0
        for b, e in ranges:
            H.set_row_range(b, e)
            S = torch.full(tuple(C.shape), float("nan"), dtype=C.dtype, device=C.device)
            H.sigma(Cp, out=S, prec=prec)
            s = S.cpu().numpy()
            assert np.isnan(s[:b]).all() and np.isnan(s[e:]).all()       # other rows untouched
            merged[b:e] = s[b:e]
            pairs += H.count_pairs()
        H.set_row_range(0, w.M)
        H.sync_status()
        assert pairs == total_pairs
        assert not np.isnan(merged).any()
        err = np.linalg.norm(merged - full) / np.linalg.norm(full)
        assert err < 1e-12, (prec, err)
        assert H.count_pairs() == total_pairs
    # FP64 against the oracle (sampled rows of the large space)
    o = Oracle.from_workload(w)
    rows = np.arange(w.M) if w.M <= 5000 else np.unique(np.random.default_rng(4).choice(w.M, 3000))
    ref = o.sigma_rows(rows, w.c)
    err = np.linalg.norm(merged_f64(H, C, ranges)[rows] - ref) / np.linalg.norm(ref)
    assert err < 1e-11, err


def merged_f64(H, C, ranges):
    S = H.torch.full(tuple(C.shape), float("nan"), dtype=C.dtype, device=C.device)
    for b, e in ranges:                 # one buffer: each range fills its rows
        H.set_row_range(b, e)
        H.sigma(C, out=S)
    H.set_row_range(0, H.M)
    return S.cpu().numpy()


def test_row_range_edges_and_errors(gpu):
    torch = gpu
    w = W.selected_30o(M=60000)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(w.c).cuda()
    full = H.sigma(C).cpu().numpy()
    for b, e in ((7, 7), (0, 1), (w.M - 1, w.M), (12345, 12346), (0, w.M // 2)):
        H.set_row_range(b, e)
        S = torch.full(tuple(C.shape), 3.25, dtype=C.dtype, device=C.device)
        H.sigma(C, out=S)
        s = S.cpu().numpy()
        assert (s[:b] == 3.25).all() and (s[e:] == 3.25).all()
        if e > b:
            assert np.allclose(s[b:e], full[b:e], rtol=1e-12, atol=1e-15)
        # host buffers: only the range's rows come back
        Sh = np.full(tuple(C.shape), 7.5)
        H.sigma_host(w.c, out=Sh)
        assert (Sh[:b] == 7.5).all() and (Sh[e:] == 7.5).all()
        if e > b:
            assert np.allclose(Sh[b:e], full[b:e], rtol=1e-12, atol=1e-15)
    for b, e in ((-1, 5), (5, 4), (0, w.M + 1)):
        with pytest.raises(sci.SciError):
            H.set_row_range(b, e)
    # a new determinant list clears the range
    H.set_row_range(10, 20)
    H.set_determinants(w.keys, w.n_alpha, w.n_beta)
    assert np.allclose(H.sigma(C).cpu().numpy(), full, rtol=1e-12, atol=1e-15)
    assert H.count_pairs() == int(H.row_costs().sum())


def test_row_split_sigma_class_one_rank(gpu):
    """RowSplitSigma on a one-rank gloo group: the whole range, the all-gather a no-op."""
    import os

    import torch.distributed as dist

    torch = gpu
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", str(29700 + os.getpid() % 200))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        w = W.fci_small_8o()
        H = sci.Hamiltonian.from_workload(w)
        C = torch.from_numpy(w.c).cuda()
        ref = H.sigma(C).cpu().numpy()
        rs = PT.RowSplitSigma.balanced(H, 1, 0)
        assert rs.ranges == [(0, w.M)]
        S = torch.empty_like(C)
        # gloo moves CPU tensors: gather on a host copy, as a CPU-side caller would
        out = rs.H.sigma(C, out=S).cpu()
        PT.gather_rows(out, rs.ranges)
        assert np.allclose(out.numpy(), ref, rtol=1e-13, atol=1e-15)
    finally:
        dist.destroy_process_group()


def test_whole_list_calls_ignore_the_row_range(gpu):
    """ENPT2 (its E2[P] sigma), the density matrices and the pair export of a context with
    a row range set still cover the whole list, as include/sci.h states."""
    torch = gpu
    w = W.random_small(305, "spin_orbitals", 10, 2, 2, naux=6, frac=0.2)
    H = sci.Hamiltonian.from_workload(w)
    ev, U = np.linalg.eigh(Oracle.from_workload(w).dense())
    C = torch.from_numpy(U[:, :2].copy()).cuda()
    ref = H.enpt2(C, ev[:2])
    g1, g2 = H.rdm12(C)
    n_all, _ = sci.sci_connections(H.ctx, 0, w.M, 0)
    H.set_row_range(w.M // 3, w.M // 2)
    got = H.enpt2(C, ev[:2])
    assert np.allclose(got[2], ref[2], rtol=1e-12) and np.allclose(got[1], ref[1], rtol=1e-12)
    h1, h2 = H.rdm12(C)
    assert torch.allclose(h1, g1, rtol=1e-12, atol=1e-14) and torch.allclose(h2, g2, rtol=1e-12, atol=1e-14)
    assert sci.sci_connections(H.ctx, 0, w.M, 0)[0] == n_all
