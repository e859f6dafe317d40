"""Deterministic accumulation of sigma (sci_set_deterministic): row sums stored per bucket
entry and summed per row in a fixed order (one warp per row, a fixed shuffle butterfly).

Repeated calls, and calls on another stream, must give bitwise equal S in every precision
mode; S must agree with the atomic accumulation (the same per-bucket row sums, added in
another order) to 1e-13 and with the oracle to 1e-11 in FP64.  With atomics, repeats differ
in the last bits (the reason for the mode).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _workload(name):
    return {"fci_8o": lambda: W.fci_small_8o(),
            "sel_30o_60k": lambda: W.selected_30o(M=60000),
            "spinor_10": lambda: W.random_small(5, "spinors", 10, 4, 0, frac=0.5)}[name]()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("name,nvec", [("fci_8o", 1), ("sel_30o_60k", 1), ("sel_30o_60k", 3), ("sel_30o_60k", 8),
                                       ("sel_30o_60k", 11), ("spinor_10", 1), ("spinor_10", 5)])
def test_deterministic_sigma_is_bitwise_reproducible(gpu, name, nvec):
    torch = gpu
    w = _workload(name)
    H = sci.Hamiltonian.from_workload(w)
    rng = np.random.default_rng(7 + nvec)
    C = rng.normal(size=(w.M, nvec)) + (1j * rng.normal(size=(w.M, nvec)) if w.mode == "spinors" else 0)
    Ct = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    precs = [sci.SCI_PREC_F64, sci.SCI_PREC_F64_DS] + ([] if w.mode == "spinors" else [sci.SCI_PREC_F32_STORE_F64_ACC])
    atomic = {}
    for prec in precs:
        Cp = Ct.float() if prec == sci.SCI_PREC_F32_STORE_F64_ACC else Ct
        atomic[prec] = H.sigma(Cp, prec=prec).cpu().numpy()
    H.set_deterministic(16)
    s2 = torch.cuda.Stream()
    for prec in precs:
        Cp = Ct.float() if prec == sci.SCI_PREC_F32_STORE_F64_ACC else Ct
        a = H.sigma(Cp, prec=prec).cpu().numpy()
        b = H.sigma(Cp, prec=prec).cpu().numpy()
        H.set_stream(s2)
        with torch.cuda.stream(s2):
            c = H.sigma(Cp, prec=prec).cpu().numpy()
        s2.synchronize()
        H.set_stream(torch.cuda.current_stream())
        assert np.array_equal(a, b) and np.array_equal(a, c), prec      # bit for bit
        assert _rel(a, atomic[prec]) < 1e-13, (prec, _rel(a, atomic[prec]))
    H.sync_status()
    o = Oracle.from_workload(w)
    rows = np.arange(w.M) if w.M <= 5000 else np.unique(rng.choice(w.M, 2000))
    det64 = H.sigma(Ct).cpu().numpy()
    assert _rel(det64[rows], o.sigma_rows(rows, C)) < 1e-11


def test_deterministic_mode_limits_and_switching(gpu):
    torch = gpu
    w = W.selected_30o(M=60000)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.random.default_rng(3).normal(size=(w.M, 4))).cuda()
    ref = H.sigma(C).cpu().numpy()
    H.set_deterministic(2)
    with pytest.raises(sci.SciError):            # more vectors than the slots hold
        H.sigma(C)
    assert _rel(H.sigma(C[:, :2].contiguous()).cpu().numpy(), ref[:, :2]) < 1e-13
    with pytest.raises(sci.SciError):            # no row range while deterministic
        H.set_row_range(0, 100)
    H.set_deterministic(0)                       # back to atomics
    assert _rel(H.sigma(C).cpu().numpy(), ref) < 1e-13
    H.set_row_range(0, 100)
    with pytest.raises(sci.SciError):            # no deterministic mode while ranged
        H.set_deterministic(4)
    H.set_row_range(0, w.M)
    H.set_deterministic(4)
    # kernel times: the fourth figure is the per-row sums
    sci.sci_profile(H.ctx, True)
    H.sigma(C)
    t = sci.sci_kernel_times(H.ctx, 4)
    assert t[3] > 0 and t[0] >= 0
    sci.sci_profile(H.ctx, False)
    # internal whole-list callers work in this mode too (ENPT2's E2[P] sigma)
    w2 = W.random_small(305, "spin_orbitals", 10, 2, 2, naux=6, frac=0.2)
    H2 = sci.Hamiltonian.from_workload(w2)
    ev, U = np.linalg.eigh(Oracle.from_workload(w2).dense())
    Cu = torch.from_numpy(U[:, :2].copy()).cuda()
    ref2 = H2.enpt2(Cu, ev[:2])
    H2.set_deterministic(2)
    got2 = H2.enpt2(Cu, ev[:2])
    assert np.allclose(got2[2], ref2[2], rtol=1e-12)
