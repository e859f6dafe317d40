"""Integrals given on the device (sci_set_integrals_ex, on_device = 1): the same tables,
diagonal and sigma as from host memory, in real and complex spinor mode, from Cholesky
vectors and from dense (pq|rs); the device-side symmetry checks reject what the host-side
checks reject, and host pointers are refused."""
import ctypes

import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sigma_pair(torch, w, use_chol):
    Hh = sci.Hamiltonian()
    Hd = sci.Hamiltonian()
    if use_chol:
        Hh.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
        Hd.set_integrals(w.mode, torch.from_numpy(w.ints.h).cuda(), chol=torch.from_numpy(w.ints.chol).cuda())
    else:
        eri = w.ints.eri()
        Hh.set_integrals(w.mode, w.ints.h, eri=eri)
        Hd.set_integrals(w.mode, torch.from_numpy(w.ints.h).cuda(), eri=torch.from_numpy(eri).cuda())
    Hh.set_determinants(w.keys, w.n_alpha, w.n_beta)
    Hd.set_determinants(w.keys, w.n_alpha, w.n_beta)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    return Hh, Hd, C


@pytest.mark.parametrize("name,use_chol", [("fci_8o", True), ("fci_8o", False), ("spinor", True), ("spinor", False),
                                           ("sel60k", True)])
def test_device_integrals_give_the_host_result(gpu, name, use_chol):
    torch = gpu
    w = {"fci_8o": lambda: W.fci_small_8o(),
         "spinor": lambda: W.random_small(41, "spinors", 10, 4, 0, naux=6, frac=0.6),
         "sel60k": lambda: W.selected_30o(M=60000)}[name]()
    Hh, Hd, C = _sigma_pair(torch, w, use_chol)
    assert torch.equal(Hh.diagonal(), Hd.diagonal())
    # the same tables: with row sums in a fixed order the two sigmas agree bit for bit
    Hh.set_deterministic(1)
    Hd.set_deterministic(1)
    Sh, Sd = Hh.sigma(C), Hd.sigma(C)
    assert torch.equal(Sh, Sd)
    if name != "sel60k":
        o = Oracle.from_workload(w)
        ref = o.sigma(w.c)
        assert np.linalg.norm(Sd.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)


def test_device_integral_checks(gpu):
    torch = gpu
    w = W.random_small(71, "spin_orbitals", 5, 2, 2)
    H = sci.Hamiltonian()
    h = torch.from_numpy(w.ints.h).cuda()
    L = torch.from_numpy(w.ints.chol).cuda()
    bad = h.clone()
    bad[0, 1] += 1.0
    with pytest.raises(sci.SciError) as e:
        H.set_integrals(w.mode, bad, chol=L)
    assert e.value.code == sci.SCI_ERR_ARG and "Hermitian" in str(e.value)
    badL = L.clone()
    badL[1, 0, 2] += 1e-3
    with pytest.raises(sci.SciError) as e:
        H.set_integrals(w.mode, h, chol=badL)
    assert e.value.code == sci.SCI_ERR_ARG and "Cholesky" in str(e.value)
    eri = torch.from_numpy(w.ints.eri()).cuda()
    bad_eri = eri.clone()
    bad_eri[0, 1, 2, 3] += 1e-3
    with pytest.raises(sci.SciError) as e:
        H.set_integrals(w.mode, h, eri=bad_eri)
    assert e.value.code == sci.SCI_ERR_ARG and "symmetry" in str(e.value)
    nan_h = h.clone()
    nan_h[2, 2] = float("nan")
    with pytest.raises(sci.SciError) as e:
        H.set_integrals(w.mode, nan_h, chol=L)
    assert e.value.code == sci.SCI_ERR_ARG and "finite" in str(e.value)
    # a host pointer with on_device = 1 is refused before anything reads it
    hn = np.ascontiguousarray(w.ints.h)
    Ln = np.ascontiguousarray(w.ints.chol)
    with pytest.raises(sci.SciError) as e:
        sci.sci_set_integrals_ex(H.ctx, sci.SCI_REAL64, sci.SCI_SPIN_ORBITALS, w.n, hn, None, Ln.shape[0], Ln, 1)
    assert e.value.code == sci.SCI_ERR_ARG
    # the context stays usable
    H.set_integrals(w.mode, h, chol=L)
    H.set_determinants(w.keys, 2, 2)
    o = Oracle.from_workload(w)
    S = H.sigma(torch.from_numpy(w.c).cuda()).cpu().numpy()
    ref = o.sigma(w.c)
    assert np.linalg.norm(S - ref) <= 1e-11 * np.linalg.norm(ref)
