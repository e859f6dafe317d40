"""Degenerate shapes for the density matrices, the batched launch and ENPT2: no beta
electrons, a fully occupied alpha shell (no alpha virtuals), a single determinant."""
import numpy as np
import pytest

from oracle import Oracle
from oracle import pt2 as PT
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(6, 3, 0), (6, 6, 2), (7, 1, 1), (5, 5, 5)]


@pytest.mark.parametrize("n,na,nb", SHAPES)
def test_rdm_degenerate_shapes(gpu, n, na, nb):
    torch = gpu
    w = W.random_small(401 + n + na, "spin_orbitals", n, na, nb, naux=4)
    H = sci.Hamiltonian.from_workload(w)
    g1, g2 = H.rdm12(torch.from_numpy(w.c).cuda())
    r1, r2 = Oracle.from_workload(w).rdm12(w.c[:, 0])
    assert np.abs(g1.cpu().numpy() - r1).max() < 1e-12 and np.abs(g2.cpu().numpy() - r2).max() < 1e-12


@pytest.mark.parametrize("schedule", [sci.SCI_SCHED_TILE, sci.SCI_SCHED_WARP, sci.SCI_SCHED_AUTO])
def test_batch_degenerate_instances(gpu, schedule):
    torch = gpu
    ws = [W.random_small(411 + i, "spin_orbitals", n, na, nb, naux=4) for i, (n, na, nb) in enumerate(SHAPES)]
    hams = [sci.Hamiltonian.from_workload(w) for w in ws]
    C = torch.from_numpy(np.concatenate([w.c[:, 0] for w in ws])).cuda()
    B = sci.Batch(hams)
    B.plan(schedule, C, torch.empty_like(C))
    S = B.sigma(C).cpu().numpy()
    for w, off in zip(ws, B.offsets):
        ref = Oracle.from_workload(w).sigma(w.c)[:, 0]
        assert np.linalg.norm(S[off:off + w.M] - ref) <= 1e-11 * max(np.linalg.norm(ref), 1e-300), w.name


@pytest.mark.parametrize("n,na,nb,frac", [(7, 3, 0, 0.4), (6, 6, 2, 0.5), (8, 2, 1, 0.3)])
def test_enpt2_degenerate_shapes(gpu, n, na, nb, frac):
    torch = gpu
    w = W.random_small(421 + n, "spin_orbitals", n, na, nb, naux=4, frac=frac)
    ev, U = np.linalg.eigh(Oracle.from_workload(w).dense())
    C, E0 = U[:, :1].copy(), ev[:1].copy()
    ref = PT.enpt2("spin_orbitals", n, na, nb, w.ints.h, w.ints.eri(), w.keys, C, E0)
    H = sci.Hamiltonian.from_workload(w)
    e2q = H.enpt2(torch.from_numpy(C).cuda(), E0)[2]
    assert np.allclose(e2q, ref, rtol=1e-10, atol=1e-14), (e2q, ref)


def test_single_determinant_everywhere(gpu):
    torch = gpu
    w = W.random_small(431, "spin_orbitals", 5, 2, 2, naux=4)
    keys = w.keys[:1]
    H = sci.Hamiltonian()
    H.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    H.set_determinants(keys, 2, 2)
    c = torch.ones((1, 1), dtype=torch.float64, device="cuda")
    g1, g2 = H.rdm12(c)
    o = Oracle(w.mode, w.n, w.ints.h, w.ints.eri(), keys)
    r1, r2 = o.rdm12(np.ones(1))
    assert np.abs(g1.cpu().numpy() - r1).max() < 1e-14 and np.abs(g2.cpu().numpy() - r2).max() < 1e-14
    B = sci.Batch([H])
    B.plan(sci.SCI_SCHED_TILE)
    assert abs(float(B.sigma(c.reshape(-1))[0]) - o.diagonal()[0]) < 1e-13
    E0 = [o.diagonal()[0]]
    ref = PT.enpt2("spin_orbitals", 5, 2, 2, w.ints.h, w.ints.eri(), keys, np.ones((1, 1)), E0)
    assert np.allclose(H.enpt2(c, E0)[2], ref, rtol=1e-10)
