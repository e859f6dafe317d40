"""GPU ENPT2 (sci_enpt2: Eqs. PT2final, EW1, EP1) against the oracle's definition over Q.

The GPU sums over the generated space W in hash-table batches and subtracts the P part;
the oracle sums Eq. ENPT2E over the explicit complement Q of P in the full space.  The
two routes share no code.  Tolerance 1e-10 relative: both are FP64 sums of the same terms
in different orders, over up to ~1e5 terms each.
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle import pt2 as PT
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [  # (seed, n, na, nb, frac, nroots)
    (301, 8, 4, 4, 0.35, 1),
    (302, 8, 3, 4, 0.5, 2),
    (303, 9, 3, 2, 0.25, 3),
    (304, 7, 2, 5, 0.6, 1),
    (305, 10, 2, 2, 0.2, 4),
]


def roots_of(w, nroots):
    ev, U = np.linalg.eigh(Oracle.from_workload(w).dense())
    return U[:, :nroots].copy(), ev[:nroots].copy()


@pytest.mark.parametrize("seed,n,na,nb,frac,nroots", CASES)
def test_enpt2_matches_oracle(gpu, seed, n, na, nb, frac, nroots):
    torch = gpu
    w = W.random_small(seed, "spin_orbitals", n, na, nb, naux=6, frac=frac)
    C, E0 = roots_of(w, nroots)
    ref = PT.enpt2("spin_orbitals", n, na, nb, w.ints.h, w.ints.eri(), w.keys, C, E0)
    H = sci.Hamiltonian.from_workload(w)
    Ct = torch.from_numpy(C).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0)
    assert np.allclose(e2q, ref, rtol=1e-10, atol=1e-14), (e2q, ref)
    assert st["batches"] >= 1 and st["distinct_W"] > 0
    # a table of 512 entries: many batches (and restarts when a batch overflows), the
    # same sums
    e2w_b, e2p_b, e2q_b, st_b = H.enpt2(Ct, E0, table_bytes=512 * (8 + 8 * nroots))
    assert st_b["batches"] > st["batches"]
    assert np.allclose(e2q_b, e2q, rtol=1e-12, atol=1e-15) and np.allclose(e2p_b, e2p, rtol=1e-14)
    # E2[P] (Eq. EP1) at exact eigenvectors equals Eq. EP2: sum c^2 (E0 - H_II)
    d = H.diagonal().cpu().numpy()
    ep2 = (C ** 2 * (E0[None, :] - d[:, None])).sum(0)
    assert np.allclose(e2p, ep2, rtol=1e-9, atol=1e-12)


def test_enpt2_screening_and_selected_space(gpu):
    """60k-determinant 30-orbital space (the selected recipe): the sum does not depend on
    the batching, and screening by |H_IJ c_J| < eps moves it by little."""
    torch = gpu
    w = W.selected_30o(M=60000)
    H = sci.Hamiltonian.from_workload(w)
    c = torch.from_numpy(w.c).cuda()
    c = c / torch.linalg.vector_norm(c)
    E0 = [float((c * H.sigma(c)).sum())]
    a = H.enpt2(c, E0, table_bytes=2 << 30)
    b = H.enpt2(c, E0, table_bytes=256 << 20)
    assert b[3]["batches"] > a[3]["batches"]
    assert abs(a[2][0] - b[2][0]) < 1e-12 * abs(a[2][0]) and a[2][0] < 0
    s = H.enpt2(c, E0, eps=1e-7, table_bytes=2 << 30)
    assert s[3]["distinct_W"] < a[3]["distinct_W"] and abs(s[2][0] - a[2][0]) < 1e-3 * abs(a[2][0])


def test_enpt2_errors(gpu):
    torch = gpu
    w = W.random_small(307, "spinors", 8, 3, 0)
    H = sci.Hamiltonian.from_workload(w)
    with pytest.raises(ValueError):     # a complex Hamiltonian takes complex coefficients
        H.enpt2(torch.zeros((w.M, 1), dtype=torch.float64, device="cuda"), [0.0])
    with pytest.raises(sci.SciError):   # nroots > 8
        H.enpt2(torch.zeros((w.M, 9), dtype=torch.complex128, device="cuda"), [0.0] * 9)
    w = W.random_small(308, "spin_orbitals", 6, 2, 2)
    H = sci.Hamiltonian.from_workload(w)
    with pytest.raises(sci.SciError):
        H.enpt2(torch.zeros((w.M, 9), dtype=torch.float64, device="cuda"), [0.0] * 9)


@pytest.fixture(scope="module")
def cut30():
    """A 1,000-determinant space of the 30-orbital recipe (HF, all singles, sampled
    doubles, triples and quadruples), its four lowest roots from the oracle's dense H, the
    oracle's E2 of Eq. ENPT2E summed over the 3e7 external determinants (sciref_enpt2),
    and the number of members of P connected to another member."""
    w = W.selected_30o_cut(1000)
    o = Oracle.from_workload(w)
    ev, U = np.linalg.eigh(o.dense())
    C, E0 = U[:, :4].copy(), ev[:4].copy()
    E2, n_ext = o.enpt2(C, E0)
    n_conn = sum(1 for r in range(w.M) if len(o.connections(r)[0]) > 0)
    return w, C, E0, E2, n_ext, n_conn


@pytest.mark.parametrize("nroots", [1, 4])
def test_enpt2_30_orbital_space_matches_oracle(gpu, cut30, nroots):
    """The GPU paths of the full-size spaces (n = 30: the GF(2) batch code over 30 beta
    orbitals, the beta-beta lookups per (occupied pair, first virtual), the bounded-probe
    hash table, H_II of external determinants by the Fock decomposition) against the
    oracle's direct sum, at 1e-10 relative; the distinct determinants summed by the GPU
    are exactly W = the oracle's external set plus the connected members of P; a table
    of 2^22 entries (several batches of the beta-string code) gives the same sums.  (The
    code batches by beta string, so every alpha excitation of the ~250 members sharing the
    HF beta string falls into one batch: about 1.5e6 distinct determinants, which no
    table below ~2^21 entries holds at any batch count.)"""
    torch = gpu
    w, C, E0, E2, n_ext, n_conn = cut30
    H = sci.Hamiltonian.from_workload(w)
    Ct = torch.from_numpy(C[:, :nroots].copy()).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0[:nroots])
    assert np.allclose(e2q, E2[:nroots], rtol=1e-10, atol=0), (e2q, E2[:nroots])
    assert st["distinct_W"] == n_ext + n_conn
    d = H.diagonal().cpu().numpy()
    ep2 = (C[:, :nroots] ** 2 * (E0[None, :nroots] - d[:, None])).sum(0)
    assert np.allclose(e2p, ep2, rtol=1e-9)
    e2w_b, e2p_b, e2q_b, st_b = H.enpt2(Ct, E0[:nroots], table_bytes=(1 << 22) * (8 + 8 * nroots))
    assert st_b["batches"] >= 8 and st_b["batches"] > st["batches"] and st_b["distinct_W"] == st["distinct_W"]
    assert np.allclose(e2q_b, E2[:nroots], rtol=1e-10, atol=0)


SPINOR_CASES = [  # (seed, n, N, frac, nroots): full spaces of 560 to 1820 determinants
    (321, 14, 4, 0.3, 1),
    (322, 16, 3, 0.2, 2),
    (323, 12, 5, 0.25, 3),
    (324, 16, 4, 0.1, 4),
]


@pytest.mark.parametrize("seed,n,N,frac,nroots", SPINOR_CASES)
def test_enpt2_spinors_matches_oracle(gpu, seed, n, N, frac, nroots):
    """Complex spinor mode (no spin conservation, complex numerators |sum_J H_IJ c_J|^2)
    against the oracle's sum over the explicit complement Q of the full space, at 1e-10;
    a 256-entry table (several batches of the whole-string code, restarts) gives the
    same."""
    torch = gpu
    w = W.random_small(seed, "spinors", n, N, 0, naux=6, frac=frac)
    C, E0 = roots_of(w, nroots)
    ref = PT.enpt2("spinors", n, N, 0, w.ints.h, w.ints.eri(), w.keys, C, E0)
    H = sci.Hamiltonian.from_workload(w)
    Ct = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0)
    assert np.allclose(e2q, ref, rtol=1e-10, atol=1e-14), (e2q, ref)
    e2w_b, e2p_b, e2q_b, st_b = H.enpt2(Ct, E0, table_bytes=256 * (8 + 16 * nroots))
    assert st_b["batches"] > st["batches"]
    assert np.allclose(e2q_b, e2q, rtol=1e-12, atol=1e-15)
    d = H.diagonal().cpu().numpy()
    ep2 = (np.abs(C) ** 2 * (E0[None, :] - d[:, None])).sum(0)
    assert np.allclose(e2p, ep2, rtol=1e-9, atol=1e-12)


@pytest.fixture(scope="module")
def cut64():
    """A 301-determinant space of the 64-spinor recipe (HF, sampled singles, doubles and
    triples), its two lowest roots from the oracle's dense H and the oracle's direct sum
    (sciref_enpt2) over its ~3e7 external determinants."""
    w = W.selected_spinor_64_cut()
    o = Oracle.from_workload(w)
    ev, U = np.linalg.eigh(o.dense())
    C, E0 = U[:, :2].copy(), ev[:2].copy()
    E2, n_ext = o.enpt2(C, E0)
    n_conn = sum(1 for r in range(w.M) if len(o.connections(r)[0]) > 0)
    return w, C, E0, E2, n_ext, n_conn


@pytest.mark.parametrize("nroots", [1, 2])
def test_enpt2_64_spinor_space_matches_oracle(gpu, cut64, nroots):
    """The spinor paths at the full-size shape (64 spinors, 14 electrons: 111,475 doubles
    per determinant, the whole-string batch code, complex tables) against the oracle at
    1e-10, with the distinct count exact; a 2^20-entry table gives the same sums."""
    torch = gpu
    w, C, E0, E2, n_ext, n_conn = cut64
    H = sci.Hamiltonian.from_workload(w)
    Ct = torch.from_numpy(C[:, :nroots].copy()).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0[:nroots])
    assert np.allclose(e2q, E2[:nroots], rtol=1e-10, atol=0), (e2q, E2[:nroots])
    assert st["distinct_W"] == n_ext + n_conn
    e2w_b, e2p_b, e2q_b, st_b = H.enpt2(Ct, E0[:nroots], table_bytes=(1 << 20) * (8 + 16 * nroots))
    assert st_b["batches"] > st["batches"] and st_b["distinct_W"] == st["distinct_W"]
    assert np.allclose(e2q_b, E2[:nroots], rtol=1e-10, atol=0)


@pytest.mark.parametrize("which,eps", [("30o", 1e-6), ("30o", 1e-4), ("64s", 1e-5)])
def test_enpt2_screening_matches_screened_oracle(gpu, which, eps):
    """Screening (eps > 0): the GPU skips whole double-excitation classes by upper bounds
    of their elements (the paper's Table 1 screening) and drops single contributions below
    eps, so its E2[W] is the sum over W with the per-element rule |H_IJ| max_k |c_Jk| < eps
    applied to every contribution (the oracle's over-W sum with that rule, at 1e-10, with
    the same number of distinct determinants), while E2[P] stays exact (Eq. EP1).  The
    screening drops a real share of W."""
    torch = gpu
    w = W.selected_30o_cut(1000) if which == "30o" else W.selected_spinor_64_cut()
    o = Oracle.from_workload(w)
    ev, U = np.linalg.eigh(o.dense())
    C, E0 = U[:, :2].copy(), ev[:2].copy()
    refW, n_w = o.enpt2(C, E0, eps=eps, over_w=True)
    H = sci.Hamiltonian.from_workload(w)
    Ct = torch.from_numpy(C).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0, eps=eps)
    x2w, x2p, x2q, xst = H.enpt2(Ct, E0)
    assert np.allclose(e2w, refW, rtol=1e-10, atol=0), (e2w, refW)
    assert st["distinct_W"] == n_w
    assert np.allclose(e2p, x2p, rtol=1e-13)                                   # E2[P] unscreened
    assert st["distinct_W"] < xst["distinct_W"] and np.all(np.abs(e2q - x2q) < 0.05 * np.abs(x2q))
