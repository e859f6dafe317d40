"""Determinants of more than 192 spin-orbitals (four-word keys, sci_set_determinants_w with
nwords = 4) against the oracle and against closed forms.

A selected 100-orbital space (200 spin-orbitals: the alpha string crosses words 0/1, the
beta string words 1, 2 and 3): connections, degrees and phases bit-exact, per-row pair
counts exact, the diagonal, sigma in every precision, the deterministic mode and row
ranges.  A three-word space given as four words.  One- and two-electron spaces of 200
complex spinors against the closed forms; the density matrices of a 200 spin-orbital
space by the energy identity; ENPT2 (at most three words) refused.
"""
import numpy as np
import pytest

from closed_forms import spinor_pair_sigma
from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def sel4w():
    w = W.selected_words(100, 2, 2, 60000, 4, naux=8, nvec=2)
    return w, Oracle.from_workload(w)


def test_four_word_connections_sigma_and_deterministic(gpu, sel4w):
    torch = gpu
    w, o = sel4w
    assert (w.keys[:, 3] != 0).any()
    H = sci.Hamiltonian.from_workload(w)
    rows = np.unique(np.concatenate([np.random.default_rng(0).choice(w.M, 300, replace=False), [0, w.M - 1]]))
    for r in rows[:40]:
        J, deg, ph = o.connections(int(r))
        got = H.connections(int(r), int(r) + 1)
        assert np.array_equal(got[1], J) and np.array_equal(got[2], deg) and np.array_equal(got[3], ph), r
    cost = H.row_costs().cpu().numpy()
    for r in rows:
        assert cost[r] == len(o.connections(int(r))[0])
    assert int(cost.sum()) == H.count_pairs()
    d = H.diagonal().cpu().numpy()
    assert np.abs(d - o.diagonal()).max() < 1e-12 * np.abs(d).max()
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    ref = o.sigma_rows(rows, w.c)
    S = H.sigma(C).cpu().numpy()
    assert _rel(S[rows], ref) < TOL
    assert _rel(H.sigma(C, prec=sci.SCI_PREC_F64_DS).cpu().numpy()[rows], ref) < TOL
    C32 = np.ascontiguousarray(w.c, dtype=np.float32)
    S32 = H.sigma(torch.from_numpy(C32).cuda(), prec=sci.SCI_PREC_F32_STORE_F64_ACC).cpu().numpy()
    ref32 = o.sigma_rows(rows, C32.astype(np.float64))
    A = o.sigma_abs_rows(rows, C32.astype(np.float64))
    assert (np.abs(S32[rows] - ref32) <= 1.05 * 2.0 ** -24 * A + 1e-300).all()
    H.set_deterministic(2)
    a, b = H.sigma(C).cpu().numpy(), H.sigma(C).cpu().numpy()
    assert np.array_equal(a, b) and _rel(a, S) < 1e-13
    H.sync_status()


def test_four_word_row_ranges(gpu, sel4w):
    """K = 3 cost-balanced ranges over 32-byte spectator strings concatenate to the
    whole-list sigma, rows outside each range untouched."""
    from paper_2501_18185_gb300.partition import balanced_ranges, row_weights
    torch = gpu
    w, _ = sel4w
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    full = H.sigma(C).cpu().numpy()
    S = np.zeros_like(full)
    pairs = 0
    for b, e in balanced_ranges(row_weights(H.row_costs().cpu().numpy(), 6), 3):
        H.set_row_range(b, e)
        St = torch.full(C.shape, 7.0, dtype=torch.float64, device="cuda")
        H.sigma(C, out=St)
        Sn = St.cpu().numpy()
        assert (Sn[:b] == 7.0).all() and (Sn[e:] == 7.0).all()
        S[b:e] = Sn[b:e]
        pairs += H.info()["pairs"]
    H.set_row_range(0, w.M)
    assert _rel(S, full) < 1e-12 and pairs == H.count_pairs()
    H.sync_status()


def test_four_word_encoding_of_a_three_word_space(gpu):
    torch = gpu
    w = W.selected_three_word(n=70, na=3, nb=3, M=60000)
    H3 = sci.Hamiltonian.from_workload(w)
    H4 = sci.Hamiltonian()
    H4.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    H4.set_determinants(np.concatenate([w.keys, np.zeros((w.M, 1), dtype=np.uint64)], axis=1), 3, 3)
    C = torch.from_numpy(w.c).cuda()
    assert H4.count_pairs() == H3.count_pairs()
    assert _rel(H4.sigma(C).cpu().numpy(), H3.sigma(C).cpu().numpy()) < 1e-14
    H4.sync_status()


def test_four_word_spinors_one_and_two_electrons(gpu):
    """200 complex spinors (bits 0..199 over four words): one electron, sigma = h c; two
    electrons on 4,000 random pairs against the closed form with the Cholesky factors."""
    torch = gpu
    n = 200
    ints = W.complex_integrals(np.random.default_rng(121), n, 4, 0.9)
    rng = np.random.default_rng(122)
    H = sci.Hamiltonian()
    H.set_integrals("spinors", ints.h, chol=ints.chol)
    H.set_determinants(W.words_from_occ(np.arange(n)[:, None], 4), 1, -1)
    c1 = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    assert _rel(H.sigma(torch.from_numpy(c1).cuda()).cpu().numpy(), ints.h @ c1) < 1e-13
    allp = np.array([(p, q) for q in range(n) for p in range(q)])
    pairs = allp[np.sort(rng.choice(len(allp), 4000, replace=False))]
    keys = W.words_from_occ(pairs, 4)
    assert np.array_equal(W.sort_words(keys), keys) and (keys[:, 3] != 0).any()
    H.set_determinants(keys, 2, -1)
    c2 = rng.standard_normal((len(pairs), 2)) + 1j * rng.standard_normal((len(pairs), 2))
    ref2 = spinor_pair_sigma(ints.h, ints.chol, pairs, c2)
    C2 = torch.from_numpy(c2).cuda()
    assert _rel(H.sigma(C2).cpu().numpy(), ref2) < TOL
    assert _rel(H.sigma(C2, prec=sci.SCI_PREC_F64_DS).cpu().numpy(), ref2) < TOL
    H.sync_status()


def test_four_word_rdm12_energy_identity_200_spin_orbitals(gpu):
    """100 orbitals, 1 + 1 electrons, HF and 600 random determinants (bits in all four
    words): on the device, sum h g1 + 1/2 sum (pq|rs) g2 = c^+ H c against sigma, the traces
    N and N(N - 1), Hermiticity of g1."""
    torch = gpu
    n = 100
    ints = W.real_integrals(np.random.default_rng(123), n, 4, 0.95)
    rng = np.random.default_rng(124)
    occ = {(0, n)}
    while len(occ) < 601:
        occ.add((int(rng.integers(n)), n + int(rng.integers(n))))
    keys = W.sort_words(W.words_from_occ(np.array(sorted(occ)), 4))
    assert (keys[:, 3] != 0).any()
    H = sci.Hamiltonian()
    H.set_integrals("spin_orbitals", ints.h, chol=ints.chol)
    H.set_determinants(keys, 1, 1)
    c = torch.from_numpy(rng.standard_normal(len(keys))).cuda()
    c = c / torch.linalg.vector_norm(c)
    g1, g2 = H.rdm12(c.reshape(-1, 1))
    h = torch.from_numpy(ints.h).cuda()
    L = torch.from_numpy(ints.chol).cuda()
    eri = torch.einsum("Ppq,Prs->pqrs", L, L)
    E1 = (h * g1[:n, :n]).sum() + (h * g1[n:, n:]).sum()
    G = g2.reshape(2, n, 2, n, 2, n, 2, n)
    E2 = sum((eri * G[a, :, a, :, b, :, b, :]).sum() for a in range(2) for b in range(2))
    E = float(E1 + 0.5 * E2)
    ref = float((c * H.sigma(c)).sum())
    assert abs(E - ref) < 1e-11 * max(1.0, abs(ref))
    assert abs(float(torch.trace(g1)) - 2) < 1e-12
    assert abs(float(torch.einsum("pprr->", g2)) - 2) < 1e-10
    assert float((g1 - g1.T).abs().max()) < 1e-14
    H.sync_status()


def test_four_word_limits(gpu, sel4w):
    """ENPT2 takes at most three words; 129 orbitals and 257 spinors are refused."""
    torch = gpu
    w, _ = sel4w
    H = sci.Hamiltonian.from_workload(w)
    with pytest.raises(sci.SciError):
        H.enpt2(torch.from_numpy(np.ascontiguousarray(w.c[:, :1])).cuda(), [-10.0])
    H2 = sci.Hamiltonian()
    with pytest.raises(sci.SciError):
        ints = W.real_integrals(np.random.default_rng(5), 129, 2, 0.95)
        H2.set_integrals("spin_orbitals", ints.h, chol=ints.chol)
    with pytest.raises(sci.SciError):
        ints = W.complex_integrals(np.random.default_rng(6), 257, 2, 0.95)
        H2.set_integrals("spinors", ints.h, chol=ints.chol)
    H.sync_status()
