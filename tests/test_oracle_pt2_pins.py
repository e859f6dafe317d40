"""Pins of the oracle's ENPT2 (oracle/pt2.py, Eq. ENPT2E).

- Against the dense Hamiltonian of the literal operator route (fock_route): the same
  definition evaluated with H[Q, P] c and H[q, q] from Eq. Hamiltonian applied operator by
  operator, no Slater-Condon closed forms.
- P = the whole space gives E2 = 0 (Q is empty).
- A two-determinant space in closed form: P = {D0} alone, Q = {D1}, E2 = H_10^2 / (H_00 - H_11).
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle import fock_route as F
from oracle import pt2 as PT
from paper_2501_18185_gb300 import workloads as W


@pytest.mark.parametrize("n,na,nb,frac,nroots", [(5, 2, 2, 0.4, 1), (6, 3, 1, 0.5, 2), (5, 3, 2, 0.3, 3)])
def test_enpt2_matches_dense_literal_route(n, na, nb, frac, nroots):
    w = W.random_small(211 + n, "spin_orbitals", n, na, nb, naux=4, frac=frac)
    h, eri = w.ints.h, w.ints.eri()
    P = w.keys
    ev, U = np.linalg.eigh(Oracle("spin_orbitals", n, h, eri, P).dense())
    C, E0 = U[:, :nroots], ev[:nroots]
    full = PT.full_space_keys("spin_orbitals", n, na, nb)
    hs, es = F.spin_orbital_integrals(h, eri)
    H = F.hamiltonian(full, hs, es)
    pos = np.searchsorted(full, P)
    q = np.setdiff1d(np.arange(len(full)), pos)
    num = H[np.ix_(q, pos)] @ C
    ref = (num ** 2 / (E0[None, :] - np.diag(H)[q][:, None])).sum(0)
    got = PT.enpt2("spin_orbitals", n, na, nb, h, eri, P, C, E0)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14)
    assert np.all(got < 0)   # lowest roots: E0 below the external diagonal here


def test_enpt2_full_space_is_zero():
    w = W.random_small(223, "spin_orbitals", 5, 2, 2, naux=4)
    o = Oracle.from_workload(w)
    ev, U = np.linalg.eigh(o.dense())
    assert np.abs(PT.enpt2("spin_orbitals", 5, 2, 2, w.ints.h, w.ints.eri(), w.keys, U[:, :2], ev[:2])).max() == 0.0


def test_enpt2_two_determinant_closed_form():
    """One electron in 2 spinors: the full space is {D0, D1}; with P = {D0} and c = 1,
    E2 = |H_10|^2 / (H_00 - H_11)."""
    rng = np.random.default_rng(5)
    h = np.array([[-1.0, 0.3 + 0.1j], [0.3 - 0.1j, 0.5]])
    L = rng.normal(size=(2, 2, 2)) * 0.1
    L = 0.5 * (L + np.swapaxes(L, 1, 2))
    eri = np.einsum("Ppq,Prs->pqrs", L, L).astype(np.complex128)
    full = PT.full_space_keys("spinors", 2, 1, 0)
    o = Oracle("spinors", 2, h, eri, full)
    H = o.dense()
    P = full[:1]
    E0 = H[0, 0].real
    ref = abs(H[1, 0]) ** 2 / (E0 - H[1, 1].real)
    got = PT.enpt2("spinors", 2, 1, 0, h, eri, P, np.ones((1, 1), dtype=np.complex128), [E0])
    assert abs(got[0] - ref) < 1e-15


@pytest.mark.parametrize("n,ne,frac,nroots", [(6, 2, 0.4, 1), (7, 3, 0.3, 2)])
def test_enpt2_spinors_matches_dense_literal_route(n, ne, frac, nroots):
    """Spinor mode (complex Hermitian h and (pq|rs), no spin conservation): the same
    definition against the dense H of Eq. Hamiltonian applied operator by operator, with
    |H_IJ c_J|^2 summed over the explicit complement Q of P."""
    w = W.random_small(241 + n, "spinors", n, ne, 0, naux=4, frac=frac)
    h, eri = w.ints.h, w.ints.eri()
    P = w.keys
    ev, U = np.linalg.eigh(Oracle("spinors", n, h, eri, P).dense())
    C, E0 = U[:, :nroots], ev[:nroots]
    full = PT.full_space_keys("spinors", n, ne, 0)
    H = F.hamiltonian(full, h, eri)
    pos = np.searchsorted(full, P)
    q = np.setdiff1d(np.arange(len(full)), pos)
    num = H[np.ix_(q, pos)] @ C
    ref = (np.abs(num) ** 2 / (E0[None, :] - np.real(np.diag(H))[q][:, None])).sum(0)
    got = PT.enpt2("spinors", n, ne, 0, h, eri, P, C, E0)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14)
    assert len(q) > 0 and np.all(got < 0)


def _q_connected(full, P, H):
    """Members of the complement Q with at least one nonzero-structure connection into P
    (excitation degree 1 or 2), counted by popcount over the dense key lists."""
    pos = np.searchsorted(full, P)
    q = np.setdiff1d(np.arange(len(full)), pos)
    x = full[q][:, None] ^ P[None, :]
    deg = np.bitwise_count(x) // 2
    return int(((deg >= 1) & (deg <= 2)).any(axis=1).sum())


@pytest.mark.parametrize("mode,n,na,nb,frac,nroots", [
    ("spin_orbitals", 5, 2, 2, 0.4, 1), ("spin_orbitals", 6, 3, 1, 0.5, 2), ("spin_orbitals", 6, 2, 3, 0.15, 3),
    ("spinors", 6, 2, 0, 0.4, 1), ("spinors", 7, 3, 0, 0.3, 2)])
def test_sciref_enpt2_matches_full_space_routes(mode, n, na, nb, frac, nroots):
    """sciref_enpt2 (excitations of P minus P, sorted by key) against the sum of Eq.
    ENPT2E over the whole complement Q of the full space (oracle/pt2.py) and against the
    dense H of the literal operator route; its external count is the number of Q members
    within a double excitation of P, counted by popcount."""
    w = W.random_small(261 + n + 7 * nroots, mode, n, na, nb, naux=4, frac=frac)
    h, eri = w.ints.h, w.ints.eri()
    P = w.keys
    o = Oracle(mode, n, h, eri, P)
    ev, U = np.linalg.eigh(o.dense())
    C, E0 = U[:, :nroots], ev[:nroots]
    got, nx = o.enpt2(C, E0)
    ref = PT.enpt2(mode, n, na, nb, h, eri, P, C, E0)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)
    full = PT.full_space_keys(mode, n, na, nb)
    if mode == "spinors":
        Hd = F.hamiltonian(full, h, eri)
    else:
        Hd = F.hamiltonian(full, *F.spin_orbital_integrals(h, eri))
    pos = np.searchsorted(full, P)
    q = np.setdiff1d(np.arange(len(full)), pos)
    num = Hd[np.ix_(q, pos)] @ C
    lit = (np.abs(num) ** 2 / (E0[None, :] - np.real(np.diag(Hd))[q][:, None])).sum(0)
    assert np.allclose(got, lit, rtol=1e-12, atol=1e-15)
    assert nx == _q_connected(full, P, Hd) and nx > 0


def test_sciref_enpt2_general_vectors_and_energies():
    """Any C and E0 (not eigenpairs), several columns with different E0: each column is the
    one-column sum (no cross-talk between columns) and matches the literal route."""
    w = W.random_small(277, "spin_orbitals", 6, 2, 2, naux=4, frac=0.3, nvec=3)
    h, eri = w.ints.h, w.ints.eri()
    o = Oracle.from_workload(w)
    E0 = np.array([-9.0, -7.5, -12.25])
    got, _ = o.enpt2(w.c, E0)
    for k in range(3):
        one, _ = o.enpt2(w.c[:, k:k + 1], E0[k:k + 1])
        assert one[0] == got[k]
    ref = PT.enpt2("spin_orbitals", 6, 2, 2, h, eri, w.keys, w.c, E0)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-15)


def test_sciref_enpt2_thread_count_does_not_change_the_sum():
    from oracle import set_threads
    w = W.random_small(281, "spinors", 7, 3, 0, naux=4, frac=0.2, nvec=2)
    o = Oracle.from_workload(w)
    E0 = np.array([-30.0, -29.0])
    try:
        set_threads(1)
        a, na_ = o.enpt2(w.c, E0)
    finally:
        set_threads(0)
    b, nb_ = o.enpt2(w.c, E0)
    assert np.array_equal(a, b) and na_ == nb_


@pytest.mark.parametrize("mode,n,na,nb,frac", [("spin_orbitals", 6, 3, 2, 0.3), ("spinors", 8, 3, 0, 0.3)])
def test_sciref_enpt2_screening_matches_masked_literal_route(mode, n, na, nb, frac):
    """With eps > 0 a contribution H_IJ c_J is dropped when |H_IJ| max_k |c_Jk| < eps: the
    same rule applied as a mask to the dense H of the literal operator route.  eps = 0 is
    the exact sum, a huge eps leaves nothing."""
    w = W.random_small(291 + n, mode, n, na, nb, naux=4, frac=frac, nvec=2)
    h, eri = w.ints.h, w.ints.eri()
    o = Oracle.from_workload(w)
    E0 = np.array([-20.0, -18.5])
    full = PT.full_space_keys(mode, n, na, 0 if mode == "spinors" else nb)
    Hd = F.hamiltonian(full, h, eri) if mode == "spinors" else F.hamiltonian(full, *F.spin_orbital_integrals(h, eri))
    pos = np.searchsorted(full, w.keys)
    q = np.setdiff1d(np.arange(len(full)), pos)
    HQP = Hd[np.ix_(q, pos)]
    cmax = np.abs(w.c).max(axis=1)
    for eps in (0.0, 1e-3, 3e-2):
        keep = np.abs(HQP) * cmax[None, :] >= eps if eps > 0 else np.ones(HQP.shape, dtype=bool)
        num = (HQP * keep) @ w.c
        ref = (np.abs(num) ** 2 / (E0[None, :] - np.real(np.diag(Hd))[q][:, None])).sum(0)
        nref = int((keep & (HQP != 0)).any(axis=1).sum()) if eps > 0 else None
        got, nx = o.enpt2(w.c, E0, eps=eps)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15), eps
        if eps > 0:
            assert nx == nref
    got, nx = o.enpt2(w.c, E0, eps=1e9)
    assert nx == 0 and np.all(got == 0)


@pytest.mark.parametrize("mode,n,na,nb,frac", [("spin_orbitals", 6, 3, 2, 0.3), ("spinors", 8, 3, 0, 0.3)])
def test_sciref_enpt2_over_w_is_eq_ew1(mode, n, na, nb, frac):
    """over_w: the sum over W (members of the list included, numerators over the other
    members) against the dense literal route with H's diagonal removed; with eps = 0,
    E2[W] - E2[P] (Eq. EP1 from the literal H) equals E2[Q] (Eq. PT2final)."""
    w = W.random_small(301 + n, mode, n, na, nb, naux=4, frac=frac, nvec=2)
    h, eri = w.ints.h, w.ints.eri()
    o = Oracle.from_workload(w)
    E0 = np.array([-20.0, -18.5])
    full = PT.full_space_keys(mode, n, na, 0 if mode == "spinors" else nb)
    Hd = F.hamiltonian(full, h, eri) if mode == "spinors" else F.hamiltonian(full, *F.spin_orbital_integrals(h, eri))
    pos = np.searchsorted(full, w.keys)
    Hoff = Hd.copy()
    np.fill_diagonal(Hoff, 0)
    HWP = Hoff[:, pos]
    cmax = np.abs(w.c).max(axis=1)
    d = np.real(np.diag(Hd))
    for eps in (0.0, 1e-3):
        keep = np.abs(HWP) * cmax[None, :] >= eps if eps > 0 else np.ones(HWP.shape, dtype=bool)
        num = (HWP * keep) @ w.c
        ref = (np.abs(num) ** 2 / (E0[None, :] - d[:, None])).sum(0)
        got, _ = o.enpt2(w.c, E0, eps=eps, over_w=True)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15), eps
    e2w, _ = o.enpt2(w.c, E0, over_w=True)
    sig = Hd[np.ix_(pos, pos)] @ w.c
    e2p = (np.abs(sig - w.c * d[pos][:, None]) ** 2 / (E0[None, :] - d[pos][:, None])).sum(0)
    e2q, _ = o.enpt2(w.c, E0)
    assert np.allclose(e2w - e2p, e2q, rtol=1e-11, atol=1e-14)
