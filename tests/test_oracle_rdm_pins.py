"""Pins of the oracle's density matrices (oracle.Oracle.rdm12).

g1[p,q] = <c|a+_p a_q|c>, g2[p,q,r,s] = <c|a+_p a+_r a_s a_q|c> over spin-orbitals.
They are pinned against:
- the literal operator route (oracle/fock_route.rdm12);
- the energy identity sum h g1 + 1/2 sum (pq|rs) g2 = c^+ H c, with H pinned separately;
- traces and permutation symmetries;
- the Hellmann-Feynman derivative dE/dh of an eigenvalue.

Together these fix the RDM index convention that the gradient semantics rely on.
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle import fock_route as F
from paper_2501_18185_gb300 import workloads as W

CASES = [("spin_orbitals", 4, 2, 1, 1.0), ("spin_orbitals", 5, 2, 2, 0.6), ("spinors", 6, 3, 0, 1.0),
         ("spinors", 7, 3, 0, 0.5)]


def _so(w):
    if w.mode == "spin_orbitals":
        return F.spin_orbital_integrals(w.ints.h, w.ints.eri())
    return w.ints.h, w.ints.eri()


@pytest.mark.parametrize("mode,n,na,nb,frac", CASES)
def test_rdm_matches_literal_route(mode, n, na, nb, frac):
    w = W.random_small(101, mode, n, na, nb, naux=4, frac=frac)
    c = w.c[:, 0]
    g1, g2 = Oracle.from_workload(w).rdm12(c)
    norb = n if mode == "spinors" else 2 * n
    l1, l2 = F.rdm12(w.keys, c, norb)
    assert np.abs(g1 - l1).max() < 1e-13 and np.abs(g2 - l2).max() < 1e-13


@pytest.mark.parametrize("mode,n,na,nb,frac", CASES + [("spin_orbitals", 8, 4, 4, 1.0)])
def test_rdm_energy_traces_symmetries(mode, n, na, nb, frac):
    w = W.random_small(103, mode, n, na, nb, naux=4, frac=frac)
    o = Oracle.from_workload(w)
    c = w.c[:, 0]
    g1, g2 = o.rdm12(c)
    hs, es = _so(w)
    E = np.einsum("pq,pq->", hs, g1) + 0.5 * np.einsum("pqrs,pqrs->", es, g2)
    assert abs(E - np.vdot(c, o.sigma(c)[:, 0])) < 1e-12
    N = na + (nb if mode == "spin_orbitals" else 0)
    assert abs(np.trace(g1) - N) < 1e-12 and abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-11
    assert np.abs(g1 - g1.conj().T).max() < 1e-14
    assert np.abs(g2 - g2.transpose(2, 3, 0, 1)).max() < 1e-14               # electron exchange
    assert np.abs(g2 - g2.transpose(1, 0, 3, 2).conj()).max() < 1e-14        # Hermiticity


def test_hellmann_feynman_one_body():
    """For an eigenvector, dE/dh_pq (h_pq and h_qp moved together) = g1_pq + g1_qp,
    checked by central differences (step 1e-5) on the dense FCI spectrum."""
    w = W.random_small(107, "spin_orbitals", 5, 2, 2, naux=4)
    h, eri = w.ints.h, w.ints.eri()
    o = Oracle("spin_orbitals", 5, h, eri, w.keys)
    ev, U = np.linalg.eigh(o.dense())
    g1, g2 = o.rdm12(U[:, 0])
    g1s = g1[:5, :5] + g1[5:, 5:]                     # spin-summed
    step = 1e-5
    for p, q in [(0, 0), (1, 3), (4, 2), (2, 2)]:
        d = np.zeros((5, 5))
        d[p, q] += 1.0
        d[q, p] += 1.0 if p != q else 0.0
        ep = np.linalg.eigvalsh(Oracle("spin_orbitals", 5, h + step * d, eri, w.keys).dense())[0]
        em = np.linalg.eigvalsh(Oracle("spin_orbitals", 5, h - step * d, eri, w.keys).dense())[0]
        fd = (ep - em) / (2 * step)
        an = g1s[p, q] + (g1s[q, p] if p != q else 0.0)
        assert abs(fd - an) < 1e-7, (p, q, fd, an)


def test_hellmann_feynman_two_body():
    """For an eigenvector, moving a whole permutation orbit of (pq|rs) by eta changes the
    eigenvalue by eta * 1/2 * sum over the orbit's distinct index tuples of the
    spin-summed Gamma[p,q,r,s] = sum_{s1,s2} g2[p s1, q s1, r s2, s s2]: the factor 1/2 of
    the gradient dE/d(pq|rs) = Gamma / 2 (central differences, step 1e-5)."""
    n = 4
    w = W.random_small(109, "spin_orbitals", n, 2, 1, naux=4)
    h, eri = w.ints.h, w.ints.eri()
    o = Oracle("spin_orbitals", n, h, eri, w.keys)
    ev, U = np.linalg.eigh(o.dense())
    _, g2 = o.rdm12(U[:, 0])
    G = sum(g2[a * n:(a + 1) * n, a * n:(a + 1) * n, b * n:(b + 1) * n, b * n:(b + 1) * n]
            for a in (0, 1) for b in (0, 1))
    step = 1e-5
    for p, q, r, s in [(0, 1, 2, 3), (1, 1, 0, 0), (2, 0, 2, 0), (3, 3, 3, 3), (0, 2, 1, 1)]:
        orbit = {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                 (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}
        d = np.zeros_like(eri)
        for t in orbit:
            d[t] = 1.0
        ep = np.linalg.eigvalsh(Oracle("spin_orbitals", n, h, eri + step * d, w.keys).dense())[0]
        em = np.linalg.eigvalsh(Oracle("spin_orbitals", n, h, eri - step * d, w.keys).dense())[0]
        fd = (ep - em) / (2 * step)
        an = 0.5 * sum(G[t] for t in orbit)
        assert abs(fd - an) < 1e-7, ((p, q, r, s), fd, an)
