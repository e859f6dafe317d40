"""Pins of the oracle on determinants of more than 64 spin-orbitals (two-word keys, the
paper's multi-word occupation strings, Sec. 3.2: orbital configurations as arrays of
64-bit words).  The oracle holds every string as a 128-bit integer; these checks run it on
40 spatial orbitals (80 spin-orbitals), where beta strings cross the word boundary:
closed forms of two-electron spaces (no bit logic on the reference side), the one-body
spectrum, the brute-force all-pairs route, Hermiticity, the alpha<->beta swap symmetry,
and the one-word encoding of the same small space."""
import itertools

import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import workloads as W


def _ints(n, seed, naux=6):
    rng = np.random.default_rng(seed)
    return W.real_integrals(rng, n, naux, 0.95)


def _keys_from_sets(sets, n):
    """[M, 2] words of the determinants given as (alpha orbitals, beta orbitals), sorted."""
    a = np.array([sum(1 << p for p in al) for al, _ in sets], dtype=np.uint64)
    b = np.array([sum(1 << p for p in be) for _, be in sets], dtype=np.uint64)
    return W.sort_words(W.two_word_keys(a, b, n))


def test_two_electron_opposite_spin_closed_form_40_orbitals():
    """One alpha + one beta electron over 40 orbitals (beta bits 40..79 cross the word
    boundary): <p q|H|r s> = h_pr d_qs + d_pr h_qs + (pr|qs), the dense 1600 x 1600
    assembly of the one-word pin, with the list in ascending 128-bit order (q major)."""
    n = 40
    ints = _ints(n, 11)
    h, eri = ints.h, ints.eri()
    keys = _keys_from_sets([((p,), (q,)) for q in range(n) for p in range(n)], n)
    o = Oracle("spin_orbitals", n, h, eri, keys)
    I = np.eye(n)
    V = eri.transpose(2, 0, 3, 1).reshape(n * n, n * n)
    expected = np.kron(I, h) + np.kron(h, I) + V
    H = o.dense()
    assert np.abs(H - expected).max() < 1e-13
    # one-body limit of the same space: with (pq|rs) = 0 the ground energy is twice the
    # lowest eigenvalue of h
    o0 = Oracle("spin_orbitals", n, h, np.zeros_like(eri), keys)
    e0 = np.linalg.eigvalsh(o0.dense())[0]
    assert abs(e0 - 2 * np.linalg.eigvalsh(h)[0]) < 1e-12


def test_two_electron_same_spin_closed_form_beta_40_orbitals():
    """Two beta electrons over 40 orbitals (bits 40..79): <pq|H|rs> = h_pr d_qs + h_qs d_pr
    - h_ps d_qr - h_qr d_ps + (pr|qs) - (ps|qr) for p<q, r<s, with the phases of strings
    that straddle the word boundary."""
    n = 40
    ints = _ints(n, 12)
    h, eri = ints.h, ints.eri()
    pairs = [(p, q) for q in range(n) for p in range(q)]
    keys = _keys_from_sets([((), (p, q)) for p, q in pairs], n)
    o = Oracle("spin_orbitals", n, h, eri, keys)
    d = lambda a, b: 1.0 if a == b else 0.0  # noqa: E731
    E = np.zeros((len(pairs), len(pairs)))
    for x, (p, q) in enumerate(pairs):
        for y, (r, s) in enumerate(pairs):
            E[x, y] = (h[p, r] * d(q, s) + h[q, s] * d(p, r) - h[p, s] * d(q, r) - h[q, r] * d(p, s)
                       + eri[p, r, q, s] - eri[p, s, q, r])
    assert np.abs(o.dense() - E).max() < 1e-13


def test_two_word_selected_space_brute_force_and_hermiticity():
    """The selected 40-orbital space (3+3 electrons): sigma by generation + lookup equals the
    all-pairs route on sampled rows, and <x, H y> = <H x, y>."""
    w = W.selected_two_word(n=40, na=3, nb=3, M=17000)
    o = Oracle.from_workload(w)
    rows = np.unique(np.random.default_rng(1).choice(w.M, 300, replace=False))
    assert np.abs(o.sigma_rows(rows, w.c) - o.sigma_brute_rows(rows, w.c)).max() < 1e-13
    rng = np.random.default_rng(2)
    x, y = rng.normal(size=w.M), rng.normal(size=w.M)
    Hx, Hy = o.sigma(x)[:, 0], o.sigma(y)[:, 0]
    assert abs(x @ Hy - Hx @ y) < 1e-12 * abs(x @ Hy)


def test_two_word_alpha_beta_swap_symmetry():
    """On a swap-closed 40-orbital space the spin swap maps sigma to itself (the reordering
    sign (-1)^(na nb) is common to all determinants)."""
    n, ne = 40, 2
    rng = np.random.default_rng(7)
    occ = lambda: tuple(sorted(rng.choice(8, ne, replace=False)))  # noqa: E731
    sets = {(occ(), occ()) for _ in range(300)}
    sets |= {(b, a) for a, b in sets}
    sets = sorted(sets)
    keys = _keys_from_sets(sets, n)
    ints = _ints(n, 13)
    o = Oracle("spin_orbitals", n, ints.h, ints.eri(), keys)
    swapped = _keys_from_sets([(b, a) for a, b in sets], n)
    # permutation: position of the swap of each key
    def as_int(k):
        return int(k[0]) | (int(k[1]) << 64)
    index = {as_int(k): i for i, k in enumerate(keys)}
    key_of = {}
    for (a, b) in sets:
        ka = _keys_from_sets([(a, b)], n)[0]
        kb = _keys_from_sets([(b, a)], n)[0]
        key_of[as_int(ka)] = as_int(kb)
    perm = np.array([index[key_of[as_int(k)]] for k in keys])
    assert sorted(perm.tolist()) == list(range(len(keys)))
    c = rng.normal(size=(len(keys), 2))
    pc = np.empty_like(c)
    pc[perm] = c
    s, ps = o.sigma(c), o.sigma(pc)
    assert np.abs(ps[perm] - s).max() < 1e-12 * np.abs(s).max()
    assert len(swapped) == len(keys)


def test_two_word_encoding_of_a_one_word_space():
    """A space of at most 64 spin-orbitals encoded as two words (high word 0) gives the
    same dense H as its one-word encoding."""
    w = W.random_small(31, "spin_orbitals", 6, 3, 2, naux=4, frac=0.5)
    k2 = np.stack([w.keys, np.zeros_like(w.keys)], axis=1)
    h, eri = w.ints.h, w.ints.eri()
    assert np.array_equal(Oracle("spin_orbitals", 6, h, eri, w.keys).dense(),
                          Oracle("spin_orbitals", 6, h, eri, k2).dense())


def _small_two_word_space(n, na, nb, keep, seed):
    """HF plus a random fraction `keep` of the other determinants of na + nb electrons over
    n orbitals (two-word keys when n > 32)."""
    rng = np.random.default_rng(seed)
    al = list(itertools.combinations(range(n), na))
    be = list(itertools.combinations(range(n), nb))
    sets = [(a, b) for a in al for b in be if (a == tuple(range(na)) and b == tuple(range(nb))) or rng.random() < keep]
    return sets


def test_rdm12_two_words_energy_traces_and_symmetries():
    """The oracle's density matrices on 40 orbitals (2 alpha + 1 beta electrons, beta bits
    40..79 across the word boundary): sum h g1 + 1/2 sum (pq|rs) g2 = c^+ H c with the
    oracle's sigma (pinned above by the closed forms), traces N and N(N - 1), Hermiticity and
    electron exchange."""
    from oracle import fock_route as F

    n, na, nb = 40, 2, 1
    ints = _ints(n, 37)
    keys = _keys_from_sets(_small_two_word_space(n, na, nb, 0.04, 5), n)
    o = Oracle("spin_orbitals", n, ints.h, ints.eri(), keys)
    c = np.random.default_rng(6).standard_normal(len(keys))
    c /= np.linalg.norm(c)
    g1, g2 = o.rdm12(c)
    hs, es = F.spin_orbital_integrals(ints.h, ints.eri())
    E = np.einsum("pq,pq->", hs, g1) + 0.5 * np.einsum("pqrs,pqrs->", es, g2)
    assert abs(E - np.vdot(c, o.sigma(c)[:, 0])) < 1e-11 * max(1.0, abs(E))
    N = na + nb
    assert abs(np.trace(g1) - N) < 1e-12 and abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-11
    assert np.abs(g1 - g1.T).max() < 1e-14
    assert np.abs(g2 - g2.transpose(2, 3, 0, 1)).max() < 1e-14
    assert np.abs(g2 - g2.transpose(1, 0, 3, 2)).max() < 1e-14
    assert len(keys) > 1000


def test_rdm12_two_word_encoding_of_a_one_word_space():
    """A space of 24 spin-orbitals given as two words (high word 0) has the density matrices
    of its one-word encoding (bit for bit on one thread), which the literal operator route
    pins."""
    w = W.random_small(107, "spin_orbitals", 12, 3, 2, naux=4, frac=0.3)
    c = w.c[:, 0]
    o1 = Oracle.from_workload(w)
    o2 = Oracle(w.mode, w.n, w.ints.h, w.ints.eri(), np.stack([w.keys, np.zeros_like(w.keys)], axis=1))
    import oracle

    oracle.set_threads(1)          # one thread: the same summation order, so equal bits
    try:
        a1, a2 = o1.rdm12(c)
        b1, b2 = o2.rdm12(c)
    finally:
        oracle.set_threads(0)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)


def test_enpt2_two_words_against_the_definition_on_the_full_space():
    """ENPT2 of a P inside the full 1 + 1-electron space of 40 orbitals (1,600 determinants,
    beta bits 40..79 across the word boundary): sciref_enpt2 (generation of the excitations
    of P, deduplication by key) against Eq. ENPT2E written out on the dense H of the whole
    space (the oracle's sigma, pinned above by the closed form), two roots with arbitrary
    E0; the external count against the size of Q."""
    n = 40
    ints = _ints(n, 53)
    full = _keys_from_sets([((p,), (q,)) for p in range(n) for q in range(n)], n)
    of = Oracle("spin_orbitals", n, ints.h, ints.eri(), full)
    Hf = of.dense()
    rng = np.random.default_rng(8)
    inP = rng.random(len(full)) < 0.3
    inP[0] = True
    P = full[inP]
    C = rng.standard_normal((len(P), 2))
    E0 = np.array([-30.0, -25.0])
    v = Hf[:, inP] @ C                       # sum_J H_IJ c_J for every I of the space
    d = np.diag(Hf)
    Q = ~inP
    ref = ((v[Q] ** 2) / (E0[None, :] - d[Q, None])).sum(axis=0)
    op = Oracle("spin_orbitals", n, ints.h, ints.eri(), P)
    E2, nx = op.enpt2(C, E0)
    assert np.allclose(E2, ref, rtol=1e-12, atol=0)
    assert nx == int(Q.sum())              # every determinant of Q is one excitation of P


def test_enpt2_two_word_encoding_of_a_one_word_space():
    """A space of 24 spin-orbitals given as two words gives the one-word ENPT2."""
    w = W.random_small(109, "spin_orbitals", 12, 3, 2, naux=4, frac=0.2, nvec=2)
    o1 = Oracle.from_workload(w)
    o2 = Oracle(w.mode, w.n, w.ints.h, w.ints.eri(), np.stack([w.keys, np.zeros_like(w.keys)], axis=1))
    E0 = np.array([-20.0, -18.0])
    a, na_ = o1.enpt2(w.c, E0)
    b, nb_ = o2.enpt2(w.c, E0)
    assert na_ == nb_ and np.allclose(a, b, rtol=1e-13, atol=0)
