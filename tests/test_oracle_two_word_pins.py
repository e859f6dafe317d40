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
