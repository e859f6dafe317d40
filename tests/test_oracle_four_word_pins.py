"""Pins of the oracle on determinants of more than 192 spin-orbitals (four-word keys, the
paper's occupation strings as arrays of 64-bit words, Sec. 3.2).  On 100 spatial orbitals
(200 spin-orbitals) the alpha string crosses words 0/1 and the beta string words 1, 2 and
3: the same-spin two-electron closed form (no bit logic on the reference side), the
brute-force all-pairs route on a selected space, and the four-word encoding of a
three-word space."""
import numpy as np

from oracle import Oracle
from paper_2501_18185_gb300 import workloads as W


def _as_int(k):
    return sum(int(w) << (64 * i) for i, w in enumerate(k))


def test_two_electron_same_spin_closed_form_beta_100_orbitals():
    """Two beta electrons over 100 orbitals (bits 100..199 over words 1, 2 and 3):
    <pq|H|rs> = h_pr d_qs + h_qs d_pr - h_ps d_qr - h_qr d_ps + (pr|qs) - (ps|qr) for p<q,
    r<s, with the phases of strings that straddle the boundaries at bits 128 and 192; as
    H X on a random block, over 1,500 of the 4,950 pairs (the closed form restricted to the
    list: coefficients outside it are zero)."""
    n = 100
    ints = W.real_integrals(np.random.default_rng(111), n, 3, 0.95)
    h, eri = ints.h, ints.eri()
    allp = np.array([(p, q) for q in range(n) for p in range(q)])
    pairs = allp[np.sort(np.random.default_rng(115).choice(len(allp), 1500, replace=False))]
    keys = W.words_from_occ(pairs + n, 4)
    assert [_as_int(k) for k in keys] == sorted(_as_int(k) for k in keys)
    assert (keys[:, 3] != 0).any() and (keys[:, 1] != 0).any()
    o = Oracle("spin_orbitals", n, h, eri, keys)
    p, q = pairs[:, 0], pairs[:, 1]
    r, s = p, q
    d = lambda a, b: (a[:, None] == b[None, :]).astype(float)  # noqa: E731
    E = (h[p][:, r] * d(q, s) + h[q][:, s] * d(p, r) - h[p][:, s] * d(q, r) - h[q][:, r] * d(p, s)
         + eri[p[:, None], r[None, :], q[:, None], s[None, :]] - eri[p[:, None], s[None, :], q[:, None], r[None, :]])
    X = np.random.default_rng(112).standard_normal((len(pairs), 2))
    assert np.abs(o.sigma(X) - E @ X).max() < 1e-12 * np.abs(E @ X).max()


def test_four_word_selected_space_brute_force_and_hermiticity():
    """A selected 100-orbital space (2 + 2 electrons, HF + singles + doubles + triples, 60,000
    determinants): sigma by generation + lookup equals the all-pairs route on sampled rows,
    and <x, H y> = <H x, y> on a cut of the list."""
    w = W.selected_words(100, 2, 2, 60000, 4, naux=6)
    o = Oracle.from_workload(w)
    rows = np.unique(np.random.default_rng(113).choice(w.M, 40, replace=False))
    assert np.abs(o.sigma_rows(rows, w.c) - o.sigma_brute_rows(rows, w.c)).max() < 1e-13
    cut = Oracle(w.mode, w.n, w.ints.h, w.ints.eri(), w.keys[:2000])
    rng = np.random.default_rng(114)
    x, y = rng.normal(size=2000), rng.normal(size=2000)
    Hx, Hy = cut.sigma(x)[:, 0], cut.sigma(y)[:, 0]
    assert abs(x @ Hy - Hx @ y) < 1e-12 * abs(x @ Hy)


def test_four_word_encoding_of_a_three_word_space():
    """A 70-orbital three-word space given as four words (top word 0) gives the sigma of
    its three-word encoding bit for bit."""
    w = W.selected_three_word(n=70, na=2, nb=1, M=12000, naux=6)
    k4 = np.concatenate([w.keys, np.zeros((w.M, 1), dtype=np.uint64)], axis=1)
    rows = np.arange(0, w.M, 11)
    h, eri = w.ints.h, w.ints.eri()
    a = Oracle("spin_orbitals", 70, h, eri, w.keys).sigma_rows(rows, w.c)
    b = Oracle("spin_orbitals", 70, h, eri, k4).sigma_rows(rows, w.c)
    assert np.array_equal(a, b)
