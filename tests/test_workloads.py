"""Seeded input generators: determinism, shapes, level counts and input symmetries."""
import hashlib
from math import comb

import numpy as np

from paper_2501_18185_gb300 import workloads as W


def _h(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_deterministic():
    a, b = W.selected_30o(M=70000), W.selected_30o(M=70000)
    assert _h(a.keys) == _h(b.keys) and _h(a.c) == _h(b.c) and _h(a.ints.chol) == _h(b.ints.chol)
    s1, s2 = W.selected_spinor_64(M=120000), W.selected_spinor_64(M=120000)
    assert _h(s1.keys) == _h(s2.keys) and _h(s1.c) == _h(s2.c)


def test_selected_30o_structure():
    w = W.selected_30o(M=70000)
    assert np.all(w.keys[1:] > w.keys[:-1])
    lv = W.excitation_level(w.keys, w.hf_key())
    n1 = 2 * 10 * 20
    n2 = 2 * comb(10, 2) * comb(20, 2) + (10 * 20) ** 2
    assert (lv == 0).sum() == 1 and (lv == 1).sum() == n1 and (lv == 2).sum() == n2
    rest = 70000 - 1 - n1 - n2
    assert (lv == 3).sum() == (rest + 1) // 2 and (lv == 4).sum() == rest // 2
    a = w.keys & np.uint64((1 << 30) - 1)
    b = w.keys >> np.uint64(30)
    assert np.all(np.bitwise_count(a) == 10) and np.all(np.bitwise_count(b) == 10)
    # |c| = exp(-level), normalised
    mag = np.abs(w.c[:, 0])
    r = mag * np.exp(lv)
    assert np.allclose(r, r[0]) and abs(np.linalg.norm(w.c) - 1) < 1e-12


def test_selected_spinor_structure():
    w = W.selected_spinor_64(M=120000)
    assert np.all(w.keys[1:] > w.keys[:-1])
    assert np.all(np.bitwise_count(w.keys) == 14)
    lv = W.excitation_level(w.keys, w.hf_key())
    assert (lv == 1).sum() == 14 * 50 and (lv == 2).sum() == comb(14, 2) * comb(50, 2)
    assert (lv == 3).sum() == 120000 - 1 - 700 - comb(14, 2) * comb(50, 2)


def test_integral_symmetries():
    r = W.fci_small_8o().ints
    e = r.eri()
    assert np.allclose(r.h, r.h.T) and np.allclose(e, e.transpose(2, 3, 0, 1)) and np.allclose(e, e.transpose(1, 0, 3, 2))
    c = W.random_small(1, "spinors", 6, 3, 0).ints
    e = c.eri()
    assert np.allclose(c.h, c.h.conj().T)
    assert np.allclose(e, e.transpose(2, 3, 0, 1)) and np.allclose(e, e.transpose(1, 0, 3, 2).conj())


def test_cholesky_decay():
    w = W.selected_30o(M=58000)
    norms = np.linalg.norm(w.ints.chol.reshape(120, -1), axis=1)
    assert np.allclose(norms, 0.3 * 30 * 0.95 ** np.arange(120))


def _as_ints(keys):
    return [sum(int(w) << (64 * i) for i, w in enumerate(k)) for k in keys]


def test_words_from_occ_against_python_integers():
    rng = np.random.default_rng(4)
    occ = np.sort(rng.choice(192, (50, 7)), axis=1)
    words = W.words_from_occ(occ, 3)
    assert _as_ints(words) == [sum(1 << int(o) for o in set(row)) for row in occ]
    assert _as_ints(W.sort_words(words)) == sorted(_as_ints(words))


def test_selected_three_word_structure():
    """HF, every single and Sz-conserving double, random triples; ascending, unique,
    3 + 3 electrons in the right spin halves."""
    n, na, nb, M = 70, 3, 3, 60000
    w = W.selected_three_word(n=n, na=na, nb=nb, M=M)
    ints = _as_ints(w.keys)
    assert ints == sorted(set(ints)) and len(ints) == M
    amask, bmask = (1 << n) - 1, ((1 << n) - 1) << n
    assert all(bin(x & amask).count("1") == na and bin(x & bmask).count("1") == nb for x in ints[::97])
    lv = W.excitation_level_words(w.keys, w.meta["hf_words"])
    singles = na * (n - na) + nb * (n - nb)
    doubles = comb(na, 2) * comb(n - na, 2) + comb(nb, 2) * comb(n - nb, 2) + na * (n - na) * nb * (n - nb)
    assert (lv == 0).sum() == 1 and (lv == 1).sum() == singles and (lv == 2).sum() == doubles
    assert (lv == 3).sum() == M - 1 - singles - doubles


def test_selected_spinor_words_structure():
    n, N, M = 136, 6, 130000
    w = W.selected_spinor_words(n=n, N=N, M=M, naux=4)
    ints = _as_ints(w.keys)
    assert ints == sorted(set(ints)) and len(ints) == M
    assert np.all(np.bitwise_count(w.keys).sum(axis=1) == N)
    lv = W.excitation_level_words(w.keys, w.meta["hf_words"])
    assert (lv == 1).sum() == N * (n - N) and (lv == 2).sum() == comb(N, 2) * comb(n - N, 2)
    assert (lv == 3).sum() == M - 1 - N * (n - N) - comb(N, 2) * comb(n - N, 2)
    assert np.isclose(np.linalg.norm(w.c), 1.0)


def test_selected_words_four_words():
    """The general generator at four words: 100 orbitals (beta bits 100..199 over words 1-3),
    ascending unique keys, 2 + 2 electrons, the level counts of the recipe."""
    n, na, nb, M = 100, 2, 2, 50000
    w = W.selected_words(n, na, nb, M, 4, naux=4)
    ints = _as_ints(w.keys)
    assert ints == sorted(set(ints)) and len(ints) == M
    assert (w.keys[:, 3] != 0).any()
    lv = W.excitation_level_words(w.keys, w.meta["hf_words"])
    singles = na * (n - na) + nb * (n - nb)
    doubles = comb(na, 2) * comb(n - na, 2) + comb(nb, 2) * comb(n - nb, 2) + na * (n - na) * nb * (n - nb)
    assert (lv == 1).sum() == singles and (lv == 2).sum() == doubles and (lv == 3).sum() == M - 1 - singles - doubles
