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
