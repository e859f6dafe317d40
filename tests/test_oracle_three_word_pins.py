"""Pins of the oracle on determinants of more than 128 spin-orbitals (three-word keys, the
paper's occupation strings as arrays of 64-bit words, Sec. 3.2).  On 70 spatial orbitals
(140 spin-orbitals) the alpha string crosses words 0/1 and the beta string words 1/2:
closed forms of two-electron spaces (no bit logic on the reference side), the brute-force
all-pairs route and Hermiticity on a selected space, and the three-word encodings of a
one-word and of a two-word space."""
import numpy as np

from oracle import Oracle
from paper_2501_18185_gb300 import workloads as W

N70 = 70


def _ints(n, seed, naux=6):
    rng = np.random.default_rng(seed)
    return W.real_integrals(rng, n, naux, 0.95)


def _keys(occ_alpha, occ_beta, n):
    """[M, 3] words of the determinants (alpha orbitals, beta orbitals), unsorted."""
    occ = np.concatenate([np.asarray(occ_alpha, dtype=np.int64), np.asarray(occ_beta, dtype=np.int64) + n], axis=1)
    return W.words_from_occ(occ, 3)


def _as_int(k):
    return int(k[0]) | (int(k[1]) << 64) | (int(k[2]) << 128)


def test_three_word_keys_from_occupations():
    """The word builder places bit b in word b // 64: alpha 69 and beta 0 (bits 69, 70) in
    word 1, beta 69 (bit 139) in word 2; sorting orders by the 192-bit value."""
    k = _keys([[0, 69]], [[0, 69]], N70)[0]
    assert _as_int(k) == (1 << 0) | (1 << 69) | (1 << 70) | (1 << 139)
    rng = np.random.default_rng(3)
    ks = _keys(np.sort(rng.choice(N70, (200, 2)), axis=1), np.sort(rng.choice(N70, (200, 2)), axis=1), N70)
    s = W.sort_words(ks)
    assert sorted(_as_int(x) for x in ks) == [_as_int(x) for x in s]


def test_two_electron_opposite_spin_closed_form_70_orbitals():
    """One alpha + one beta electron over 70 orbitals (beta bits 70..139 across words 1 and
    2, alpha 64..69 in word 1): <p q|H|r s> = h_pr d_qs + d_pr h_qs + (pr|qs), checked as
    H X on a random block X of the 4,900-determinant space (q major = ascending order)."""
    n = N70
    ints = _ints(n, 71)
    h, eri = ints.h, ints.eri()
    P, Q = np.meshgrid(np.arange(n), np.arange(n))           # row q, column p
    keys = _keys(P.reshape(-1, 1), Q.reshape(-1, 1), n)
    assert [_as_int(k) for k in keys] == sorted(_as_int(k) for k in keys)
    o = Oracle("spin_orbitals", n, h, eri, keys)
    I = np.eye(n)
    V = eri.transpose(2, 0, 3, 1).reshape(n * n, n * n)
    expected = np.kron(I, h) + np.kron(h, I) + V
    X = np.random.default_rng(4).standard_normal((n * n, 2))
    got = o.sigma(X)
    assert np.abs(got - expected @ X).max() < 1e-12 * np.abs(expected @ X).max()


def test_two_electron_same_spin_closed_form_beta_70_orbitals():
    """Two beta electrons over 70 orbitals (bits 70..139): <pq|H|rs> = h_pr d_qs + h_qs d_pr
    - h_ps d_qr - h_qr d_ps + (pr|qs) - (ps|qr) for p<q, r<s, with the phases of strings that
    straddle the word boundary at bit 128; as H X on a random block."""
    n = N70
    ints = _ints(n, 72)
    h, eri = ints.h, ints.eri()
    pairs = np.array([(p, q) for q in range(n) for p in range(q)])
    keys = _keys(np.zeros((len(pairs), 0)), pairs, n)
    o = Oracle("spin_orbitals", n, h, eri, keys)
    p, q = pairs[:, 0], pairs[:, 1]
    r, s = p, q
    d = lambda a, b: (a[:, None] == b[None, :]).astype(float)  # noqa: E731
    E = (h[p][:, r] * d(q, s) + h[q][:, s] * d(p, r) - h[p][:, s] * d(q, r) - h[q][:, r] * d(p, s)
         + eri[p[:, None], r[None, :], q[:, None], s[None, :]] - eri[p[:, None], s[None, :], q[:, None], r[None, :]])
    X = np.random.default_rng(5).standard_normal((len(pairs), 2))
    assert np.abs(o.sigma(X) - E @ X).max() < 1e-12 * np.abs(E @ X).max()


def test_three_word_selected_space_brute_force_and_hermiticity():
    """The selected 70-orbital space (3+3 electrons, 60,000 determinants): sigma by
    generation + lookup equals the all-pairs route on sampled rows, and <x, H y> = <H x, y>
    on a cut of the list."""
    w = W.selected_three_word()
    o = Oracle.from_workload(w)
    rows = np.unique(np.random.default_rng(1).choice(w.M, 80, replace=False))
    assert np.abs(o.sigma_rows(rows, w.c) - o.sigma_brute_rows(rows, w.c)).max() < 1e-13
    cut = Oracle(w.mode, w.n, w.ints.h, w.ints.eri(), w.keys[:4000])
    rng = np.random.default_rng(2)
    x, y = rng.normal(size=4000), rng.normal(size=4000)
    Hx, Hy = cut.sigma(x)[:, 0], cut.sigma(y)[:, 0]
    assert abs(x @ Hy - Hx @ y) < 1e-12 * abs(x @ Hy)


def test_three_word_encoding_of_one_and_two_word_spaces():
    """A space of at most 64 spin-orbitals as three words, and a 40-orbital two-word space
    as three words (top word 0), give the dense H of their own encodings."""
    w = W.random_small(31, "spin_orbitals", 6, 3, 2, naux=4, frac=0.5)
    z = np.zeros_like(w.keys)
    h, eri = w.ints.h, w.ints.eri()
    assert np.array_equal(Oracle("spin_orbitals", 6, h, eri, w.keys).dense(),
                          Oracle("spin_orbitals", 6, h, eri, np.stack([w.keys, z, z], axis=1)).dense())
    w2 = W.selected_two_word(n=40, na=2, nb=1, M=5000)
    k3 = np.concatenate([w2.keys, np.zeros((w2.M, 1), dtype=np.uint64)], axis=1)
    h, eri = w2.ints.h, w2.ints.eri()
    rows = np.arange(0, w2.M, 7)
    a = Oracle("spin_orbitals", 40, h, eri, w2.keys).sigma_rows(rows, w2.c)
    b = Oracle("spin_orbitals", 40, h, eri, k3).sigma_rows(rows, w2.c)
    assert np.array_equal(a, b)


def test_spinor_closed_forms_against_the_oracle():
    """The one- and two-electron spinor closed forms used on more than 128 spinors, checked
    here against the oracle's dense H on 24 complex spinors (one word)."""
    from closed_forms import spinor_pair_sigma

    n = 24
    ints = W.complex_integrals(np.random.default_rng(81), n, 5, 0.95)
    rng = np.random.default_rng(82)
    one = np.array([1 << p for p in range(n)], dtype=np.uint64)
    o1 = Oracle("spinors", n, ints.h, ints.eri(), one)
    c1 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.abs(o1.sigma(c1)[:, 0] - ints.h @ c1).max() < 1e-13
    pairs = np.array([(p, q) for q in range(n) for p in range(q)])
    keys = np.array([(1 << int(p)) | (1 << int(q)) for p, q in pairs], dtype=np.uint64)
    assert np.all(np.diff(keys.astype(np.float64)) > 0)
    o2 = Oracle("spinors", n, ints.h, ints.eri(), keys)
    c2 = rng.standard_normal((len(pairs), 2)) + 1j * rng.standard_normal((len(pairs), 2))
    ref = spinor_pair_sigma(ints.h, ints.chol, pairs, c2)
    assert np.abs(o2.sigma(c2) - ref).max() < 1e-12 * np.abs(ref).max()


def _spin_block_energy(h, eri, g1, g2):
    """sum h g1 + 1/2 sum (pq|rs) g2 over spin-orbitals p = (sigma, p'), with the spin-orbital
    integrals of a spin-free H: h and (pq|rs) inside each spin block, zero across."""
    n = h.shape[0]
    E1 = np.einsum("pq,pq->", h, g1[:n, :n]) + np.einsum("pq,pq->", h, g1[n:, n:])
    G = g2.reshape(2, n, 2, n, 2, n, 2, n)
    E2 = sum(np.einsum("pqrs,pqrs->", eri, G[a, :, a, :, b, :, b, :]) for a in range(2) for b in range(2))
    return E1 + 0.5 * E2


def test_rdm12_three_words_energy_traces_and_symmetries_65_orbitals():
    """The oracle's density matrices on 65 orbitals (130 spin-orbitals: alpha 64 in word 1,
    beta 63..64 at bits 128..129 of word 2), HF and 400 random 2 alpha + 1 beta
    determinants: the energy identity against c^+ H c with the oracle's sigma (pinned above
    by the closed forms), the traces N and N(N - 1), Hermiticity of g1 and the pair
    symmetries of g2 on sampled elements."""
    n, na, nb = 65, 2, 1
    ints = _ints(n, 97, naux=4)
    h, eri = ints.h, ints.eri()
    rng = np.random.default_rng(98)
    occ = {(tuple(range(na)), tuple(range(nb)))}
    while len(occ) < 401:
        occ.add((tuple(sorted(rng.choice(n, na, replace=False))), tuple(sorted(rng.choice(n, nb, replace=False)))))
    occ = sorted(occ)
    keys = W.sort_words(_keys([a for a, _ in occ], [b for _, b in occ], n))
    assert (keys[:, 2] != 0).any()
    o = Oracle("spin_orbitals", n, h, eri, keys)
    c = rng.standard_normal(len(keys))
    c /= np.linalg.norm(c)
    g1, g2 = o.rdm12(c)
    E = _spin_block_energy(h, eri, g1, g2)
    assert abs(E - np.vdot(c, o.sigma(c)[:, 0])) < 1e-11 * max(1.0, abs(E))
    N = na + nb
    assert abs(np.trace(g1) - N) < 1e-12
    assert abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-10
    assert np.abs(g1 - g1.T).max() < 1e-14
    idx = rng.integers(0, 2 * n, size=(20000, 4))
    p, q, r, s = idx.T
    assert np.abs(g2[p, q, r, s] - g2[r, s, p, q]).max() < 1e-14
    assert np.abs(g2[p, q, r, s] - g2[q, p, s, r]).max() < 1e-14


def test_rdm12_three_word_encoding_of_a_two_word_space():
    """A 40-orbital two-word space given as three words (top word 0) has the density
    matrices of its two-word encoding, bit for bit on one thread."""
    import oracle

    n = 40
    rng = np.random.default_rng(99)
    occ = {((0, 1), (0,))}
    while len(occ) < 500:
        occ.add((tuple(sorted(rng.choice(n, 2, replace=False))), tuple(sorted(rng.choice(n, 1, replace=False)))))
    occ = np.array([list(a) + [b[0] + n] for a, b in sorted(occ)])
    k2 = W.sort_words(W.words_from_occ(occ, 2))
    k3 = np.concatenate([k2, np.zeros((len(k2), 1), dtype=np.uint64)], axis=1)
    ints = _ints(n, 100, naux=4)
    c = rng.standard_normal(len(k2))
    o2 = Oracle("spin_orbitals", n, ints.h, ints.eri(), k2)
    o3 = Oracle("spin_orbitals", n, ints.h, ints.eri(), k3)
    oracle.set_threads(1)
    try:
        a1, a2 = o2.rdm12(c)
        b1, b2 = o3.rdm12(c)
    finally:
        oracle.set_threads(0)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)


def test_enpt2_three_words_against_the_definition_on_the_full_space():
    """ENPT2 of a P inside the full 1 + 1-electron space of 65 orbitals (4,225 determinants;
    alpha orbital 64 in word 1, beta orbitals 63 and 64 at bits 128 and 129 of word 2):
    sciref_enpt2 (generation of the excitations of P, deduplication by three-word key)
    against Eq. ENPT2E written out with H of the whole space (the oracle's sigma and
    diagonal, pinned above by the closed form), two roots with arbitrary E0; the external
    count against the size of Q."""
    n = 65
    ints = _ints(n, 101, naux=4)
    P_, Q_ = np.meshgrid(np.arange(n), np.arange(n))
    full = _keys(P_.reshape(-1, 1), Q_.reshape(-1, 1), n)
    assert [_as_int(k) for k in full] == sorted(_as_int(k) for k in full)
    of = Oracle("spin_orbitals", n, ints.h, ints.eri(), full)
    rng = np.random.default_rng(102)
    inP = rng.random(len(full)) < 0.3
    inP[0] = True
    P = full[inP]
    C = rng.standard_normal((len(P), 2))
    E0 = np.array([-30.0, -25.0])
    Cf = np.zeros((len(full), 2))
    Cf[inP] = C
    v = of.sigma(Cf)                         # sum_J H_IJ c_J over J in P, for every I
    d = of.diagonal()
    Q = ~inP
    ref = ((v[Q] ** 2) / (E0[None, :] - d[Q, None])).sum(axis=0)
    op = Oracle("spin_orbitals", n, ints.h, ints.eri(), P)
    E2, nx = op.enpt2(C, E0)
    assert np.allclose(E2, ref, rtol=1e-12, atol=0)
    assert nx == int(Q.sum())


def test_enpt2_three_word_encoding_of_a_two_word_space():
    """A 40-orbital two-word list given as three words gives the two-word ENPT2."""
    n = 40
    rng = np.random.default_rng(103)
    occ = {((0, 1), (0,))}
    while len(occ) < 300:
        occ.add((tuple(sorted(rng.choice(n, 2, replace=False))), tuple(sorted(rng.choice(n, 1, replace=False)))))
    occ = np.array([list(a) + [b[0] + n] for a, b in sorted(occ)])
    k2 = W.sort_words(W.words_from_occ(occ, 2))
    k3 = np.concatenate([k2, np.zeros((len(k2), 1), dtype=np.uint64)], axis=1)
    ints = _ints(n, 104, naux=4)
    C = rng.standard_normal((len(k2), 2))
    E0 = np.array([-20.0, -18.0])
    a, na_ = Oracle("spin_orbitals", n, ints.h, ints.eri(), k2).enpt2(C, E0)
    b, nb_ = Oracle("spin_orbitals", n, ints.h, ints.eri(), k3).enpt2(C, E0)
    assert na_ == nb_ and np.allclose(a, b, rtol=1e-13, atol=0)
