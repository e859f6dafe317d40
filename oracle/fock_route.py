"""Second oracle route for tiny spaces: H assembled literally from the operator form.

TEST INFRASTRUCTURE ONLY.  No Slater-Condon closed form is used here.  H restricted to
a determinant list is built from the paper's Eq. Hamiltonian (Sec. 2.1),

    H = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs (pq|rs) a+_p a+_r a_s a_q,

by applying each operator string, one creation/annihilation operator at a time, to every
ket of the list at once (vectorised over kets) and reading off which bra it lands on.
Sign convention: |D> = a+_{p1} a+_{p2} ... |0>, p1 < p2 < ... in bit order, so a_p and
a+_p on D pick up (-1)^(number of occupied bits below p).

The decomposition of Eq. decompositionH (H_1^0 + H_2^0 + H_1^1 + H_2^1 + H_2^2) is also
assembled here from the same operator strings, to check the paper's identity.
"""
from __future__ import annotations

import numpy as np


def _popcount(x: np.ndarray) -> np.ndarray:
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(x).astype(np.int64)
    cnt = np.zeros(x.shape, dtype=np.int64)
    for b in range(64):
        cnt += ((x >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return cnt


def spin_orbital_integrals(h: np.ndarray, eri: np.ndarray):
    """Spatial (n) -> spin-orbital (2n) integrals: bit p < n is alpha p, bit n+p beta p;
    (pq|rs) survives only for spin(p) = spin(q) and spin(r) = spin(s)."""
    n = h.shape[0]
    spin = np.array([0] * n + [1] * n)
    sp = np.concatenate([np.arange(n), np.arange(n)])
    hs = h[np.ix_(sp, sp)] * (spin[:, None] == spin[None, :])
    es = eri[np.ix_(sp, sp, sp, sp)].copy()
    es *= (spin[:, None, None, None] == spin[None, :, None, None])
    es *= (spin[None, None, :, None] == spin[None, None, None, :])
    return hs, es


class _Kets:
    """A batch of occupation strings with a running sign and validity mask."""

    def __init__(self, keys: np.ndarray):
        self.s = keys.astype(np.uint64).copy()
        self.sign = np.ones(len(keys), dtype=np.int64)
        self.ok = np.ones(len(keys), dtype=bool)

    def annihilate(self, p: int):
        bit = np.uint64(1) << np.uint64(p)
        occ = (self.s & bit) != 0
        self.ok &= occ
        below = _popcount(self.s & (bit - np.uint64(1)))
        self.sign *= np.where(below % 2 == 1, -1, 1)
        self.s = self.s & ~bit
        return self

    def create(self, p: int):
        bit = np.uint64(1) << np.uint64(p)
        occ = (self.s & bit) != 0
        self.ok &= ~occ
        below = _popcount(self.s & (bit - np.uint64(1)))
        self.sign *= np.where(below % 2 == 1, -1, 1)
        self.s = self.s | bit
        return self


def _accumulate(H, keys, kets: _Kets, coef):
    """H[bra, ket] += coef * sign for every ket whose image is in the list."""
    idx = np.searchsorted(keys, kets.s)
    idx = np.minimum(idx, len(keys) - 1)
    hit = kets.ok & (keys[idx] == kets.s)
    cols = np.nonzero(hit)[0]
    H[idx[cols], cols] += coef * kets.sign[cols]


def _apply_string(keys, ops):
    """ops: list of ('c'|'a', p) applied right-to-left as written, i.e. ops[-1] first."""
    k = _Kets(keys)
    for kind, p in reversed(ops):
        (k.create if kind == "c" else k.annihilate)(p)
    return k


def hamiltonian(keys: np.ndarray, h_so: np.ndarray, eri_so: np.ndarray) -> np.ndarray:
    """Dense H on the (sorted) list from Eq. Hamiltonian; h_so, eri_so over all bits."""
    keys = np.asarray(keys, dtype=np.uint64)
    norb = h_so.shape[0]
    dt = np.complex128 if (np.iscomplexobj(h_so) or np.iscomplexobj(eri_so)) else np.float64
    M = len(keys)
    H = np.zeros((M, M), dtype=dt)
    for p in range(norb):
        for q in range(norb):
            if h_so[p, q] == 0:
                continue
            _accumulate(H, keys, _apply_string(keys, [("c", p), ("a", q)]), h_so[p, q])
    nz = np.argwhere(eri_so != 0)
    for p, q, r, s in nz:
        ops = [("c", p), ("c", r), ("a", s), ("a", q)]
        _accumulate(H, keys, _apply_string(keys, ops), 0.5 * eri_so[p, q, r, s])
    return H


def rdm12(keys: np.ndarray, c: np.ndarray, norb: int):
    """<c|a+_p a_q|c> and <c|a+_p a+_r a_s a_q|c> by applying each operator string to c
    (c indexed like the sorted keys; unnormalised)."""
    keys = np.asarray(keys, dtype=np.uint64)
    c = np.asarray(c).reshape(-1)
    dt = np.complex128 if np.iscomplexobj(c) else np.float64
    g1 = np.zeros((norb, norb), dtype=dt)
    g2 = np.zeros((norb,) * 4, dtype=dt)

    def expect(ops):
        k = _apply_string(keys, ops)
        idx = np.minimum(np.searchsorted(keys, k.s), len(keys) - 1)
        hit = k.ok & (keys[idx] == k.s)
        return np.sum(np.conj(c[idx[hit]]) * c[hit] * k.sign[hit])

    for p in range(norb):
        for q in range(norb):
            g1[p, q] = expect([("c", p), ("a", q)])
    for p in range(norb):
        for q in range(norb):
            for r in range(norb):
                for s in range(norb):
                    if p == r or q == s:
                        continue
                    g2[p, q, r, s] = expect([("c", p), ("c", r), ("a", s), ("a", q)])
    return g1, g2


def hamiltonian_decomposed(keys: np.ndarray, h_so: np.ndarray, eri_so: np.ndarray,
                           printed_h20: bool = False) -> np.ndarray:
    """H from Eq. decompositionH: H_1^0 + H_1^1 + H_2^0 + H_2^1 + H_2^2.

    Reading of the printed text: in H_2^0 the exchange coefficient of e_{ij,ji} is read
    as (ij|ji) (the printed (ij|jj) cannot follow from Eq. Hamiltonian), and in H_2^1 the
    range "i != j != k" is read as i, j, k pairwise distinct.  E_ij = a+_i a_j and
    e_{ij,kl} = a+_i a+_k a_l a_j (Eq. sym_op).  printed_h20=True uses the coefficient
    as printed, (ij|jj), to show that it does not reproduce Eq. Hamiltonian.
    """
    keys = np.asarray(keys, dtype=np.uint64)
    norb = h_so.shape[0]
    dt = np.complex128 if (np.iscomplexobj(h_so) or np.iscomplexobj(eri_so)) else np.float64
    M = len(keys)
    H = np.zeros((M, M), dtype=dt)
    g = eri_so

    def E(i, j):
        return [("c", i), ("a", j)]

    def e(i, j, k, l):
        return [("c", i), ("c", k), ("a", l), ("a", j)]

    def add(ops, coef):
        if coef != 0:
            _accumulate(H, keys, _apply_string(keys, ops), coef)

    for i in range(norb):                                   # H_1^0
        add(E(i, i), h_so[i, i])
    for i in range(norb):                                   # H_1^1
        for j in range(norb):
            if i != j:
                add(E(i, j), h_so[i, j])
    for i in range(norb):                                   # H_2^0
        # 1/2 (ii|ii) E_ii (E_ii - 1)
        add(E(i, i) + E(i, i), 0.5 * g[i, i, i, i])
        add(E(i, i), -0.5 * g[i, i, i, i])
        for j in range(i + 1, norb):
            add(E(i, i) + E(j, j), g[i, i, j, j])
            add(e(i, j, j, i), g[i, j, j, j] if printed_h20 else g[i, j, j, i])
    for i in range(norb):                                   # H_2^1
        for j in range(norb):
            if i == j:
                continue
            # (ii|ij) (E_ii - 1) E_ij + (ij|jj) E_ij (E_jj - 1)
            add(E(i, i) + E(i, j), g[i, i, i, j])
            add(E(i, j), -g[i, i, i, j])
            add(E(i, j) + E(j, j), g[i, j, j, j])
            add(E(i, j), -g[i, j, j, j])
            for k in range(norb):
                if k == i or k == j:
                    continue
                add(E(i, j) + E(k, k), g[i, j, k, k])
                add(e(i, k, k, j), g[i, k, k, j])
    for i in range(norb):                                   # H_2^2
        for k in range(i, norb):
            for j in range(norb):
                for l in range(j, norb):
                    if j in (i, k) or l in (i, k):
                        continue
                    w = 0.5 if (i == k and j == l) else 1.0
                    add(e(i, j, k, l), w * g[i, j, k, l])
                    if i != k and j != l:
                        add(e(i, l, k, j), g[i, l, k, j])
    return H
