"""Seeded synthetic inputs for the selected-CI sigma path.

This module only draws inputs: one-electron integrals h, Cholesky factors L^P of the
two-electron integrals, determinant lists and coefficient vectors.  It contains none of
the method's arithmetic (no matrix elements, phases or connection search), so both the
CPU oracle and the CUDA path consume it without sharing any computation.

Workloads are shaped like the paper's showcases (Sec. 4, Table CmprNonRelaRela:
|P| ~ 1.9M CSFs for sf-X2C Br/DZ and ~1.0M for 4C Br/DZ), but are synthetic; the
molecular integrals of the paper are not available.

Conventions (shared by every consumer, stated once here):
  * Spin-orbital mode (n spatial orbitals, n <= 32): bit p of a determinant key is the
    alpha spin-orbital p, bit n+p is the beta spin-orbital p.
  * Spinor mode (n spinors, n <= 64): bit p is spinor p.
  * "HF" is the determinant with the lowest n_alpha alpha and lowest n_beta beta
    orbitals occupied (spinor mode: lowest N spinors).
  * The excitation level of a determinant D is popcount(D xor HF) / 2.

Random draws use numpy.random.default_rng(SEED_BASE + k) for workload k, in the order
written in each function.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from math import comb

import numpy as np

SEED_BASE = 2501181850


# --------------------------------------------------------------------------- integrals
def sym_normal(rng: np.random.Generator, n: int, sd: float) -> np.ndarray:
    """Symmetric n x n matrix: upper triangle (with diagonal) ~ N(0, sd), mirrored."""
    iu = np.triu_indices(n)
    vals = rng.normal(0.0, sd, size=len(iu[0]))
    m = np.zeros((n, n))
    m[iu] = vals
    m = m + m.T - np.diag(np.diag(m))
    return m


def herm_normal(rng: np.random.Generator, n: int, sd: float) -> np.ndarray:
    """Hermitian (B + B^H)/2 with Re B, Im B ~ N(0, sd^2 / 2) elementwise."""
    s = sd / np.sqrt(2.0)
    b = rng.normal(0.0, s, size=(n, n)) + 1j * rng.normal(0.0, s, size=(n, n))
    return 0.5 * (b + b.conj().T)


@dataclass
class Integrals:
    """h (n x n) and Cholesky factors chol (naux x n x n) with (pq|rs) = sum_P L^P_pq L^P_rs."""
    h: np.ndarray
    chol: np.ndarray
    complex_: bool = False

    @property
    def n(self) -> int:
        return self.h.shape[0]

    def eri(self) -> np.ndarray:
        """Dense (pq|rs) in Mulliken order [p,q,r,s] (definition of the synthetic input)."""
        return np.einsum("Ppq,Prs->pqrs", self.chol, self.chol, optimize=True)


def real_integrals(rng, n: int, naux: int, decay: float | None) -> Integrals:
    """h = sym N(0, 0.1) + linspace(-2, 0, n) on the diagonal; L^P symmetric.

    decay None: each L^P ~ sym N(0, 0.3).  decay d: L^P is a sym N(0, 1) matrix rescaled
    to Frobenius norm 0.3 * n * d**P (P = 0 matches the undecayed scale).
    Draw order: h, then L^0 .. L^{naux-1}.
    """
    h = sym_normal(rng, n, 0.1)
    h[np.diag_indices(n)] += np.linspace(-2.0, 0.0, n)
    chol = np.empty((naux, n, n))
    for P in range(naux):
        if decay is None:
            chol[P] = sym_normal(rng, n, 0.3)
        else:
            m = sym_normal(rng, n, 1.0)
            chol[P] = m * (0.3 * n * decay ** P / np.linalg.norm(m))
    return Integrals(h=h, chol=chol, complex_=False)


def complex_integrals(rng, n: int, naux: int, decay: float) -> Integrals:
    """Hermitian complex h (sd 0.1 plus the real ascending diagonal) and Hermitian L^P.

    Draw order: h, then L^0 .. L^{naux-1}; each L^P is herm_normal(sd 0.3) rescaled to
    Frobenius norm 0.3 * n * decay**P.  With Hermitian L^P the dense (pq|rs) obeys
    (pq|rs) = (rs|pq) = (qp|sr)^*.
    """
    h = herm_normal(rng, n, 0.1)
    h[np.diag_indices(n)] += np.linspace(-2.0, 0.0, n)
    chol = np.empty((naux, n, n), dtype=np.complex128)
    for P in range(naux):
        m = herm_normal(rng, n, 0.3)
        chol[P] = m * (0.3 * n * decay ** P / np.linalg.norm(m))
    return Integrals(h=h, chol=chol, complex_=True)


# --------------------------------------------------------------------------- strings
def _bits_to_mask(cols: np.ndarray) -> np.ndarray:
    """Rows of orbital indices -> uint64 bit masks."""
    if cols.size == 0:
        return np.zeros(cols.shape[0], dtype=np.uint64)
    return np.bitwise_or.reduce(np.left_shift(np.uint64(1), cols.astype(np.uint64)), axis=1)


def _combos(items, k) -> np.ndarray:
    c = list(itertools.combinations(items, k))
    if k == 0:
        return np.zeros((1, 0), dtype=np.int64)
    return np.array(c, dtype=np.int64).reshape(len(c), k)


def strings_at_level(n: int, nocc: int, level: int) -> np.ndarray:
    """All occupation strings of n orbitals with nocc electrons at excitation level
    `level` from the lowest-nocc reference, as uint64, in (holes, particles)
    lexicographic order."""
    ref = np.uint64((1 << nocc) - 1)
    hole_masks = _bits_to_mask(_combos(range(nocc), level))
    part_masks = _bits_to_mask(_combos(range(nocc, n), level))
    s = (ref ^ hole_masks)[:, None] | part_masks[None, :]
    return s.reshape(-1).astype(np.uint64)


def n_strings_at_level(n: int, nocc: int, level: int) -> int:
    return comb(nocc, level) * comb(n - nocc, level)


def all_strings(n: int, nocc: int) -> np.ndarray:
    """Every string with nocc of n bits set, ascending."""
    return np.sort(np.concatenate([strings_at_level(n, nocc, L) for L in range(min(nocc, n - nocc) + 1)]))


# --------------------------------------------------------------------------- spaces
@dataclass
class Workload:
    name: str
    mode: str                 # "spin_orbitals" | "spinors"
    n: int                    # spatial orbitals (spin_orbitals) or spinors
    n_alpha: int
    n_beta: int               # -1 in spinor mode
    keys: np.ndarray          # uint64, strictly ascending
    ints: Integrals
    c: np.ndarray             # [M][nvec] float64 or complex128
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.keys.shape[0])

    @property
    def n_electrons(self) -> int:
        return self.n_alpha + (self.n_beta if self.mode == "spin_orbitals" else 0)

    def hf_key(self) -> np.uint64:
        if self.mode == "spinors":
            return np.uint64((1 << self.n_alpha) - 1)
        return np.uint64(((1 << self.n_alpha) - 1) | (((1 << self.n_beta) - 1) << self.n))


def excitation_level(keys: np.ndarray, hf: np.uint64) -> np.ndarray:
    return (np.bitwise_count(keys ^ hf) // 2).astype(np.int64)


def coefficient_vector(rng, keys, hf, nvec=1, complex_=False, decay_by_level=True) -> np.ndarray:
    """|c_I| = exp(-level_I) with a random sign (complex: random phase e^{i theta}),
    each column normalised in the 2-norm.  decay_by_level False: N(0,1) entries."""
    M = len(keys)
    cols = []
    for _ in range(nvec):
        if decay_by_level:
            mag = np.exp(-excitation_level(keys, hf).astype(np.float64))
            if complex_:
                ph = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=M))
                v = mag * ph
            else:
                v = mag * rng.choice(np.array([-1.0, 1.0]), size=M)
        else:
            v = rng.normal(size=M)
            if complex_:
                v = v + 1j * rng.normal(size=M)
        cols.append(v / np.linalg.norm(v))
    return np.stack(cols, axis=1)


def fci_keys(n: int, n_alpha: int, n_beta: int) -> np.ndarray:
    a = all_strings(n, n_alpha)
    b = all_strings(n, n_beta)
    keys = (a[None, :] | (b[:, None] << np.uint64(n))).reshape(-1)
    return np.sort(keys)


def fci_spinor_keys(n: int, N: int) -> np.ndarray:
    return all_strings(n, N)


def _sample_split_excitations(rng, n, na, nb, splits, count):
    """Uniform sample without replacement over the union of all (ka, kb) splits."""
    sizes = [n_strings_at_level(n, na, ka) * n_strings_at_level(n, nb, kb) for ka, kb in splits]
    total = int(sum(sizes))
    idx = np.sort(rng.choice(total, size=count, replace=False))
    out = []
    off = 0
    for (ka, kb), sz in zip(splits, sizes):
        sel = idx[(idx >= off) & (idx < off + sz)] - off
        off += sz
        if sel.size == 0:
            continue
        A = strings_at_level(n, na, ka)
        B = strings_at_level(n, nb, kb)
        ia, ib = sel // len(B), sel % len(B)
        out.append(A[ia] | (B[ib] << np.uint64(n)))
    return np.concatenate(out) if out else np.zeros(0, dtype=np.uint64)


def selected_spin_orbital_keys(rng, n, na, nb, M) -> tuple[np.ndarray, dict]:
    """HF + all singles + all doubles (Sz-conserving) + random triples/quadruples.

    The M - 1 - (#singles + #doubles) remaining slots are split half triples, half
    quadruples (odd remainder to triples), each drawn uniformly without replacement
    over all Sz-conserving spin splits of that level.
    """
    hf_a = np.uint64((1 << na) - 1)
    hf_b = np.uint64((1 << nb) - 1)
    parts = []
    counts = {}
    for level in range(3):
        for ka in range(level + 1):
            kb = level - ka
            if ka > min(na, n - na) or kb > min(nb, n - nb):
                continue
            A = strings_at_level(n, na, ka)
            B = strings_at_level(n, nb, kb)
            parts.append((A[None, :] | (B[:, None] << np.uint64(n))).reshape(-1))
        counts[level] = int(sum(len(p) for p in parts)) - sum(counts.values())
    rest = M - sum(counts.values())
    if rest < 0:
        raise ValueError("M smaller than HF+singles+doubles")
    n_trip = (rest + 1) // 2
    n_quad = rest - n_trip
    for level, cnt in ((3, n_trip), (4, n_quad)):
        splits = [(ka, level - ka) for ka in range(level + 1)
                  if ka <= min(na, n - na) and level - ka <= min(nb, n - nb)]
        parts.append(_sample_split_excitations(rng, n, na, nb, splits, cnt))
        counts[level] = cnt
    keys = np.sort(np.concatenate(parts))
    assert len(keys) == M
    return keys, {"level_counts": counts}


def selected_spinor_keys(rng, n, N, M) -> tuple[np.ndarray, dict]:
    """HF + all singles + all doubles + random triples (uniform, without replacement)."""
    parts = [strings_at_level(n, N, L) for L in range(3)]
    base = sum(len(p) for p in parts)
    n_trip = M - base
    total3 = n_strings_at_level(n, N, 3)
    sel = np.sort(rng.choice(total3, size=n_trip, replace=False))
    T = strings_at_level(n, N, 3)
    parts.append(T[sel])
    keys = np.sort(np.concatenate(parts))
    assert len(keys) == M
    return keys, {"level_counts": {0: 1, 1: len(parts[1]), 2: len(parts[2]), 3: n_trip}}


# --------------------------------------------------------------------------- configs
def fci_small_8o(seed_offset: int = 1) -> Workload:
    """8 spatial orbitals, 4+4 electrons, full CI (4,900 determinants); 16 Cholesky
    vectors of sym N(0, 0.3); one seeded N(0,1) unit vector c.
    Draw order: integrals, then c."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    ints = real_integrals(rng, 8, 16, None)
    keys = fci_keys(8, 4, 4)
    c = coefficient_vector(rng, keys, np.uint64(0), 1, False, decay_by_level=False)
    return Workload("fci_8o_4a4b", "spin_orbitals", 8, 4, 4, keys, ints, c)


def selected_30o(M: int = 2_000_000, nvec: int = 1, seed_offset: int = 2) -> Workload:
    """30 spatial orbitals, 10+10 electrons, selected space of M determinants;
    120 Cholesky vectors with Frobenius norms 0.3*n*0.95^P; |c| = exp(-level).
    Draw order: integrals, determinant space, c."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    ints = real_integrals(rng, 30, 120, 0.95)
    keys, meta = selected_spin_orbital_keys(rng, 30, 10, 10, M)
    w = Workload(f"sel_30o_10a10b_M{M}", "spin_orbitals", 30, 10, 10, keys, ints, None, meta)
    w.c = coefficient_vector(rng, keys, w.hf_key(), nvec, False)
    return w


def selected_30o_cut(M: int = 1000, seed: int = 7) -> Workload:
    """A small selected space of the 30-orbital recipe, for checks against slow routes:
    the integrals of selected_30o() and, from its 60,000-determinant space, HF, all 400
    singles, then M//3 doubles, M//4 triples and the rest quadruples drawn uniformly
    without replacement (rng seeded by `seed`), sorted.  c as in selected_30o()
    (|c| = exp(-level), random signs, normalised; drawn from the same seeded rng)."""
    base = selected_30o(M=60000)
    hf = base.hf_key()
    lev = excitation_level(base.keys, hf)
    rng = np.random.default_rng(seed)
    keep = [np.flatnonzero(lev <= 1)]
    n2, n3 = M // 3, M // 4
    n4 = M - len(keep[0]) - n2 - n3
    if n4 < 0:
        raise ValueError("M too small for HF + singles")
    for level, cnt in ((2, n2), (3, n3), (4, n4)):
        keep.append(rng.choice(np.flatnonzero(lev == level), cnt, replace=False))
    keys = base.keys[np.sort(np.concatenate(keep))]
    w = Workload(f"sel_30o_10a10b_cut{M}_s{seed}", "spin_orbitals", 30, 10, 10, keys, base.ints, None,
                 {"from": base.name})
    w.c = coefficient_vector(rng, keys, hf, 1, False)
    return w


def selected_spinor_64_cut(n1: int = 200, n2: int = 60, n3: int = 40, seed: int = 9) -> Workload:
    """A small selected space of the 64-spinor recipe, for checks against slow routes: the
    integrals of selected_spinor_64() and, from its 120,000-determinant space, HF plus n1
    singles, n2 doubles and n3 triples drawn uniformly without replacement (rng seeded by
    `seed`), sorted; complex c with |c| = exp(-level) and random phases, normalised."""
    base = selected_spinor_64(M=120000)
    hf = base.hf_key()
    lev = excitation_level(base.keys, hf)
    rng = np.random.default_rng(seed)
    keep = [np.flatnonzero(lev == 0)]
    for level, cnt in ((1, n1), (2, n2), (3, n3)):
        keep.append(rng.choice(np.flatnonzero(lev == level), cnt, replace=False))
    keys = base.keys[np.sort(np.concatenate(keep))]
    w = Workload(f"sel_64s_14e_cut{len(keys)}_s{seed}", "spinors", 64, 14, -1, keys, base.ints, None,
                 {"from": base.name})
    w.c = coefficient_vector(rng, keys, hf, 1, True)
    return w


def two_word_keys(alpha: np.ndarray, beta: np.ndarray, n: int) -> np.ndarray:
    """Spin-orbital keys of more than 64 bits (alpha string in bits 0..n-1, beta string in
    bits n..2n-1, 2n <= 128) as [M, 2] uint64 words, word 0 holding bits 0..63."""
    a = np.asarray(alpha, dtype=np.uint64)
    b = np.asarray(beta, dtype=np.uint64)
    lo = a | (b << np.uint64(n)) if n < 64 else a
    hi = b >> np.uint64(64 - n) if n < 64 else b << np.uint64(n - 64)
    return np.stack([lo, hi], axis=1)


def sort_words(keys: np.ndarray) -> np.ndarray:
    """[M, K] word keys in ascending order as (64 K)-bit integers (word K-1 most
    significant)."""
    return keys[np.lexsort(tuple(keys[:, w] for w in range(keys.shape[1])))]


def occ_at_level(n: int, nocc: int, level: int) -> np.ndarray:
    """Occupied-orbital lists [count, nocc] (ascending in each row) of the strings of
    strings_at_level(n, nocc, level), in the same (holes, particles) order; no 64-orbital
    limit."""
    holes = _combos(range(nocc), level)
    parts = _combos(range(nocc, n), level)
    out = []
    for h in holes:
        kept = np.array([i for i in range(nocc) if i not in set(h.tolist())], dtype=np.int64)
        out.append(np.concatenate([np.broadcast_to(kept, (len(parts), len(kept))), parts], axis=1))
    return np.concatenate(out) if out else np.zeros((0, nocc), dtype=np.int64)


def words_from_occ(occ: np.ndarray, nwords: int) -> np.ndarray:
    """[M, nwords] uint64 words of the determinants whose occupied bits are the rows of
    `occ` (bit b in word b // 64, position b % 64)."""
    occ = np.asarray(occ, dtype=np.int64)
    out = np.zeros((occ.shape[0], nwords), dtype=np.uint64)
    if occ.shape[1] == 0:
        return out
    one = np.uint64(1)
    for w in range(nwords):
        bits = np.where((occ >> 6) == w, np.left_shift(one, (occ & 63).astype(np.uint64)), np.uint64(0))
        out[:, w] = np.bitwise_or.reduce(bits, axis=1)
    return out


def excitation_level_words(keys: np.ndarray, hf: np.ndarray) -> np.ndarray:
    x = keys ^ hf[None, :]
    return (np.bitwise_count(x).sum(axis=1) // 2).astype(np.int64)


def selected_two_word(n: int = 40, na: int = 4, nb: int = 4, M: int = 40000, naux: int = 40, nvec: int = 1,
                      seed: int = 2501181860) -> Workload:
    """A selected space of more than 64 spin-orbitals (two-word keys): n spatial orbitals
    (2n > 64), na + nb electrons, HF + all singles + all Sz-conserving doubles + random
    triples (uniform over all spin splits, without replacement) up to M determinants,
    sorted as 128-bit integers; real integrals with naux Cholesky vectors of Frobenius norms
    0.3 n 0.95^P; |c| = exp(-level) with random signs, normalised.
    Draw order: integrals, triples, c."""
    rng = np.random.default_rng(seed)
    ints = real_integrals(rng, n, naux, 0.95)
    parts = []
    for level in range(3):
        for ka in range(level + 1):
            kb = level - ka
            if ka > min(na, n - na) or kb > min(nb, n - nb):
                continue
            A = strings_at_level(n, na, ka)
            B = strings_at_level(n, nb, kb)
            parts.append(two_word_keys(np.repeat(A, len(B)), np.tile(B, len(A)), n))
    base = np.concatenate(parts)
    rest = M - len(base)
    if rest < 0:
        raise ValueError("M smaller than HF+singles+doubles")
    splits = [(ka, 3 - ka) for ka in range(4) if ka <= min(na, n - na) and 3 - ka <= min(nb, n - nb)]
    sizes = [n_strings_at_level(n, na, ka) * n_strings_at_level(n, nb, kb) for ka, kb in splits]
    idx = np.sort(rng.choice(int(sum(sizes)), size=rest, replace=False))
    trip, off = [], 0
    for (ka, kb), sz in zip(splits, sizes):
        sel = idx[(idx >= off) & (idx < off + sz)] - off
        off += sz
        if sel.size:
            A = strings_at_level(n, na, ka)
            B = strings_at_level(n, nb, kb)
            trip.append(two_word_keys(A[sel // len(B)], B[sel % len(B)], n))
    keys = sort_words(np.concatenate([base] + trip))
    assert len(keys) == M
    hf = two_word_keys(np.array([(1 << na) - 1], dtype=np.uint64), np.array([(1 << nb) - 1], dtype=np.uint64), n)[0]
    lev = excitation_level_words(keys, hf)
    cols = []
    for _ in range(nvec):
        v = np.exp(-lev.astype(np.float64)) * rng.choice(np.array([-1.0, 1.0]), size=M)
        cols.append(v / np.linalg.norm(v))
    w = Workload(f"sel2w_{n}o_{na}a{nb}b_M{M}", "spin_orbitals", n, na, nb, keys, ints, np.stack(cols, axis=1),
                 {"hf_words": hf})
    return w


def selected_three_word(n: int = 70, na: int = 3, nb: int = 3, M: int = 60000, naux: int = 40, nvec: int = 1,
                        seed: int = 2501181861) -> Workload:
    """A selected space of more than 128 spin-orbitals (three-word keys): n spatial orbitals
    (2n > 128), the recipe of selected_two_word (HF + all singles + all Sz-conserving
    doubles + random triples over the spin splits, without replacement, up to M
    determinants; real integrals with naux Cholesky vectors of Frobenius norms 0.3 n 0.95^P;
    |c| = exp(-level) with random signs, normalised), built from occupied-orbital lists
    and sorted as (64 x 3)-bit integers.  Alpha bits 0..n-1, beta bits n..2n-1: for
    64 < n <= 96 the alpha string crosses words 0/1 and the beta string words 1/2.
    Draw order: integrals, triples, c."""
    return selected_words(n, na, nb, M, 3, naux, nvec, seed, "sel3w")


def selected_words(n: int, na: int, nb: int, M: int, nwords: int, naux: int = 40, nvec: int = 1,
                   seed: int = 2501181863, tag: str | None = None) -> Workload:
    """The recipe of selected_three_word with keys of `nwords` words (64 nwords >= 2n): for
    96 < n <= 128 and four words the beta string crosses words 1, 2 and 3."""
    rng = np.random.default_rng(seed)
    ints = real_integrals(rng, n, naux, 0.95)

    def dets(A, B):
        return words_from_occ(np.concatenate([A, B + n], axis=1), nwords)

    parts = []
    for level in range(3):
        for ka in range(level + 1):
            kb = level - ka
            if ka > min(na, n - na) or kb > min(nb, n - nb):
                continue
            A = occ_at_level(n, na, ka)
            B = occ_at_level(n, nb, kb)
            parts.append(dets(np.repeat(A, len(B), axis=0), np.tile(B, (len(A), 1))))
    base = np.concatenate(parts)
    rest = M - len(base)
    if rest < 0:
        raise ValueError("M smaller than HF+singles+doubles")
    splits = [(ka, 3 - ka) for ka in range(4) if ka <= min(na, n - na) and 3 - ka <= min(nb, n - nb)]
    sizes = [n_strings_at_level(n, na, ka) * n_strings_at_level(n, nb, kb) for ka, kb in splits]
    idx = np.sort(rng.choice(int(sum(sizes)), size=rest, replace=False))
    trip, off = [], 0
    for (ka, kb), sz in zip(splits, sizes):
        sel = idx[(idx >= off) & (idx < off + sz)] - off
        off += sz
        if sel.size:
            A = occ_at_level(n, na, ka)
            B = occ_at_level(n, nb, kb)
            trip.append(dets(A[sel // len(B)], B[sel % len(B)]))
    keys = sort_words(np.concatenate([base] + trip))
    assert len(keys) == M
    hf = dets(np.arange(na)[None, :], np.arange(nb)[None, :])[0]
    lev = excitation_level_words(keys, hf)
    cols = []
    for _ in range(nvec):
        v = np.exp(-lev.astype(np.float64)) * rng.choice(np.array([-1.0, 1.0]), size=M)
        cols.append(v / np.linalg.norm(v))
    return Workload(f"{tag or f'sel{nwords}w'}_{n}o_{na}a{nb}b_M{M}", "spin_orbitals", n, na, nb, keys, ints,
                    np.stack(cols, axis=1), {"hf_words": hf})


def selected_spinor_words(n: int = 136, N: int = 14, M: int = 1_000_000, naux: int = 80, nvec: int = 1,
                          seed: int = 2501181862) -> Workload:
    """A selected spinor space of n > 128 spinors (three-word keys), N electrons: HF + all
    singles + all doubles + random triples (uniform, without replacement) up to M
    determinants, sorted as (64 x 3)-bit integers; complex integrals as selected_spinor_64
    (naux Cholesky vectors, decay 0.95); |c| = exp(-level) with random complex phases,
    normalised.  Draw order: integrals, triples, c."""
    rng = np.random.default_rng(seed)
    ints = complex_integrals(rng, n, naux, 0.95)
    parts = [words_from_occ(occ_at_level(n, N, L), 3) for L in range(3)]
    rest = M - sum(len(x) for x in parts)
    if rest < 0:
        raise ValueError("M smaller than HF+singles+doubles")
    holes = _combos(range(N), 3)
    kept = np.array([[i for i in range(N) if i not in set(h.tolist())] for h in holes], dtype=np.int64)
    prt = _combos(range(N, n), 3)
    idx = np.sort(rng.choice(len(holes) * len(prt), size=rest, replace=False))
    occ = np.concatenate([kept[idx // len(prt)], prt[idx % len(prt)]], axis=1)
    keys = sort_words(np.concatenate(parts + [words_from_occ(occ, 3)]))
    assert len(keys) == M
    hf = words_from_occ(np.arange(N)[None, :], 3)[0]
    lev = excitation_level_words(keys, hf)
    cols = []
    for _ in range(nvec):
        v = np.exp(-lev.astype(np.float64)) * np.exp(2j * np.pi * rng.random(M))
        cols.append(v / np.linalg.norm(v))
    return Workload(f"sel_{n}s_{N}e_M{M}", "spinors", n, N, -1, keys, ints, np.stack(cols, axis=1), {"hf_words": hf})


def selected_spinor_64(M: int = 1_000_000, nvec: int = 1, seed_offset: int = 4) -> Workload:
    """64 spinors, 14 electrons, selected space of M determinants (HF + singles + doubles
    + random triples); 80 Hermitian complex Cholesky vectors; complex c.
    Draw order: integrals, determinant space, c."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    ints = complex_integrals(rng, 64, 80, 0.95)
    keys, meta = selected_spinor_keys(rng, 64, 14, M)
    w = Workload(f"sel_64s_14e_M{M}", "spinors", 64, 14, -1, keys, ints, None, meta)
    w.c = coefficient_vector(rng, keys, w.hf_key(), nvec, True)
    return w


def random_small(seed: int, mode: str, n: int, na: int, nb: int, naux: int = 6,
                 frac: float = 1.0, nvec: int = 1) -> Workload:
    """Small test system: FCI space (frac=1) or a random subset of it that always keeps
    HF.  Integrals as in the 8-orbital workload (spin_orbitals) or complex Hermitian
    (spinors; nb ignored).  c ~ N(0,1) per column, normalised.
    Draw order: integrals, subset, c."""
    rng = np.random.default_rng(seed)
    if mode == "spin_orbitals":
        ints = real_integrals(rng, n, naux, None)
        keys = fci_keys(n, na, nb)
    else:
        ints = complex_integrals(rng, n, naux, 0.95)
        keys = fci_spinor_keys(n, na)
        nb = -1
    w = Workload(f"small_{mode}_{n}_{na}_{nb}_s{seed}", mode, n, na, nb, keys, ints, None)
    if frac < 1.0:
        hf = w.hf_key()
        keep = rng.random(len(keys)) < frac
        keep |= keys == hf
        w.keys = keys[keep]
    w.c = coefficient_vector(rng, w.keys, w.hf_key(), nvec, mode == "spinors", decay_by_level=False)
    return w


def batch_instances(count: int = 64, max_dim: int = 200_000, seed_offset: int = 3) -> list[Workload]:
    """Heterogeneous small full-CI instances: (n, n_alpha, n_beta) drawn uniformly from
    n in 6..16 and 2..8 electrons per spin (with n_sigma <= n), rejected when the FCI
    dimension C(n, n_alpha) C(n, n_beta) exceeds `max_dim`.  Each instance has integrals
    as in the 8-orbital workload with n Cholesky vectors of sym N(0, 0.3), and one
    N(0,1) unit vector c.
    Draw order: all shapes first, then per instance its integrals and c."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    shapes = []
    while len(shapes) < count:
        n = int(rng.integers(6, 17))
        na, nb = int(rng.integers(2, 9)), int(rng.integers(2, 9))
        if na > n or nb > n or comb(n, na) * comb(n, nb) > max_dim:
            continue
        shapes.append((n, na, nb))
    out = []
    for i, (n, na, nb) in enumerate(shapes):
        ints = real_integrals(rng, n, n, None)
        keys = fci_keys(n, na, nb)
        c = coefficient_vector(rng, keys, np.uint64(0), 1, False, decay_by_level=False)
        out.append(Workload(f"fci_{n}o_{na}a{nb}b_i{i}", "spin_orbitals", n, na, nb, keys, ints, c))
    return out
