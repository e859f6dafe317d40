"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle (oracle/sciref.c through oracle.Oracle, and the NumPy
operator route oracle/fock_route.py) against something other than itself: closed forms
of two-electron spaces, the one-body (non-interacting) limit, invariance of the FCI
spectrum under orbital rotations and permutations, the paper's Eq. decompositionH,
brute-force enumeration, and combinatorial connection counts.  A dropped term, a wrong
sign, a transposed index or a Mulliken/physicist mix-up fails at least one of them.
"""
import itertools

import numpy as np
import pytest

from oracle import Oracle
from oracle import fock_route as F
from paper_2501_18185_gb300 import workloads as W


def _small(seed, mode, n, na, nb, frac=1.0, naux=5):
    return W.random_small(seed, mode, n, na, nb, naux=naux, frac=frac)


def _so_ints(w):
    eri = w.ints.eri()
    if w.mode == "spin_orbitals":
        return F.spin_orbital_integrals(w.ints.h, eri)
    return w.ints.h, eri


def _oracle_dense(mode, n, h, eri, keys):
    return Oracle(mode, n, h, eri, keys).dense()


def _random_unitary(rng, n, complex_):
    a = rng.normal(size=(n, n)) + (1j * rng.normal(size=(n, n)) if complex_ else 0)
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _rotate(h, eri, U):
    """Orbital rotation phi'_p = sum_q phi_q U_qp: h' = U^+ h U, (pq|rs)' likewise."""
    h2 = U.conj().T @ h @ U
    e2 = np.einsum("ap,bq,cr,ds,abcd->pqrs", U.conj(), U, U.conj(), U, eri, optimize=True)
    return h2, e2


# ---------------------------------------------------------------- closed forms
def test_two_electron_opposite_spin_closed_form():
    """One alpha + one beta electron: |p_a q_b> = a+_p a+_{n+q}|0>.  With no exchange
    between different spins, <p q|H|r s> = h_pr d_qs + d_pr h_qs + (pr|qs): a dense
    n^2 x n^2 assembly with no bit logic (pins Mulliken vs physicist notation)."""
    w = _small(3, "spin_orbitals", 4, 1, 1)
    n, h, eri = w.n, w.ints.h, w.ints.eri()
    # list order is ascending key = 2^p + 2^(n+q): q major, p minor
    I = np.eye(n)
    V = eri.transpose(2, 0, 3, 1).reshape(n * n, n * n)       # [(q,p),(s,r)] = (pr|qs)
    expected = np.kron(I, h) + np.kron(h, I) + V
    Ho = _oracle_dense(w.mode, n, h, eri, w.keys)
    assert np.abs(Ho - expected).max() < 1e-13
    hs, es = _so_ints(w)
    assert np.abs(F.hamiltonian(w.keys, hs, es) - expected).max() < 1e-13


@pytest.mark.parametrize("mode", ["spin_orbitals", "spinors"])
def test_two_electron_same_spin_closed_form(mode):
    """Two electrons of one kind, |pq> = a+_p a+_q|0>, p<q:
    <pq|H|rs> = h_pr d_qs + h_qs d_pr - h_ps d_qr - h_qr d_ps + (pr|qs) - (ps|qr).
    Pins the antisymmetrisation, the exchange sign and (complex) index order."""
    if mode == "spin_orbitals":
        w = _small(5, mode, 5, 2, 0)
    else:
        w = _small(5, mode, 6, 2, 0)
    n, h, eri = w.n, w.ints.h, w.ints.eri()
    pairs = [(p, q) for q in range(n) for p in range(q)]              # ascending key order
    assert np.array_equal(np.array([(1 << p) | (1 << q) for p, q in pairs], dtype=np.uint64), w.keys)
    d = lambda a, b: 1.0 if a == b else 0.0  # noqa: E731
    E = np.zeros((len(pairs), len(pairs)), dtype=np.result_type(h, eri))
    for x, (p, q) in enumerate(pairs):
        for y, (r, s) in enumerate(pairs):
            E[x, y] = (h[p, r] * d(q, s) + h[q, s] * d(p, r) - h[p, s] * d(q, r) - h[q, r] * d(p, s)
                       + eri[p, r, q, s] - eri[p, s, q, r])
    Ho = _oracle_dense(w.mode, n, h, eri, w.keys)
    assert np.abs(Ho - E).max() < 1e-13


# ---------------------------------------------------------------- textbook limits
@pytest.mark.parametrize("mode,n,na,nb", [("spin_orbitals", 6, 3, 2), ("spinors", 8, 3, 0)])
def test_one_body_limit_spectrum(mode, n, na, nb):
    """With (pq|rs) = 0 every FCI eigenvalue is a sum of occupied orbital energies
    (eigenvalues of h): the full spectrum must equal all such sums."""
    w = _small(7, mode, n, na, nb)
    h = w.ints.h
    eri = np.zeros((n,) * 4, dtype=h.dtype)
    Ho = _oracle_dense(mode, n, h, eri, w.keys)
    ev = np.linalg.eigvalsh(h)
    if mode == "spinors":
        sums = [sum(c) for c in itertools.combinations(ev, na)]
    else:
        sums = [sum(a) + sum(b) for a in itertools.combinations(ev, na) for b in itertools.combinations(ev, nb)]
    assert np.allclose(np.sort(np.linalg.eigvalsh(Ho)), np.sort(sums), atol=1e-12)


@pytest.mark.parametrize("mode,n,na,nb", [("spin_orbitals", 7, 3, 2), ("spinors", 9, 4, 0)])
def test_single_determinant_energy_density_matrix_form(mode, n, na, nb):
    """<D|H|D> against the textbook density-matrix expression
    E = tr(h g) + 1/2 sum (pq|rs) (g_qp g_sr - g_sp g_qr), g = projector on occupied
    spin-orbitals, evaluated by tensor contraction over all spin-orbitals."""
    w = _small(9, mode, n, na, nb, frac=0.3)
    o = Oracle.from_workload(w)
    diag = o.diagonal()
    hs, es = _so_ints(w)
    norb = hs.shape[0]
    for I in range(0, w.M, max(1, w.M // 15)):
        occ = [p for p in range(norb) if (int(w.keys[I]) >> p) & 1]
        g = np.zeros((norb, norb))
        g[occ, occ] = 1.0
        e = (np.einsum("pq,qp->", hs, g) + 0.5 * np.einsum("pqrs,qp,sr->", es, g, g)
             - 0.5 * np.einsum("pqrs,sp,qr->", es, g, g))
        assert abs(diag[I] - e) < 1e-12


# ---------------------------------------------------------------- invariances
@pytest.mark.parametrize("mode,n,na,nb", [("spin_orbitals", 5, 2, 2), ("spinors", 7, 3, 0)])
def test_orbital_rotation_invariance(mode, n, na, nb):
    """A unitary (real: orthogonal) rotation of the orbitals leaves the FCI spectrum
    unchanged; any inconsistency among diagonal, single and double elements breaks it."""
    w = _small(13, mode, n, na, nb)
    h, eri = w.ints.h, w.ints.eri()
    U = _random_unitary(np.random.default_rng(1), n, mode == "spinors")
    h2, e2 = _rotate(h, eri, U)
    if mode == "spin_orbitals":
        h2, e2 = h2.real, e2.real
    ev1 = np.linalg.eigvalsh(_oracle_dense(mode, n, h, eri, w.keys))
    ev2 = np.linalg.eigvalsh(_oracle_dense(mode, n, h2, e2, w.keys))
    assert np.abs(ev1 - ev2).max() < 1e-10


@pytest.mark.parametrize("mode,n,na,nb", [("spin_orbitals", 6, 3, 2), ("spinors", 8, 3, 0)])
def test_orbital_permutation_on_selected_space(mode, n, na, nb):
    """Relabel orbitals by a permutation pi on a selected (non-FCI) space: the relabelled
    list, re-sorted, with permuted integrals gives the same spectrum.  Pins the phases and
    their interplay with the sort order, which the relabelling reshuffles."""
    w = _small(17, mode, n, na, nb, frac=0.45)
    h, eri = w.ints.h, w.ints.eri()
    perm = np.random.default_rng(2).permutation(n)       # orbital p -> perm[p]
    inv = np.argsort(perm)
    h2 = h[np.ix_(inv, inv)]
    e2 = eri[np.ix_(inv, inv, inv, inv)]
    norb = n if mode == "spinors" else 2 * n
    bitmap = perm if mode == "spinors" else np.concatenate([perm, perm + n])
    new = []
    for k in w.keys:
        k = int(k)
        new.append(sum(1 << int(bitmap[p]) for p in range(norb) if (k >> p) & 1))
    keys2 = np.sort(np.array(new, dtype=np.uint64))
    ev1 = np.linalg.eigvalsh(_oracle_dense(mode, n, h, eri, w.keys))
    ev2 = np.linalg.eigvalsh(_oracle_dense(mode, n, h2, e2, keys2))
    assert np.abs(ev1 - ev2).max() < 1e-10


@pytest.mark.parametrize("mode,n,na,nb,frac", [("spin_orbitals", 6, 3, 3, 0.5), ("spinors", 8, 3, 0, 0.6)])
def test_hermiticity(mode, n, na, nb, frac):
    w = _small(19, mode, n, na, nb, frac=frac)
    H = Oracle.from_workload(w).dense()
    assert np.abs(H - H.conj().T).max() < 1e-14


# ---------------------------------------------------------------- independent routes
@pytest.mark.parametrize("mode,n,na,nb,frac", [
    ("spin_orbitals", 4, 2, 1, 1.0), ("spin_orbitals", 5, 2, 2, 0.6),
    ("spinors", 7, 3, 0, 1.0), ("spinors", 8, 3, 0, 0.5)])
def test_operator_route_matches_oracle(mode, n, na, nb, frac):
    """H assembled literally from Eq. Hamiltonian (no Slater-Condon rules) equals the
    oracle's Slater-Condon H element by element."""
    w = _small(23, mode, n, na, nb, frac=frac)
    hs, es = _so_ints(w)
    Hf = F.hamiltonian(w.keys, hs, es)
    Ho = Oracle.from_workload(w).dense()
    assert np.abs(Hf - Ho).max() < 1e-12


@pytest.mark.parametrize("mode,n,na,nb", [("spin_orbitals", 4, 2, 2), ("spinors", 6, 3, 0)])
def test_decomposition_identity(mode, n, na, nb):
    """Eq. decompositionH, with the exchange coefficient of H_2^0 read as (ij|ji),
    reproduces Eq. Hamiltonian; the printed coefficient (ij|jj) does not."""
    w = _small(29, mode, n, na, nb)
    hs, es = _so_ints(w)
    Hf = F.hamiltonian(w.keys, hs, es)
    Hd = F.hamiltonian_decomposed(w.keys, hs, es)
    assert np.abs(Hf - Hd).max() < 1e-12
    Hp = F.hamiltonian_decomposed(w.keys, hs, es, printed_h20=True)
    assert np.abs(Hf - Hp).max() > 1e-3


@pytest.mark.parametrize("mode,n,na,nb,frac", [
    ("spin_orbitals", 6, 3, 2, 0.4), ("spinors", 9, 4, 0, 0.3), ("spin_orbitals", 7, 3, 3, 0.15)])
def test_brute_force_matches_generation(mode, n, na, nb, frac):
    """All-pairs enumeration (every J tested by counting differing bits) and
    generation + lookup give the same sigma, nvec = 3."""
    w = _small(31, mode, n, na, nb, frac=frac)
    o = Oracle.from_workload(w)
    rng = np.random.default_rng(3)
    C = rng.normal(size=(w.M, 3)) + (1j * rng.normal(size=(w.M, 3)) if mode == "spinors" else 0)
    rows = np.arange(w.M)
    S1 = o.sigma_rows(rows, C)
    S2 = o.sigma_brute_rows(rows, C)
    assert np.abs(S1 - S2).max() < 1e-12 * max(1.0, np.abs(S1).max())


def test_brute_force_matches_generation_selected_30o():
    """The same on sampled rows of a 60,000-determinant selected space of the 30-orbital
    workload (all singles/doubles plus random triples/quadruples)."""
    w = W.selected_30o(M=60000)
    o = Oracle.from_workload(w)
    rows = np.sort(np.random.default_rng(4).choice(w.M, 24, replace=False))
    rows[0] = 0
    S1 = o.sigma_rows(rows, w.c)
    S2 = o.sigma_brute_rows(rows, w.c)
    assert np.abs(S1 - S2).max() < 1e-13


# ---------------------------------------------------------------- combinatorial counts
def test_pair_count_fci_8o():
    """Full CI, 8 orbitals, 4+4: each determinant connects to 16+16 singles, 36+36
    same-spin doubles and 16*16 opposite-spin doubles: 360 * 4900 ordered pairs."""
    w = W.fci_small_8o()
    assert w.M == 4900
    assert Oracle.from_workload(w).count_pairs() == 4900 * 360


@pytest.mark.parametrize("which", ["30o", "64s"])
def test_reference_row_connects_to_every_single_and_double(which):
    """The reference determinant of the selected spaces connects to all of its singles
    and doubles, which are all in the list: 10*20*2 + 2*C(10,2)C(20,2) + (10*20)^2 =
    57,500 (30 orbitals, 10+10) and 14*50 + C(14,2)C(50,2) = 112,175 (64 spinors, 14)."""
    w = W.selected_30o(M=60000) if which == "30o" else W.selected_spinor_64(M=120000)
    o = Oracle.from_workload(w)
    row = int(np.searchsorted(w.keys, w.hf_key()))
    J, deg, ph = o.connections(row)
    expected = 57500 if which == "30o" else 112175
    assert len(J) == expected
    n1 = 400 if which == "30o" else 700
    assert int((deg == 1).sum()) == n1 and int((deg == 2).sum()) == expected - n1
    assert set(np.unique(ph)) <= {-1, 1}


def _spin_swap(keys, n):
    """Exchange the alpha bits [0, n) and the beta bits [n, 2n) of every key."""
    keys = np.asarray(keys, dtype=np.uint64)
    mask = np.uint64((1 << n) - 1)
    return (keys >> np.uint64(n)) | ((keys & mask) << np.uint64(n))


@pytest.mark.parametrize("n,ne,frac", [(6, 3, 0.45), (7, 2, 0.6)])
def test_alpha_beta_swap_symmetry(n, ne, frac):
    """With spin-free integrals and n_alpha = n_beta, exchanging the spin labels maps H to
    itself: S|D> = (-1)^(n_alpha n_beta) |swap D> with the same sign for every D, so on a
    space closed under the swap sigma(P c) = P sigma(c) for the permutation P of the
    determinants.  A spin-dependent slip (an exchange term kept between opposite spins,
    an alpha-beta phase that depends on the spin order) breaks it."""
    w = _small(500 + n, "spin_orbitals", n, ne, ne, frac=frac)
    keys = np.unique(np.concatenate([w.keys, _spin_swap(w.keys, n)]))
    assert len(keys) > len(w.keys)                         # the closure added determinants
    o = Oracle("spin_orbitals", n, w.ints.h, w.ints.eri(), keys)
    perm = np.searchsorted(keys, _spin_swap(keys, n))
    assert np.array_equal(keys[perm], _spin_swap(keys, n))
    rng = np.random.default_rng(n)
    c = rng.normal(size=(len(keys), 2))
    pc = np.empty_like(c)
    pc[perm] = c
    s, ps = o.sigma(c), o.sigma(pc)
    assert np.abs(ps[perm] - s).max() < 1e-12 * np.abs(s).max()


@pytest.mark.parametrize("mode,n,na,nb,frac", [("spin_orbitals", 5, 2, 2, 0.7), ("spinors", 7, 3, 0, 0.5)])
def test_sigma_abs_rows_matches_literal_route(mode, n, na, nb, frac):
    """The magnitude row sums A = |H| |C| (the scale of sigma's rounding errors) against
    the dense H of the literal operator route, and |sigma| <= A row by row."""
    w = W.random_small(71 + n, mode, n, na, nb, naux=4, frac=frac, nvec=3)
    Hf = F.hamiltonian(w.keys, *_so_ints(w))
    o = Oracle.from_workload(w)
    rows = np.arange(w.M)
    A = o.sigma_abs_rows(rows, w.c)
    ref = np.abs(Hf) @ np.abs(w.c)
    assert np.allclose(A, ref, rtol=1e-13, atol=1e-15)
    assert np.all(np.abs(o.sigma(w.c)) <= A * (1 + 1e-12) + 1e-15)
    # equality when every term of a row has one sign: c >= 0 against |H|'s own signs
    c = np.sign(Hf[0]).real.astype(np.float64) if mode == "spin_orbitals" else None
    if c is not None:
        c[c == 0] = 1.0
        assert abs(abs(o.sigma_rows([0], c)[0, 0]) - o.sigma_abs_rows([0], c)[0, 0]) < 1e-12
