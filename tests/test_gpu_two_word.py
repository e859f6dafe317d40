"""Determinants of more than 64 spin-orbitals (two-word keys, sci_set_determinants_w)
against the oracle, which holds every string as a 128-bit integer.

The selected 40-orbital space (80 spin-orbitals: beta strings cross the word boundary):
connections, degrees and phases bit-exact, per-row pair counts exact, the diagonal to 1e-12,
FP64 and paired-FP32 sigma to 1e-11, FP32-storage sigma within its per-row bound, the
deterministic mode bit for bit; the density matrices and their spin sums against the oracle.  The opposite-spin two-electron closed form on 40 orbitals
and a 72-spinor space are checked as dense matrices.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def sel2w():
    w = W.selected_two_word(n=40, na=4, nb=4, M=40000, nvec=3)
    return w, Oracle.from_workload(w)


def _rows(w, k=600, seed=0):
    r = np.random.default_rng(seed).choice(w.M, k, replace=False)
    return np.unique(np.concatenate([r, [0, w.M - 1]]))


def test_two_word_connections_counts_and_diagonal(gpu, sel2w):
    torch = gpu
    w, o = sel2w
    H = sci.Hamiltonian.from_workload(w)
    rows = _rows(w, 200)
    for r in rows[:60]:
        J, deg, ph = o.connections(int(r))
        got = H.connections(int(r), int(r) + 1)
        assert np.array_equal(got[1], J) and np.array_equal(got[2], deg) and np.array_equal(got[3], ph), r
    cost = H.row_costs().cpu().numpy()
    for r in rows:
        assert cost[r] == len(o.connections(int(r))[0])
    assert int(cost.sum()) == H.count_pairs()
    d = H.diagonal().cpu().numpy()
    ref = o.diagonal()
    assert np.abs(d - ref).max() < 1e-12 * np.abs(ref).max()


def test_two_word_sigma_all_precisions(gpu, sel2w):
    torch = gpu
    w, o = sel2w
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    rows = _rows(w)
    ref = o.sigma_rows(rows, w.c)
    assert _rel(H.sigma(C).cpu().numpy()[rows], ref) < TOL
    assert _rel(H.sigma(C, prec=sci.SCI_PREC_F64_DS).cpu().numpy()[rows], ref) < TOL
    # FP32 storage: within 2^-24 of each row's magnitude sum, against the oracle on the
    # FP32-rounded vectors (the pair table's one rounding)
    C32 = np.ascontiguousarray(w.c, dtype=np.float32)
    S32 = H.sigma(torch.from_numpy(C32).cuda(), prec=sci.SCI_PREC_F32_STORE_F64_ACC).cpu().numpy()
    ref32 = o.sigma_rows(rows, C32.astype(np.float64))
    A = o.sigma_abs_rows(rows, C32.astype(np.float64))
    assert (np.abs(S32[rows] - ref32) <= 1.05 * 2.0 ** -24 * A + 1e-300).all()
    # deterministic accumulation: bit for bit, and the atomic result to 1e-13
    at = H.sigma(C).cpu().numpy()
    H.set_deterministic(3)
    a, b = H.sigma(C).cpu().numpy(), H.sigma(C).cpu().numpy()
    assert np.array_equal(a, b) and _rel(a, at) < 1e-13
    H.sync_status()


def test_two_word_opposite_spin_closed_form_and_one_word_encoding(gpu):
    """1 alpha + 1 beta over 40 orbitals: H from sigma on the unit vectors equals
    h x 1 + 1 x h + V; and a one-word space given as two words gives the one-word sigma."""
    torch = gpu
    n = 40
    rng = np.random.default_rng(11)
    ints = W.real_integrals(rng, n, 6, 0.95)
    a = np.array([1 << p for q in range(n) for p in range(n)], dtype=np.uint64)
    b = np.array([1 << q for q in range(n) for p in range(n)], dtype=np.uint64)
    keys = W.sort_words(W.two_word_keys(a, b, n))
    H = sci.Hamiltonian()
    H.set_integrals("spin_orbitals", ints.h, chol=ints.chol)
    H.set_determinants(keys, 1, 1)
    E = torch.eye(n * n, dtype=torch.float64, device="cuda")
    Hd = H.sigma(E).cpu().numpy()
    h, eri = ints.h, ints.eri()
    expected = np.kron(np.eye(n), h) + np.kron(h, np.eye(n)) + eri.transpose(2, 0, 3, 1).reshape(n * n, n * n)
    assert np.abs(Hd - expected).max() < 1e-12 * np.abs(expected).max()
    # one-word space as two words
    w = W.random_small(31, "spin_orbitals", 6, 3, 2, naux=4, frac=0.5)
    H1 = sci.Hamiltonian.from_workload(w)
    H2 = sci.Hamiltonian()
    H2.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    H2.set_determinants(np.stack([w.keys, np.zeros_like(w.keys)], axis=1), w.n_alpha, w.n_beta)
    C = torch.from_numpy(w.c).cuda()
    assert _rel(H2.sigma(C).cpu().numpy(), H1.sigma(C).cpu().numpy()) < 1e-14


def test_two_word_spinors(gpu):
    """72 complex spinors, 3 electrons on a random subset: dense H by sigma against the
    oracle's dense H (elements by operator application)."""
    torch = gpu
    n, N = 72, 3
    rng = np.random.default_rng(21)
    ints = W.complex_integrals(rng, n, 5, 0.95)
    import itertools
    occ = [c for c in itertools.combinations(range(n), N) if rng.random() < 0.004 or c == (0, 1, 2)]
    lo = np.array([sum(1 << p for p in c if p < 64) for c in occ], dtype=np.uint64)
    hi = np.array([sum(1 << (p - 64) for p in c if p >= 64) for c in occ], dtype=np.uint64)
    keys = W.sort_words(np.stack([lo, hi], axis=1))
    o = Oracle("spinors", n, ints.h, ints.eri(), keys)
    H = sci.Hamiltonian()
    H.set_integrals("spinors", ints.h, chol=ints.chol)
    H.set_determinants(keys, N, -1)
    M = len(keys)
    E = torch.eye(M, dtype=torch.complex128, device="cuda")
    Hd = H.sigma(E).cpu().numpy()
    ref = o.dense()
    assert np.abs(Hd - ref).max() < 1e-12 * np.abs(ref).max()
    assert M > 200


def test_two_word_row_ranges(gpu, sel2w):
    """Row ranges on two-word lists (range tables with 16-byte spectator strings): K = 3 and
    5 cost-balanced ranges concatenate to the whole-list sigma (FP64 and paired FP32), the
    rows outside a range stay untouched, and the range pair counts sum to the total."""
    from paper_2501_18185_gb300.partition import balanced_ranges, row_weights
    torch = gpu
    w, o = sel2w
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    for prec in (sci.SCI_PREC_F64, sci.SCI_PREC_F64_DS):
        full = H.sigma(C, prec=prec).cpu().numpy()
        for K in (3, 5):
            ranges = balanced_ranges(row_weights(H.row_costs().cpu().numpy(), 28), K)
            S = np.zeros_like(full)
            pairs = 0
            for b, e in ranges:
                H.set_row_range(b, e)
                St = torch.full(C.shape, 7.0, dtype=torch.float64, device="cuda")
                H.sigma(C, out=St, prec=prec)
                Sn = St.cpu().numpy()
                assert (Sn[:b] == 7.0).all() and (Sn[e:] == 7.0).all()
                S[b:e] = Sn[b:e]
                pairs += H.info()["pairs"]
            H.set_row_range(0, w.M)
            assert _rel(S, full) < 1e-12
            assert pairs == H.count_pairs()
    H.sync_status()


def test_two_word_limits(gpu, sel2w):
    torch = gpu
    w, _ = sel2w
    H = sci.Hamiltonian.from_workload(w)
    with pytest.raises(sci.SciError):            # more than 64 spin-orbitals need two words
        sci.sci_set_determinants(H.ctx, np.ascontiguousarray(w.keys[:, 0]), w.M, 4, 4, 0)
    bad = w.keys.copy()
    bad[[3, 4]] = bad[[4, 3]]
    with pytest.raises(sci.SciError):
        H.set_determinants(bad, 4, 4)            # not ascending as 128-bit integers


def test_two_word_full_size_sampled(gpu):
    """The 80 spin-orbital bench space (40 orbitals, 8 + 8 electrons, 2,000,000 determinants)
    in the launch configuration the bench times: FP64 and paired-FP32 sigma on 1,000 sampled
    rows (plus the first, last and HF rows) against the oracle, connections of row blocks
    bit-exact, and the per-row connection counts summing to the pair count."""
    torch = gpu
    w = W.selected_two_word(n=40, na=8, nb=8, M=2_000_000)
    o = Oracle.from_workload(w)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    hf = W.two_word_keys(np.array([(1 << 8) - 1], dtype=np.uint64), np.array([(1 << 8) - 1], dtype=np.uint64), 40)[0]
    ihf = int(np.nonzero((w.keys[:, 0] == hf[0]) & (w.keys[:, 1] == hf[1]))[0][0])
    rows = np.unique(np.concatenate([np.random.default_rng(3).choice(w.M, 1000, replace=False), [0, ihf, w.M - 1]]))
    ref = o.sigma_rows(rows, w.c)
    S = H.sigma(C).cpu().numpy().reshape(w.M, -1)
    assert _rel(S[rows], ref) < TOL
    Sds = H.sigma(C, prec=sci.SCI_PREC_F64_DS).cpu().numpy().reshape(w.M, -1)
    assert _rel(Sds[rows], ref) < TOL
    for a, b in ((0, 100), (ihf, ihf + 1), (w.M // 2, w.M // 2 + 100), (w.M - 100, w.M)):
        _, J, deg, ph = H.connections(a, b)
        conn = [o.connections(r) for r in range(a, b)]
        assert np.array_equal(J, np.concatenate([x[0] for x in conn]))
        assert np.array_equal(deg, np.concatenate([x[1] for x in conn]))
        assert np.array_equal(ph, np.concatenate([x[2] for x in conn]))
    assert int(H.row_costs().sum()) == H.count_pairs()
    H.sync_status()


def test_two_word_rdm12_and_grads(gpu):
    """Density matrices on 40 orbitals (80 spin-orbitals, 2 + 2 electrons, 10,000 selected
    determinants), two weighted vectors, against the oracle's per-vector matrices; the spin
    sums and the Cholesky contraction of sci_rdm_grads against numpy on them."""
    torch = gpu
    w = W.selected_two_word(n=40, na=2, nb=2, M=10000, nvec=2)
    o = Oracle.from_workload(w)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    wt = np.array([1.0, -0.5])
    g1, g2 = H.rdm12(C, weights=wt)
    r1 = np.zeros((80, 80))
    r2 = np.zeros((80,) * 4)
    for k in range(2):
        a1, a2 = o.rdm12(w.c[:, k])
        r1 += wt[k] * a1
        r2 += wt[k] * a2
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    assert np.abs(g1 - r1).max() < 1e-12 * np.abs(r1).max()
    assert np.abs(g2 - r2).max() < 1e-12 * np.abs(r2).max()
    n = 40
    gamma, Gamma, gL = H.rdm_grads(C, weights=wt, chol=torch.from_numpy(w.ints.chol.copy()).cuda(), Gamma=True)
    gr = r1[:n, :n] + r1[n:, n:]
    Gr = (r2[:n, :n, :n, :n] + r2[:n, :n, n:, n:] + r2[n:, n:, :n, :n] + r2[n:, n:, n:, n:])
    assert np.abs(gamma.cpu().numpy() - gr).max() < 1e-12 * np.abs(gr).max()
    assert np.abs(Gamma.cpu().numpy() - Gr).max() < 1e-12 * np.abs(Gr).max()
    L = w.ints.chol
    ref = (Gr.reshape(n * n, n * n) @ L.reshape(L.shape[0], n * n).T).T.reshape(L.shape[0], n, n)
    assert np.abs(gL.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    H.sync_status()


def _enpt2_case(w, o, seed):
    """Normalised random vectors, E0 one below the lowest diagonal element, the oracle's
    E2 over Q (sciref_enpt2) and the members of P connected to another member.  E2[W] -
    E2[P] = E2[Q] holds for any c and E0 (Eqs. PT2final, EW1, EP1)."""
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((w.M, 2)) * (1.0 if not np.iscomplexobj(w.ints.h) else 1.0)
    if np.iscomplexobj(w.ints.h):
        C = C + 1j * rng.standard_normal((w.M, 2))
    C /= np.linalg.norm(C, axis=0)
    d = o.diagonal().real
    E0 = np.array([d.min() - 1.0, d.min() - 2.0])
    E2, n_ext = o.enpt2(C, E0)
    n_conn = sum(1 for r in range(w.M) if len(o.connections(r)[0]) > 0)
    return C, E0, E2, n_ext, n_conn


def test_two_word_enpt2_real(gpu):
    """ENPT2 on 40 orbitals (2 alpha + 1 beta electrons, 5,000 selected determinants; the
    beta string crosses the word boundary): 128-bit hash keys by 16-byte CAS, the beta
    batch code over 40 orbitals, H_II of the external determinants over both words; two
    roots against the oracle's direct sum at 1e-10, the distinct count exact, and a small
    table (many batches) giving the same sums."""
    torch = gpu
    w = W.selected_two_word(n=40, na=2, nb=1, M=5000)
    o = Oracle.from_workload(w)
    C, E0, E2, n_ext, n_conn = _enpt2_case(w, o, 11)
    H = sci.Hamiltonian.from_workload(w)
    Ct = torch.from_numpy(C).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0)
    assert np.allclose(e2q, E2, rtol=1e-10, atol=0), (e2q, E2)
    assert st["distinct_W"] == n_ext + n_conn
    b = H.enpt2(Ct, E0, table_bytes=(1 << 12) * 32)
    assert b[3]["batches"] > st["batches"] and b[3]["distinct_W"] == st["distinct_W"]
    assert np.allclose(b[2], E2, rtol=1e-10, atol=0)
    H.sync_status()


def test_two_word_enpt2_spinors(gpu):
    """Complex spinor ENPT2 on 72 spinors (3 electrons, HF and 600 random determinants):
    the whole-string batch code over both words, complex numerators; two roots against the
    oracle at 1e-10, the distinct count exact, and a small table giving the same sums."""
    torch = gpu
    import itertools
    n, N = 72, 3
    rng = np.random.default_rng(23)
    ints = W.complex_integrals(rng, n, 5, 0.95)
    allc = list(itertools.combinations(range(n), N))
    pick = [allc[0]] + [allc[i] for i in rng.choice(np.arange(1, len(allc)), 600, replace=False)]
    lo = np.array([sum(1 << p for p in c if p < 64) for c in pick], dtype=np.uint64)
    hi = np.array([sum(1 << (p - 64) for p in c if p >= 64) for c in pick], dtype=np.uint64)
    keys = W.sort_words(np.stack([lo, hi], axis=1))

    class _W:
        pass

    w = _W()
    w.M, w.ints, w.keys = len(keys), ints, keys
    o = Oracle("spinors", n, ints.h, ints.eri(), keys)
    C, E0, E2, n_ext, n_conn = _enpt2_case(w, o, 12)
    H = sci.Hamiltonian()
    H.set_integrals("spinors", ints.h, chol=ints.chol)
    H.set_determinants(keys, N, -1)
    Ct = torch.from_numpy(C).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0)
    assert np.allclose(e2q, E2, rtol=1e-10, atol=0), (e2q, E2)
    assert st["distinct_W"] == n_ext + n_conn
    b = H.enpt2(Ct, E0, table_bytes=(1 << 15) * 48)
    assert b[3]["batches"] > st["batches"] and b[3]["distinct_W"] == st["distinct_W"]
    assert np.allclose(b[2], E2, rtol=1e-10, atol=0)
    H.sync_status()


def test_two_word_edge_cases(gpu):
    """An empty two-word list, and one determinant: sigma is H_II c (no pairs), ENPT2 and
    the density matrices run."""
    torch = gpu
    n = 40
    ints = W.real_integrals(np.random.default_rng(71), n, 4, 0.95)
    H = sci.Hamiltonian()
    H.set_integrals("spin_orbitals", ints.h, chol=ints.chol)
    H.set_determinants(np.zeros((0, 2), dtype=np.uint64), 1, 1)
    S = H.sigma(torch.zeros((0, 1), dtype=torch.float64, device="cuda"))
    assert S.shape[0] == 0 and H.count_pairs() == 0
    one = W.two_word_keys(np.array([1], dtype=np.uint64), np.array([1 << 30], dtype=np.uint64), n)  # beta bit 70
    H.set_determinants(one, 1, 1)
    o = Oracle("spin_orbitals", n, ints.h, ints.eri(), one)
    c = torch.tensor([[0.5]], dtype=torch.float64, device="cuda")
    S = H.sigma(c).cpu().numpy()
    d = o.diagonal()
    assert H.count_pairs() == 0 and abs(S[0, 0] - 0.5 * d[0]) < 1e-12 * abs(d[0])
    E2, nx = o.enpt2(np.array([[1.0]]), [d[0].real - 1.0])
    e2w, e2p, e2q, st = H.enpt2(torch.tensor([[1.0]], dtype=torch.float64, device="cuda"), [d[0].real - 1.0])
    assert np.allclose(e2q, E2, rtol=1e-10, atol=0) and st["distinct_W"] == nx + 0
    g1, g2 = H.rdm12(torch.tensor([[1.0]], dtype=torch.float64, device="cuda"))
    r1, r2 = o.rdm12(np.array([1.0]))
    assert np.abs(g1.cpu().numpy() - r1).max() < 1e-14 and np.abs(g2.cpu().numpy() - r2).max() < 1e-14
    H.sync_status()
