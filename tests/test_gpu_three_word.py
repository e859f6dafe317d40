"""Determinants of more than 128 spin-orbitals (three-word keys, sci_set_determinants_w with
nwords = 3) against the oracle, which holds every string as an array of three 64-bit
words, and against closed forms.

The selected 70-orbital space (140 spin-orbitals: the alpha string crosses words 0/1, the
beta string words 1/2): connections, degrees and phases bit-exact, per-row pair counts
exact, the diagonal to 1e-12, FP64 and paired-FP32 sigma to 1e-11, FP32-storage sigma
within its per-row bound, the deterministic mode bit for bit, row ranges concatenating to
the whole-list sigma.  One- and two-electron spaces of 136 complex spinors against the
closed forms; one- and two-word spaces given as three words against their own encodings.
"""
import numpy as np
import pytest

from closed_forms import spinor_pair_sigma
from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def sel3w():
    w = W.selected_three_word(n=70, na=3, nb=3, M=60000, nvec=3)
    return w, Oracle.from_workload(w)


def _rows(w, k=600, seed=0):
    r = np.random.default_rng(seed).choice(w.M, k, replace=False)
    return np.unique(np.concatenate([r, [0, w.M - 1]]))


def test_three_word_connections_counts_and_diagonal(gpu, sel3w):
    w, o = sel3w
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
    H.sync_status()


def test_three_word_sigma_all_precisions(gpu, sel3w):
    torch = gpu
    w, o = sel3w
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


def test_three_word_row_ranges(gpu, sel3w):
    """Row ranges on three-word lists (range tables with 24-byte spectator strings): K = 3
    cost-balanced ranges concatenate to the whole-list sigma (FP64 and paired FP32), the
    rows outside a range stay untouched, and the range pair counts sum to the total."""
    from paper_2501_18185_gb300.partition import balanced_ranges, row_weights
    torch = gpu
    w, o = sel3w
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    for prec in (sci.SCI_PREC_F64, sci.SCI_PREC_F64_DS):
        full = H.sigma(C, prec=prec).cpu().numpy()
        ranges = balanced_ranges(row_weights(H.row_costs().cpu().numpy(), 28), 3)
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


def test_three_word_encodings_of_one_and_two_word_spaces(gpu):
    """A one-word space and a two-word space given as three words (top words 0) give the
    sigma of their own encodings."""
    torch = gpu
    w = W.random_small(31, "spin_orbitals", 6, 3, 2, naux=4, frac=0.5)
    z = np.zeros_like(w.keys)
    H1 = sci.Hamiltonian.from_workload(w)
    H3 = sci.Hamiltonian()
    H3.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    H3.set_determinants(np.stack([w.keys, z, z], axis=1), w.n_alpha, w.n_beta)
    C = torch.from_numpy(w.c).cuda()
    assert _rel(H3.sigma(C).cpu().numpy(), H1.sigma(C).cpu().numpy()) < 1e-14
    w2 = W.selected_two_word(n=40, na=3, nb=3, M=17000)
    H2 = sci.Hamiltonian.from_workload(w2)
    H3 = sci.Hamiltonian()
    H3.set_integrals(w2.mode, w2.ints.h, chol=w2.ints.chol)
    H3.set_determinants(np.concatenate([w2.keys, np.zeros((w2.M, 1), dtype=np.uint64)], axis=1), 3, 3)
    C = torch.from_numpy(w2.c).cuda()
    assert H3.count_pairs() == H2.count_pairs()
    assert _rel(H3.sigma(C).cpu().numpy(), H2.sigma(C).cpu().numpy()) < 1e-14
    H3.sync_status()


def test_three_word_spinors_one_and_two_electrons(gpu):
    """136 complex spinors (bits 0..135 over three words): one electron, sigma = h c; two
    electrons on 4,000 of the 9,180 pairs (the whole pair space, one (N-2) bucket of 9,180
    members, is a case of the tiled-walk tests), sigma against the closed form with the
    Cholesky factors (no dense integrals; coefficients outside the list are zero), two
    vectors, FP64 and paired FP32."""
    torch = gpu
    n = 136
    ints = W.complex_integrals(np.random.default_rng(91), n, 6, 0.9)
    rng = np.random.default_rng(92)
    one = W.words_from_occ(np.arange(n)[:, None], 3)
    H = sci.Hamiltonian()
    H.set_integrals("spinors", ints.h, chol=ints.chol)
    H.set_determinants(one, 1, -1)
    c1 = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    ref1 = ints.h @ c1
    assert _rel(H.sigma(torch.from_numpy(c1).cuda()).cpu().numpy(), ref1) < 1e-13
    allp = np.array([(p, q) for q in range(n) for p in range(q)])
    pairs = allp[np.sort(rng.choice(len(allp), 4000, replace=False))]
    keys = W.words_from_occ(pairs, 3)
    keys_sorted = W.sort_words(keys)
    assert np.array_equal(keys_sorted, keys)       # q major is ascending
    H.set_determinants(keys, 2, -1)
    c2 = rng.standard_normal((len(pairs), 2)) + 1j * rng.standard_normal((len(pairs), 2))
    ref2 = spinor_pair_sigma(ints.h, ints.chol, pairs, c2)
    C2 = torch.from_numpy(c2).cuda()
    assert _rel(H.sigma(C2).cpu().numpy(), ref2) < TOL
    assert _rel(H.sigma(C2, prec=sci.SCI_PREC_F64_DS).cpu().numpy(), ref2) < TOL
    assert H.count_pairs() == len(pairs) * (len(pairs) - 1)
    H.sync_status()


def test_three_word_full_size_sampled(gpu):
    """A 140 spin-orbital space of bench size (70 orbitals, 4 + 4 electrons, 1,000,000
    determinants): FP64 and paired-FP32 sigma on 1,000 sampled rows (plus the first, last and
    HF rows) against the oracle, connections of row blocks bit-exact, and the per-row
    connection counts summing to the pair count."""
    torch = gpu
    w = W.selected_three_word(n=70, na=4, nb=4, M=1_000_000)
    o = Oracle.from_workload(w)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    hf = w.meta["hf_words"]
    ihf = int(np.nonzero((w.keys == hf[None, :]).all(axis=1))[0][0])
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


def test_three_word_rdm12_and_grads(gpu):
    """Density matrices on 65 orbitals (130 spin-orbitals: alpha orbital 64 in word 1, beta
    orbitals 63 and 64 at bits 128 and 129 of word 2), 2 + 1 electrons, the 10,500
    determinants of HF, singles, doubles and triples, two weighted vectors, against the
    oracle's per-vector matrices (1e-12); the spin sums and the Cholesky contraction of
    sci_rdm_grads against numpy on them."""
    torch = gpu
    n = 65
    w = W.selected_three_word(n=n, na=2, nb=1, M=10500, naux=8, nvec=2)
    assert (w.keys[:, 2] != 0).any()
    o = Oracle.from_workload(w)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    wt = np.array([1.0, -0.5])
    g1, g2 = H.rdm12(C, weights=wt)
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    r1 = np.zeros_like(g1)
    r2 = np.zeros_like(g2)
    for k in range(2):
        a1, a2 = o.rdm12(w.c[:, k])
        r1 += wt[k] * a1
        r2 += wt[k] * a2
        del a2
    assert np.abs(g1 - r1).max() < 1e-12 * np.abs(r1).max()
    assert np.abs(g2 - r2).max() < 1e-12 * np.abs(r2).max()
    del g2
    gamma, Gamma, gL = H.rdm_grads(C, weights=wt, chol=torch.from_numpy(w.ints.chol.copy()).cuda(), Gamma=True)
    gr = r1[:n, :n] + r1[n:, n:]
    Gr = r2[:n, :n, :n, :n] + r2[:n, :n, n:, n:] + r2[n:, n:, :n, :n] + r2[n:, n:, n:, n:]
    del r2
    assert np.abs(gamma.cpu().numpy() - gr).max() < 1e-12 * np.abs(gr).max()
    assert np.abs(Gamma.cpu().numpy() - Gr).max() < 1e-12 * np.abs(Gr).max()
    L = w.ints.chol
    ref = (Gr.reshape(n * n, n * n) @ L.reshape(L.shape[0], n * n).T).T.reshape(L.shape[0], n, n)
    assert np.abs(gL.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    H.sync_status()


def test_three_word_rdm12_172_spin_orbitals_global_diagonal(gpu):
    """172 spin-orbitals (86 orbitals, 2 + 2 electrons, 40,000 determinants): the diagonal
    class's [norb]^2 sums no longer fit shared memory and go to global memory.  On the
    device: the energy identity sum h g1 + 1/2 sum (pq|rs) g2 = c^+ H c against sigma, the
    traces N and N(N - 1), and Hermiticity of g1."""
    torch = gpu
    n = 86
    w = W.selected_three_word(n=n, na=2, nb=2, M=40000, naux=6)
    H = sci.Hamiltonian.from_workload(w)
    c = torch.from_numpy(np.ascontiguousarray(w.c[:, 0])).cuda()
    c = c / torch.linalg.vector_norm(c)
    g1, g2 = H.rdm12(c.reshape(-1, 1))
    h = torch.from_numpy(w.ints.h).cuda()
    L = torch.from_numpy(w.ints.chol).cuda()
    eri = torch.einsum("Ppq,Prs->pqrs", L, L)
    E1 = (h * g1[:n, :n]).sum() + (h * g1[n:, n:]).sum()
    G = g2.reshape(2, n, 2, n, 2, n, 2, n)
    E2 = sum((eri * G[a, :, a, :, b, :, b, :]).sum() for a in range(2) for b in range(2))
    E = float(E1 + 0.5 * E2)
    ref = float((c * H.sigma(c)).sum())
    assert abs(E - ref) < 1e-11 * max(1.0, abs(ref))
    assert abs(float(torch.trace(g1)) - 4) < 1e-12
    assert abs(float(torch.einsum("pprr->", g2)) - 12) < 1e-10
    assert float((g1 - g1.T).abs().max()) < 1e-14
    H.sync_status()


def test_three_word_enpt2_spinors(gpu):
    """Complex spinor ENPT2 on 130 spinors (three-word keys; 3 electrons, HF and 300 random
    determinants): the whole-string batch code over three words, keys claimed by a 128-bit
    compare-and-swap of words 0-1 and a 64-bit one of word 2, H_II over three words; two
    roots against the oracle's sum over the deduplicated external determinants at 1e-10,
    the distinct count exact, and a small table (many batches) giving the same sums."""
    torch = gpu
    n, N = 130, 3
    ints = W.complex_integrals(np.random.default_rng(105), n, 4, 0.9)
    rng = np.random.default_rng(106)
    occ = {(0, 1, 2)}
    while len(occ) < 301:
        occ.add(tuple(sorted(rng.choice(n, N, replace=False))))
    keys = W.sort_words(W.words_from_occ(np.array(sorted(occ)), 3))
    assert (keys[:, 2] != 0).any()
    o = Oracle("spinors", n, ints.h, ints.eri(), keys)
    C = rng.standard_normal((len(keys), 2)) + 1j * rng.standard_normal((len(keys), 2))
    C /= np.linalg.norm(C, axis=0)
    d = o.diagonal().real
    E0 = np.array([d.min() - 1.0, d.min() - 2.0])
    E2, n_ext = o.enpt2(C, E0)
    n_conn = sum(1 for r in range(len(keys)) if len(o.connections(r)[0]) > 0)
    H = sci.Hamiltonian()
    H.set_integrals("spinors", ints.h, chol=ints.chol)
    H.set_determinants(keys, N, -1)
    Ct = torch.from_numpy(C).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0)
    assert np.allclose(e2q, E2, rtol=1e-10, atol=0), (e2q, E2)
    assert st["distinct_W"] == n_ext + n_conn
    b = H.enpt2(Ct, E0, table_bytes=(1 << 16) * 48)
    assert b[3]["batches"] > st["batches"] and b[3]["distinct_W"] == st["distinct_W"]
    assert np.allclose(b[2], E2, rtol=1e-10, atol=0)
    H.sync_status()


@pytest.mark.parametrize("n,m", [(70, 1500), (90, 500)])
def test_three_word_enpt2_spin_orbitals(gpu, n, m):
    """Real spin-orbital ENPT2 on 70 and 90 orbitals (three-word keys: the alpha string
    crosses words 0/1 and the beta string words 1/2; the generator holds each as two words;
    at 180 spin-orbitals the evaluation reads G from global memory), 2 alpha + 1 beta
    electrons, HF and m random determinants: two roots against the oracle's sum over the
    deduplicated external determinants at 1e-10, the distinct count exact, and a small
    table (many batches) giving the same sums."""
    torch = gpu
    na, nb = 2, 1
    ints = W.real_integrals(np.random.default_rng(107), n, 4, 0.95)
    rng = np.random.default_rng(108)
    occ = {((0, 1), (0,))}
    while len(occ) < m + 1:
        occ.add((tuple(sorted(rng.choice(n, na, replace=False))), tuple(sorted(rng.choice(n, nb, replace=False)))))
    occ = np.array([list(a) + [b[0] + n] for a, b in sorted(occ)])
    keys = W.sort_words(W.words_from_occ(occ, 3))
    assert (keys[:, 2] != 0).any() and (keys[:, 1] != 0).any()
    o = Oracle("spin_orbitals", n, ints.h, ints.eri(), keys)
    C = rng.standard_normal((len(keys), 2))
    C /= np.linalg.norm(C, axis=0)
    d = o.diagonal()
    E0 = np.array([d.min() - 1.0, d.min() - 2.0])
    E2, n_ext = o.enpt2(C, E0)
    n_conn = sum(1 for r in range(len(keys)) if len(o.connections(r)[0]) > 0)
    H = sci.Hamiltonian()
    H.set_integrals("spin_orbitals", ints.h, chol=ints.chol)
    H.set_determinants(keys, na, nb)
    Ct = torch.from_numpy(C).cuda()
    e2w, e2p, e2q, st = H.enpt2(Ct, E0)
    assert np.allclose(e2q, E2, rtol=1e-10, atol=0), (e2q, E2)
    assert st["distinct_W"] == n_ext + n_conn
    b = H.enpt2(Ct, E0, table_bytes=(1 << 15) * 32)
    assert b[3]["batches"] > st["batches"] and b[3]["distinct_W"] == st["distinct_W"]
    assert np.allclose(b[2], E2, rtol=1e-10, atol=0)
    H.sync_status()


def test_three_word_limits_and_rejections(gpu, sel3w):
    """Keys of too few words for the orbital count and keys out of 192-bit order are
    refused with an error, never a wrong result."""
    torch = gpu
    w, o = sel3w
    H = sci.Hamiltonian.from_workload(w)
    with pytest.raises(sci.SciError):            # 140 spin-orbitals need three words
        sci.sci_set_determinants_w(H.ctx, np.ascontiguousarray(w.keys[:, :2]), 2, w.M, 3, 3, 0)
    bad = w.keys.copy()
    bad[[3, 4]] = bad[[4, 3]]
    with pytest.raises(sci.SciError):
        H.set_determinants(bad, 3, 3)            # not ascending as 192-bit integers
    H.set_determinants(w.keys, 3, 3)
    assert _rel(H.sigma(torch.from_numpy(np.ascontiguousarray(w.c)).cuda()).cpu().numpy()[:5],
                o.sigma_rows(np.arange(5), w.c)) < TOL
    H.sync_status()


def test_three_word_edge_cases(gpu):
    """An empty three-word list, and one determinant with bits in all three words: sigma is
    H_II c (no pairs)."""
    torch = gpu
    n = 70
    ints = W.real_integrals(np.random.default_rng(73), n, 4, 0.95)
    H = sci.Hamiltonian()
    H.set_integrals("spin_orbitals", ints.h, chol=ints.chol)
    H.set_determinants(np.zeros((0, 3), dtype=np.uint64), 1, 1)
    S = H.sigma(torch.zeros((0, 1), dtype=torch.float64, device="cuda"))
    assert S.shape[0] == 0 and H.count_pairs() == 0
    one = W.words_from_occ(np.array([[69, n + 69]]), 3)              # bits 69 and 139
    assert one[0, 0] == 0 and one[0, 1] != 0 and one[0, 2] != 0
    H.set_determinants(one, 1, 1)
    o = Oracle("spin_orbitals", n, ints.h, ints.eri(), one)
    S = H.sigma(torch.tensor([[0.5]], dtype=torch.float64, device="cuda")).cpu().numpy()
    d = o.diagonal()
    assert H.count_pairs() == 0 and abs(S[0, 0] - 0.5 * d[0]) < 1e-12 * abs(d[0])
    H.sync_status()
