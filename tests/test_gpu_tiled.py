"""The tiled walk of large (N-2) buckets (sci_set_tile_threshold): buckets of more than the
threshold's members are walked by k_doubles_tiled, their members streamed through shared
memory in column tiles, and the rest by the window kernels.

With the threshold lowered so that most or all buckets take the tiled kernel, sigma in
every precision mode equals the oracle on sampled rows (1e-11; FP32 storage within its
per-row bound) and the default sigma (1e-13), on one-, two- and three-word spin-orbital
spaces and a complex 64-spinor space; the deterministic mode stays bit for bit
reproducible; row ranges concatenate to the whole-list sigma.  The full two-electron
space of 136 spinors, whose single (N-2) bucket holds all 9,180 determinants (past any
shared-memory window), runs by default and matches the closed form.
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


def _spaces():
    return {
        "sel_30o_cut": lambda: W.selected_30o_cut(M=3000, seed=11),
        "sel2w_40o": lambda: W.selected_two_word(n=40, na=3, nb=3, M=17000, nvec=2),
        "sel3w_70o": lambda: W.selected_three_word(n=70, na=3, nb=3, M=60000, nvec=2),
        "sel_64s_cut": lambda: W.selected_spinor_64_cut(),
    }


@pytest.fixture(scope="module", params=list(_spaces()))
def space(request):
    w = _spaces()[request.param]()
    return w, Oracle.from_workload(w)


def _rows(M, k=400, seed=0):
    r = np.random.default_rng(seed).choice(M, min(k, M), replace=False)
    return np.unique(np.concatenate([r, [0, M - 1]]))


@pytest.mark.parametrize("threshold", [1, 6, 40])
def test_tiled_sigma_all_precisions(gpu, space, threshold):
    torch = gpu
    w, o = space
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    cplx = np.iscomplexobj(w.c)
    ref_default = H.sigma(C).cpu().numpy()
    pairs = H.count_pairs()
    H.set_tile_threshold(threshold)
    assert H.count_pairs() == pairs
    rows = _rows(w.M)
    ref = o.sigma_rows(rows, w.c)
    S = H.sigma(C).cpu().numpy()
    assert _rel(S[rows], ref) < TOL
    assert _rel(S, ref_default) < 1e-13
    assert _rel(H.sigma(C, prec=sci.SCI_PREC_F64_DS).cpu().numpy()[rows], ref) < TOL
    if not cplx:
        C32 = np.ascontiguousarray(w.c, dtype=np.float32)
        S32 = H.sigma(torch.from_numpy(C32).cuda(), prec=sci.SCI_PREC_F32_STORE_F64_ACC).cpu().numpy()
        ref32 = o.sigma_rows(rows, C32.astype(np.float64))
        A = o.sigma_abs_rows(rows, C32.astype(np.float64))
        assert (np.abs(S32[rows] - ref32) <= 1.05 * 2.0 ** -24 * A + 1e-300).all()
    # eight vectors (the window kernels' widest group) through the tiled kernel
    rng = np.random.default_rng(5)
    C8 = rng.standard_normal((w.M, 8)) + (1j * rng.standard_normal((w.M, 8)) if cplx else 0)
    S8 = H.sigma(torch.from_numpy(C8).cuda()).cpu().numpy()
    assert _rel(S8[rows], o.sigma_rows(rows, C8)) < TOL
    H.set_tile_threshold(0)
    assert _rel(H.sigma(C).cpu().numpy(), ref_default) < 1e-13
    H.sync_status()


def test_tiled_deterministic_and_row_ranges(gpu, space):
    from paper_2501_18185_gb300.partition import balanced_ranges, row_weights
    torch = gpu
    w, o = space
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    H.set_tile_threshold(4)
    full = H.sigma(C).cpu().numpy()
    ranges = balanced_ranges(row_weights(H.row_costs().cpu().numpy(), 28), 3)
    S = np.zeros_like(full)
    for b, e in ranges:
        H.set_row_range(b, e)
        St = torch.full(C.shape, 7.0, dtype=C.dtype, device="cuda")
        H.sigma(C, out=St)
        Sn = St.cpu().numpy()
        assert (Sn[:b] == 7.0).all() and (Sn[e:] == 7.0).all()
        S[b:e] = Sn[b:e]
    H.set_row_range(0, w.M)
    assert _rel(S, full) < 1e-12
    H.set_deterministic(w.c.shape[1])
    a, b_ = H.sigma(C).cpu().numpy(), H.sigma(C).cpu().numpy()
    assert np.array_equal(a, b_) and _rel(a, full) < 1e-13
    # the deterministic result does not depend on which kernel walked a bucket
    H.set_tile_threshold(0)
    d0 = H.sigma(C).cpu().numpy()
    assert _rel(d0, a) < 1e-13
    H.sync_status()


def test_one_bucket_of_all_9180_pairs_of_136_spinors(gpu):
    """Two electrons in 136 complex spinors, every pair: one (N-2) bucket (the empty string)
    of 9,180 members, far above any shared-memory window: sigma by the tiled kernel
    (default threshold) against the closed form, FP64 and paired FP32, two vectors, and the
    deterministic mode bit for bit."""
    torch = gpu
    n = 136
    ints = W.complex_integrals(np.random.default_rng(93), n, 6, 0.9)
    pairs = np.array([(p, q) for q in range(n) for p in range(q)])
    keys = W.words_from_occ(pairs, 3)
    H = sci.Hamiltonian()
    H.set_integrals("spinors", ints.h, chol=ints.chol)
    H.set_determinants(keys, 2, -1)
    assert H.info()["max_bucket"] >= len(pairs)
    rng = np.random.default_rng(94)
    c = rng.standard_normal((len(pairs), 2)) + 1j * rng.standard_normal((len(pairs), 2))
    ref = spinor_pair_sigma(ints.h, ints.chol, pairs, c)
    C = torch.from_numpy(c).cuda()
    assert _rel(H.sigma(C).cpu().numpy(), ref) < TOL
    assert _rel(H.sigma(C, prec=sci.SCI_PREC_F64_DS).cpu().numpy(), ref) < TOL
    assert H.count_pairs() == len(pairs) * (len(pairs) - 1)
    H.set_deterministic(2)
    a, b = H.sigma(C).cpu().numpy(), H.sigma(C).cpu().numpy()
    assert np.array_equal(a, b) and _rel(a, ref) < TOL
    H.sync_status()


def test_tile_threshold_errors(gpu):
    """A threshold outside [0, 65535] is refused; one that would leave the 9,180-member
    bucket of the full 136-spinor pair space to the window kernels (past a one-vector
    complex window) is refused, and the previous threshold stays in force."""
    torch = gpu
    n = 136
    ints = W.complex_integrals(np.random.default_rng(95), n, 4, 0.9)
    pairs = np.array([(p, q) for q in range(n) for p in range(q)])
    H = sci.Hamiltonian()
    H.set_integrals("spinors", ints.h, chol=ints.chol)
    H.set_determinants(W.words_from_occ(pairs, 3), 2, -1)
    c = np.random.default_rng(96).standard_normal((len(pairs), 1)) + 0j
    C = torch.from_numpy(c).cuda()
    ref = spinor_pair_sigma(ints.h, ints.chol, pairs, c)
    with pytest.raises(sci.SciError):
        H.set_tile_threshold(-1)
    with pytest.raises(sci.SciError):
        H.set_tile_threshold(1 << 16)
    with pytest.raises(sci.SciError):
        H.set_tile_threshold(65535)
    assert _rel(H.sigma(C).cpu().numpy(), ref) < TOL
    H.set_tile_threshold(500)
    assert _rel(H.sigma(C).cpu().numpy(), ref) < TOL
    H.sync_status()


@pytest.mark.parametrize("npairs", [513, 1025])
def test_tile_edges_ragged_row_and_column_tiles(gpu, npairs):
    """Two electrons in 60 complex spinors on npairs random pairs: one (N-2) bucket of 513
    (row tiles of 256, 256 and 1) or 1,025 members (five row tiles, and two column tiles of
    1,024 and 1 split over two CTA rows), against the closed form with one and four
    vectors, FP64 and paired FP32; the window walk (threshold npairs) agrees, and the
    deterministic mode (one CTA per row tile) is bit for bit reproducible."""
    torch = gpu
    n = 60
    ints = W.complex_integrals(np.random.default_rng(131), n, 4, 0.9)
    rng = np.random.default_rng(132)
    allp = np.array([(p, q) for q in range(n) for p in range(q)])
    pairs = allp[np.sort(rng.choice(len(allp), npairs, replace=False))]
    keys = np.array([(1 << int(p)) | (1 << int(q)) for p, q in pairs], dtype=np.uint64)
    H = sci.Hamiltonian()
    H.set_integrals("spinors", ints.h, chol=ints.chol)
    H.set_determinants(keys, 2, -1)
    assert H.info()["max_bucket"] == npairs
    H.set_tile_threshold(npairs - 1)           # the one bucket is tiled
    for nv in (1, 4):
        c = rng.standard_normal((npairs, nv)) + 1j * rng.standard_normal((npairs, nv))
        ref = spinor_pair_sigma(ints.h, ints.chol, pairs, c)
        C = torch.from_numpy(c).cuda()
        S = H.sigma(C).cpu().numpy()
        assert _rel(S, ref) < TOL
        assert _rel(H.sigma(C, prec=sci.SCI_PREC_F64_DS).cpu().numpy(), ref) < TOL
        H.set_tile_threshold(npairs)           # the window walk
        assert _rel(H.sigma(C).cpu().numpy(), S) < 1e-13
        H.set_tile_threshold(npairs - 1)
    H.set_deterministic(4)
    a, b = H.sigma(C).cpu().numpy(), H.sigma(C).cpu().numpy()
    assert np.array_equal(a, b) and _rel(a, ref) < TOL
    H.sync_status()
