"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Connection lists, excitation degrees and phases must match bit for bit; FP64 sigma must
match to 1e-11 relative in the 2-norm; the diagonal to 1e-12 relative.
"""
import json
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-11
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pair_counts.json")

CASES = {
    "fci_8o_4a4b": lambda: W.fci_small_8o(),
    "so_sel_7o": lambda: W.random_small(41, "spin_orbitals", 7, 3, 2, frac=0.5),
    "so_fci_10o_4a3b": lambda: W.random_small(43, "spin_orbitals", 10, 4, 3),
    "so_32o_1a1b": lambda: W.random_small(44, "spin_orbitals", 32, 1, 1, naux=3),
    "spinor_fci_12_4": lambda: W.random_small(47, "spinors", 12, 4, 0),
    "spinor_sel_16_5": lambda: W.random_small(53, "spinors", 16, 5, 0, frac=0.3),
    "spinor_64_2": lambda: W.random_small(59, "spinors", 64, 2, 0, naux=3),
    "sel_30o_60k": lambda: W.selected_30o(M=60000),
    "sel_64s_120k": lambda: W.selected_spinor_64(M=120000),
}
_cache = {}


def case(name):
    if name not in _cache:
        w = CASES[name]()
        _cache[name] = (w, Oracle.from_workload(w))
    return _cache[name]


def gpu_ham(w, torch):
    return sci.Hamiltonian.from_workload(w)


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# FP32 storage (SCI_PREC_F32_STORE_F64_ACC) against the FP64 oracle run on the FP32-rounded
# vectors.  With C already in FP32, the one rounding left is that of the pair table: each
# double-excitation element t = (ai|bj) - (aj|bi) is rounded to float once, |dt| <= 2^-24
# |t|; the products t32 * c32 are exact, the per-bucket sums compensated (errors ~2^-44 of
# the sum of magnitudes), singles and the diagonal FP64-accurate, accumulation FP64.  So
# row I of sigma is off by at most 2^-24 sum_J |t_IJ| |c_J| <= 2^-24 A_I, with
# A_I = |H_II c_I| + sum_J |H_IJ| |c_J| from the oracle.  The bound is asserted row by row
# and element by element, with 5% for the compensated sums and the FP64 atomics.
U32 = 2.0 ** -24


def assert_fp32_rows(S, C32, o, rows):
    ref = o.sigma_rows(rows, C32.astype(np.float64))
    A = o.sigma_abs_rows(rows, C32.astype(np.float64))
    err = np.abs(S[rows].reshape(ref.shape) - ref)
    bound = 1.05 * U32 * A + 1e-300
    worst = float((err / bound).max())
    assert worst <= 1.0, (worst, int(np.argmax((err / bound).max(axis=1))))
    return worst


def sample_rows(w, k, seed=0):
    if w.M <= k:
        return np.arange(w.M)
    r = np.random.default_rng(seed).choice(w.M, k, replace=False)
    hf = int(np.searchsorted(w.keys, w.hf_key()))
    extra = [0, w.M - 1] + ([hf] if hf < w.M and w.keys[hf] == w.hf_key() else [])
    return np.unique(np.concatenate([r, extra]))


@pytest.mark.parametrize("name", list(CASES))
def test_connections_bit_exact(gpu, name):
    w, o = case(name)
    H = gpu_ham(w, gpu)
    rb, re = (0, w.M) if w.M <= 6000 else (0, 1500)
    rows, J, deg, ph = H.connections(rb, re)
    ref = [o.connections(r) for r in range(rb, re)]
    rr = np.concatenate([np.full(len(x[0]), r) for r, x in zip(range(rb, re), ref)])
    assert np.array_equal(rows, rr)
    assert np.array_equal(J, np.concatenate([x[0] for x in ref]))
    assert np.array_equal(deg, np.concatenate([x[1] for x in ref]))
    assert np.array_equal(ph, np.concatenate([x[2] for x in ref]))
    if w.M > 6000:  # also the reference row and the last rows
        hf = int(np.searchsorted(w.keys, w.hf_key()))
        for a, b in ((hf, hf + 1), (w.M - 300, w.M)):
            rows, J, deg, ph = H.connections(a, b)
            ref = [o.connections(r) for r in range(a, b)]
            assert np.array_equal(J, np.concatenate([x[0] for x in ref]))
            assert np.array_equal(ph, np.concatenate([x[2] for x in ref]))


@pytest.mark.parametrize("name", list(CASES))
def test_pair_count(gpu, name):
    w, o = case(name)
    H = gpu_ham(w, gpu)
    if w.M <= 60000:
        assert H.count_pairs() == o.count_pairs()
    else:
        golden = json.load(open(GOLDEN)) if os.path.exists(GOLDEN) else {}
        if w.name in golden:
            assert H.count_pairs() == golden[w.name]["pairs"]


@pytest.mark.parametrize("name", list(CASES))
def test_diagonal(gpu, name):
    w, o = case(name)
    H = gpu_ham(w, gpu)
    d = H.diagonal().cpu().numpy()
    ref = o.diagonal().real
    assert rel_err(d, ref) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nvec", [1, 3])
def test_sigma_fp64(gpu, name, nvec):
    torch = gpu
    w, o = case(name)
    H = gpu_ham(w, torch)
    rng = np.random.default_rng(100 + nvec)
    C = w.c if nvec == 1 else rng.normal(size=(w.M, nvec)) + (1j * rng.normal(size=(w.M, nvec)) if w.mode == "spinors" else 0)
    C = np.ascontiguousarray(C)
    Ct = torch.from_numpy(C).cuda()
    S = H.sigma(Ct.reshape(w.M, -1)).cpu().numpy().reshape(w.M, -1)
    H.sync_status()
    rows = sample_rows(w, 3000)
    ref = o.sigma_rows(rows, C)
    assert rel_err(S[rows], ref) < TOL


@pytest.mark.parametrize("name", ["fci_8o_4a4b", "so_sel_7o", "spinor_sel_16_5", "spinor_64_2", "sel_30o_60k",
                                  "sel_64s_120k"])
@pytest.mark.parametrize("nvec", [1, 3])
def test_sigma_paired_fp32_matches_fp64_tolerance(gpu, name, nvec):
    """SCI_PREC_F64_DS (double-excitation products and bucket sums in paired FP32) is
    held to the same 1e-11 bar against the FP64 oracle as the FP64 path."""
    torch = gpu
    w, o = case(name)
    H = gpu_ham(w, torch)
    rng = np.random.default_rng(200 + nvec)
    C = w.c if nvec == 1 else rng.normal(size=(w.M, nvec)) + (1j * rng.normal(size=(w.M, nvec)) if w.mode == "spinors" else 0)
    C = np.ascontiguousarray(C)
    S = H.sigma(torch.from_numpy(C).cuda().reshape(w.M, -1), prec=sci.SCI_PREC_F64_DS).cpu().numpy().reshape(w.M, -1)
    H.sync_status()
    rows = sample_rows(w, 3000)
    assert rel_err(S[rows], o.sigma_rows(rows, C)) < TOL


@pytest.mark.parametrize("name", ["fci_8o_4a4b", "so_sel_7o", "sel_30o_60k"])
@pytest.mark.parametrize("nvec", [1, 8])
def test_sigma_fp32_storage(gpu, name, nvec):
    """SCI_PREC_F32_STORE_F64_ACC: C and the pair table in FP32, exact products,
    compensated sums.  Against the FP64 oracle run on the FP32-rounded C, every row and
    vector is within 2^-24 of its magnitude sum A_I (the table's one rounding; see
    assert_fp32_rows)."""
    torch = gpu
    w, o = case(name)
    H = gpu_ham(w, torch)
    rng = np.random.default_rng(300 + nvec)
    C = w.c if nvec == 1 else rng.normal(size=(w.M, nvec))
    C32 = np.ascontiguousarray(C, dtype=np.float32)
    S = H.sigma(torch.from_numpy(C32).cuda().reshape(w.M, -1),
                prec=sci.SCI_PREC_F32_STORE_F64_ACC).cpu().numpy().reshape(w.M, -1)
    H.sync_status()
    rows = sample_rows(w, 2000)
    assert_fp32_rows(S, C32, o, rows)


def test_sigma_nvec8_and_repeat(gpu):
    torch = gpu
    w, o = case("sel_30o_60k")
    H = gpu_ham(w, torch)
    C = np.random.default_rng(5).normal(size=(w.M, 8))
    Ct = torch.from_numpy(C).cuda()
    S1 = H.sigma(Ct).cpu().numpy()
    S2 = H.sigma(Ct).cpu().numpy()
    rows = sample_rows(w, 1500)
    ref = o.sigma_rows(rows, C)
    assert rel_err(S1[rows], ref) < TOL and rel_err(S2, S1) < 1e-14


@pytest.mark.parametrize("name,nvec", [("sel_30o_60k", 11), ("sel_30o_60k", 16), ("sel_64s_120k", 5)])
def test_sigma_wide_blocks_all_precisions(gpu, name, nvec):
    """Blocks wider than one vector group (8 real / 4 complex vectors per kernel pass),
    with a ragged last group: FP64 and paired FP32 against the oracle on sampled rows,
    FP32 storage against the oracle run on the FP32-rounded vectors."""
    torch = gpu
    w, o = case(name)
    H = gpu_ham(w, torch)
    rng = np.random.default_rng(400 + nvec)
    C = rng.normal(size=(w.M, nvec)) + (1j * rng.normal(size=(w.M, nvec)) if w.mode == "spinors" else 0)
    Ct = torch.from_numpy(C).cuda()
    rows = sample_rows(w, 400)
    ref = o.sigma_rows(rows, C)
    assert rel_err(H.sigma(Ct).cpu().numpy()[rows], ref) < TOL
    assert rel_err(H.sigma(Ct, prec=sci.SCI_PREC_F64_DS).cpu().numpy()[rows], ref) < TOL
    if w.mode != "spinors":
        C32 = np.ascontiguousarray(C, dtype=np.float32)
        S32 = H.sigma(torch.from_numpy(C32).cuda(), prec=sci.SCI_PREC_F32_STORE_F64_ACC).cpu().numpy()
        assert_fp32_rows(S32, C32, o, rows)


def test_keys_on_device_and_stream(gpu):
    torch = gpu
    w, o = case("so_sel_7o")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        H = sci.Hamiltonian()
        H.set_integrals(w.mode, w.ints.h, eri=w.ints.eri())
        H.set_determinants(torch.from_numpy(w.keys.view(np.int64)).cuda(), w.n_alpha, w.n_beta)
        C = torch.from_numpy(w.c).cuda()
        S = H.sigma(C)
    s.synchronize()
    assert rel_err(S.cpu().numpy(), o.sigma(w.c)) < TOL


# ------------------------------------------------------------------ edge cases
def test_empty_and_single_determinant(gpu):
    torch = gpu
    w = W.random_small(61, "spin_orbitals", 5, 2, 1)
    H = sci.Hamiltonian()
    H.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    H.set_determinants(np.zeros(0, dtype=np.uint64), 2, 1)
    assert H.count_pairs() == 0
    H.sigma(torch.zeros((0, 1), dtype=torch.float64, device="cuda"))
    H.set_determinants(w.keys[3:4], 2, 1)
    c = torch.tensor([[0.7]], dtype=torch.float64, device="cuda")
    o = Oracle(w.mode, w.n, w.ints.h, w.ints.eri(), w.keys[3:4])
    assert abs(H.sigma(c).item() - o.diagonal()[0] * 0.7) < 1e-13


@pytest.mark.parametrize("mode,n,na,nb", [("spinors", 6, 1, 0), ("spinors", 5, 0, 0),
                                          ("spin_orbitals", 6, 0, 2), ("spin_orbitals", 6, 3, 0)])
def test_degenerate_electron_counts(gpu, mode, n, na, nb):
    torch = gpu
    w = W.random_small(67, mode, n, na, nb, naux=3)
    o = Oracle.from_workload(w)
    H = gpu_ham(w, torch)
    S = H.sigma(torch.from_numpy(w.c).cuda()).cpu().numpy()
    assert rel_err(S, o.sigma(w.c)) < TOL
    assert H.count_pairs() == o.count_pairs()


def test_invalid_inputs_return_codes(gpu):
    torch = gpu
    w = W.random_small(71, "spin_orbitals", 5, 2, 2)
    H = sci.Hamiltonian()
    with pytest.raises(sci.SciError) as e:
        H.sigma(torch.zeros((4, 1), dtype=torch.float64, device="cuda"))
    assert e.value.code == sci.SCI_ERR_STATE
    with pytest.raises(sci.SciError) as e:
        H.set_determinants(w.keys, 2, 2)
    assert e.value.code == sci.SCI_ERR_STATE
    bad_h = w.ints.h.copy()
    bad_h[0, 1] += 1.0
    with pytest.raises(sci.SciError) as e:
        H.set_integrals(w.mode, bad_h, chol=w.ints.chol)
    assert e.value.code == sci.SCI_ERR_ARG
    H.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
    k = w.keys.copy()
    for keys, code in [(k[::-1].copy(), sci.SCI_ERR_UNSORTED),
                       (np.concatenate([k[:3], k[2:]]), sci.SCI_ERR_DUPLICATE),
                       (np.concatenate([k[:-1], [k[-1] | np.uint64(1 << 40)]]), sci.SCI_ERR_POPCOUNT),
                       (np.concatenate([[np.uint64(0b111)], k[1:]]), sci.SCI_ERR_POPCOUNT)]:
        with pytest.raises(sci.SciError) as e:
            H.set_determinants(keys, 2, 2)
        assert e.value.code == code, (code, e.value)
    # the context stays usable
    H.set_determinants(w.keys, 2, 2)
    o = Oracle.from_workload(w)
    S = H.sigma(torch.from_numpy(w.c).cuda()).cpu().numpy()
    assert rel_err(S, o.sigma(w.c)) < TOL
    with pytest.raises(sci.SciError) as e:
        sci.sci_sigma(H.ctx, torch.from_numpy(w.c).cuda(), torch.empty_like(torch.from_numpy(w.c)).cuda(), 0, 1)
    assert e.value.code == sci.SCI_ERR_ARG


# ------------------------------------------------------------------ Davidson
def test_davidson_mixed_matches_fp64_selected_space(gpu):
    """Block Davidson (4 roots) on the 60,000-determinant space: the FP32-storage solver
    with FP64 refinement reaches the plain FP64 solver's energies (residual 1e-8) to
    1e-9 Eh, and its returned vectors have exact FP64 residuals below the tolerance."""
    torch = gpu
    from paper_2501_18185_gb300.davidson import davidson, davidson_mixed

    w, o = case("sel_30o_60k")
    H = gpu_ham(w, torch)
    diag = H.diagonal()
    hi = lambda X: H.sigma(X.contiguous())  # noqa: E731
    lo = lambda X: H.sigma(X.to(torch.float32).contiguous(), prec=sci.SCI_PREC_F32_STORE_F64_ACC)  # noqa: E731
    ref = davidson(hi, diag, nroots=4, tol=1e-8, max_iter=600)
    mix = davidson_mixed(lo, hi, diag, nroots=4, tol=1e-7)
    assert ref.converged and mix.converged
    assert np.abs(mix.energies.cpu().numpy() - ref.energies.cpu().numpy()).max() < 1e-9
    X = mix.vectors
    R = hi(X) - X * mix.energies
    assert float(torch.linalg.vector_norm(R, dim=0).max()) <= 1e-7
    # the Rayleigh quotient of the first vector against the oracle's sigma on sampled rows
    rows = sample_rows(w, 500)
    x0 = X[:, 0].cpu().numpy()
    s = o.sigma_rows(rows, x0[:, None])[:, 0]
    assert np.allclose(s, hi(X[:, :1]).cpu().numpy()[rows, 0], rtol=0, atol=1e-11)


def test_davidson_fci_8o_matches_dense_eigh(gpu):
    torch = gpu
    from paper_2501_18185_gb300.davidson import davidson

    w, o = case("fci_8o_4a4b")
    Hd = o.dense()
    e_ref = np.linalg.eigvalsh(Hd)[:2]
    H = gpu_ham(w, torch)
    res = davidson(lambda X: H.sigma(X), H.diagonal(), nroots=2, tol=1e-8)
    assert res.converged
    assert np.abs(res.energies.cpu().numpy() - e_ref).max() < 1e-10


# ------------------------------------------------------------------ full-size workloads
FULL = {"sel_30o_full": lambda: W.selected_30o(), "sel_64s_full": lambda: W.selected_spinor_64()}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_sampled(gpu, name):
    """The bench workloads at full size, in the launch configuration bench.py times:
    sigma on 2,000 sampled rows (plus the first, last and reference rows) against the
    oracle, connection lists of row blocks bit-exact, and the pair count against the
    oracle's count when it is stored."""
    torch = gpu
    w = FULL[name]()
    o = Oracle.from_workload(w)
    H = gpu_ham(w, torch)
    S = H.sigma(torch.from_numpy(w.c).cuda()).cpu().numpy().reshape(w.M, -1)
    H.sync_status()
    rows = sample_rows(w, 2000, seed=7)
    assert rel_err(S[rows], o.sigma_rows(rows, w.c)) < TOL
    hf = int(np.searchsorted(w.keys, w.hf_key()))
    for a, b in ((0, 200), (hf, hf + 1), (w.M // 2, w.M // 2 + 200), (w.M - 200, w.M)):
        rr, J, deg, ph = H.connections(a, b)
        ref = [o.connections(r) for r in range(a, b)]
        assert np.array_equal(J, np.concatenate([x[0] for x in ref]))
        assert np.array_equal(deg, np.concatenate([x[1] for x in ref]))
        assert np.array_equal(ph, np.concatenate([x[2] for x in ref]))
    golden = json.load(open(GOLDEN)) if os.path.exists(GOLDEN) else {}
    if w.name in golden:
        assert H.count_pairs() == golden[w.name]["pairs"]
