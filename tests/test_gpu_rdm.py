"""GPU density matrices (sci_rdm12) and the autograd energy, against the oracle.

- g1 and g2 element by element against the oracle's operator-application RDMs (real and
  complex, FCI and selected spaces, up to the 60-spin-orbital 60k space);
- linearity in the weights, and rdm2 = NULL;
- on the full 2M-determinant space with 4 roots: the energy identity
  sum h gamma + 1/2 sum (pq|rs) Gamma = sum_k w_k c_k^T H c_k;
- autograd of E = c^T H c / c^T c against central finite differences (step 1e-5) on 50
  integral entries (h, dense (pq|rs) symmetry orbits, Cholesky factors) and along a
  random direction in c.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2501_18185_gb300 import sci
from paper_2501_18185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = {
    "fci_8o_4a4b": lambda: W.fci_small_8o(),
    "so_sel_7o": lambda: W.random_small(41, "spin_orbitals", 7, 3, 2, frac=0.5),
    "so_fci_10o_4a3b": lambda: W.random_small(43, "spin_orbitals", 10, 4, 3),
    "so_fci_6o_3a0b": lambda: W.random_small(45, "spin_orbitals", 6, 3, 0),
    "spinor_fci_12_4": lambda: W.random_small(47, "spinors", 12, 4, 0),
    "spinor_sel_16_5": lambda: W.random_small(53, "spinors", 16, 5, 0, frac=0.3),
    "spinor_64_2": lambda: W.random_small(59, "spinors", 64, 2, 0, naux=3),
}


def _rdm_gpu(torch, w, C, weights=None, rdm2=True):
    H = sci.Hamiltonian.from_workload(w)
    g1, g2 = H.rdm12(torch.from_numpy(np.ascontiguousarray(C)).cuda(), weights=weights, rdm2=rdm2)
    return g1.cpu().numpy(), (g2.cpu().numpy() if g2 is not None else None)


@pytest.mark.parametrize("name", list(SMALL))
def test_rdm_matches_oracle_small(gpu, name):
    w = SMALL[name]()
    o = Oracle.from_workload(w)
    c = w.c[:, 0]
    r1, r2 = o.rdm12(c)
    g1, g2 = _rdm_gpu(gpu, w, c)
    assert np.abs(g1 - r1).max() < 1e-12
    assert np.abs(g2 - r2).max() < 1e-12


def test_rdm_matches_oracle_selected_60k(gpu):
    """The 60-spin-orbital selected space: every one of the 60^4 elements of g2.  The
    largest elements (occupations ~0.9) are sums of up to M = 6e4 products taken in a
    different order on each side: the FP64 bound M u sum|terms| is ~7e-12, so 1e-11."""
    w = W.selected_30o(M=60000)
    o = Oracle.from_workload(w)
    c = w.c[:, 0]
    r1, r2 = o.rdm12(c)
    g1, g2 = _rdm_gpu(gpu, w, c)
    assert np.abs(g1 - r1).max() < 1e-11
    assert np.abs(g2 - r2).max() < 1e-11


def test_rdm_weights_linear_and_rdm1_only(gpu):
    torch = gpu
    w = W.random_small(71, "spinors", 10, 4, 0, frac=0.7)
    rng = np.random.default_rng(3)
    C = rng.normal(size=(w.M, 11)) + 1j * rng.normal(size=(w.M, 11))   # two walks of <= 8 vectors
    wt = rng.uniform(-1, 2, 11)
    g1, g2 = _rdm_gpu(torch, w, C, weights=wt)
    o = Oracle.from_workload(w)
    r1, r2 = 0, 0
    for k in range(11):
        a, b = o.rdm12(C[:, k])
        r1, r2 = r1 + wt[k] * a, r2 + wt[k] * b
    scale = max(1.0, np.abs(r2).max())
    assert np.abs(g1 - r1).max() < 1e-12 * scale and np.abs(g2 - r2).max() < 1e-12 * scale
    h1, none = _rdm_gpu(torch, w, C, weights=wt, rdm2=False)
    assert none is None and np.abs(h1 - g1).max() < 1e-12 * scale


def spin_sum_rdm(g1, g2, n: int):
    """Spin-orbital (2n) -> spatial (n) density matrices by indexing, as a reference:
    gamma[p,q] = sum_s g1[ps, qs], Gamma[p,q,r,s] = sum_{s,t} g2[ps, qs, rt, st]
    (bit p < n is alpha p, bit n+p beta p)."""
    g = g1.reshape(2, n, 2, n)
    gamma = g[0, :, 0, :] + g[1, :, 1, :]
    if g2 is None:
        return gamma, None
    G = g2.reshape(2, n, 2, n, 2, n, 2, n)
    Gamma = sum(G[s, :, s, :, t, :, t, :] for s in range(2) for t in range(2))
    return gamma, Gamma


@pytest.mark.parametrize("name", ["fci_8o", "sel_30o_60k"])
def test_rdm_grads_spin_sums_and_cholesky_contraction(gpu, name):
    """sci_rdm_grads against the spin sums of sci_rdm12's matrices (indexing, above) and
    the contraction gchol[P] = sum_rs Gamma[:, :, r, s] L[P, r, s] done in numpy."""
    torch = gpu
    w = W.fci_small_8o() if name == "fci_8o" else W.selected_30o(M=60000, nvec=3)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(np.ascontiguousarray(w.c)).cuda()
    wt = np.array([1.0, -0.5, 2.0])[: C.shape[1]]
    g1, g2 = H.rdm12(C, weights=wt)
    gamma_r, Gamma_r = spin_sum_rdm(g1.cpu().numpy(), g2.cpu().numpy(), w.n)
    L = torch.from_numpy(w.ints.chol.copy()).cuda()
    gamma, Gamma, gL = H.rdm_grads(C, weights=wt, chol=L, Gamma=True)
    scale = np.abs(Gamma_r).max()
    assert np.abs(gamma.cpu().numpy() - gamma_r).max() < 1e-12 * np.abs(gamma_r).max()
    assert np.abs(Gamma.cpu().numpy() - Gamma_r).max() < 1e-12 * scale
    n, naux = w.n, w.ints.chol.shape[0]
    ref = (Gamma_r.reshape(n * n, n * n) @ w.ints.chol.reshape(naux, n * n).T).T.reshape(naux, n, n)
    assert np.abs(gL.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    # 1-RDM only: no 2-RDM walk, the same gamma
    g_only, none1, none2 = H.rdm_grads(C, weights=wt)
    assert none1 is None and none2 is None and torch.allclose(g_only, gamma, rtol=0, atol=1e-13 * float(gamma.abs().max()))


def test_rdm_energy_identity_full_space_4_roots(gpu):
    """2M-determinant space, 4 vectors: sum h gamma + 1/2 sum (pq|rs) Gamma equals
    sum_k w_k c_k^T sigma_k (spin-summed spatial density matrices)."""
    torch = gpu

    w = W.selected_30o(nvec=4)
    H = sci.Hamiltonian.from_workload(w)
    C = torch.from_numpy(w.c).cuda()
    wt = np.array([1.0, 0.5, -0.25, 2.0])
    g1, g2 = H.rdm12(C, weights=wt)
    gamma, Gamma = spin_sum_rdm(g1, g2, w.n)
    h = torch.from_numpy(w.ints.h).cuda()
    eri = torch.from_numpy(w.ints.eri()).cuda()
    E_rdm = float((h * gamma).sum() + 0.5 * (eri * Gamma).sum())
    S = H.sigma(C)
    E_sig = float(((C * S).sum(0) * torch.from_numpy(wt).cuda()).sum())
    assert abs(E_rdm - E_sig) < 1e-11 * abs(E_sig)
    # traces: sum_p gamma_pp = N sum w |c|^2, Gamma_pprr = N(N-1) sum w |c|^2
    norms = float(((C * C).sum(0) * torch.from_numpy(wt).cuda()).sum())
    assert abs(float(torch.trace(gamma)) - 20 * norms) < 1e-10
    assert abs(float(torch.einsum("pprr->", Gamma)) - 20 * 19 * norms) < 1e-8


def test_autograd_matches_finite_differences(gpu):
    """E = sum_k g_k c_k^T H c_k / c_k^T c_k on the 2M space with 4 Davidson roots:
    analytic gradients against central differences (step 1e-5) on 50 integral entries:
    16 of h (h_pq and h_qp moved together), 18 symmetry orbits of the dense (pq|rs),
    16 Cholesky entries (L^P_pq and L^P_qp together), and along a random direction in c."""
    torch = gpu
    from paper_2501_18185_gb300.autograd import orbit_mask, rayleigh_energy
    from paper_2501_18185_gb300.davidson import davidson

    w = W.selected_30o()
    n = w.n
    H = sci.Hamiltonian.from_workload(w)
    roots = davidson(lambda X: H.sigma(X.contiguous()), H.diagonal(), nroots=4, tol=1e-4)
    C = roots.vectors.detach().clone()
    gw = torch.tensor([1.0, -0.5, 0.25, 0.75], dtype=torch.float64, device="cuda")
    h0 = torch.from_numpy(w.ints.h.copy()).cuda()
    L0 = torch.from_numpy(w.ints.chol.copy()).cuda()
    eri0 = torch.from_numpy(w.ints.eri()).cuda()
    rng = np.random.default_rng(2025)
    step = 1e-5

    def loss(h, L, c, kind):
        return (rayleigh_energy(h, L, c, H, kind) * gw).sum()

    # analytic
    h = h0.clone().requires_grad_(True)
    L = L0.clone().requires_grad_(True)
    loss(h, L, C, "chol").backward()
    e = eri0.clone().requires_grad_(True)
    h2 = h0.clone().requires_grad_(True)
    loss(h2, e, C, "eri").backward()
    assert torch.allclose(h.grad, h2.grad, rtol=0, atol=1e-12)

    def fd(fn):
        return (fn(step) - fn(-step)) / (2 * step)

    checked = 0
    for _ in range(16):
        p, q = rng.integers(0, n, 2)
        d = torch.zeros_like(h0)
        d[p, q] += 1.0
        if p != q:
            d[q, p] += 1.0
        num = fd(lambda s: float(loss(h0 + s * d, L0, C, "chol")))
        ana = float((h.grad * d).sum())
        assert abs(num - ana) < 1e-6 * max(1.0, abs(ana)), (p, q, num, ana)
        checked += 1
    for _ in range(18):
        idx = tuple(int(v) for v in rng.integers(0, n, 4))
        d = torch.from_numpy(orbit_mask(n, idx)).cuda()
        num = fd(lambda s: float(loss(h0, eri0 + s * d, C, "eri")))
        ana = float((e.grad * d).sum())
        assert abs(num - ana) < 1e-6 * max(1.0, abs(ana)), (idx, num, ana)
        checked += 1
    for _ in range(16):
        P = int(rng.integers(0, L0.shape[0]))
        p, q = rng.integers(0, n, 2)
        d = torch.zeros_like(L0)
        d[P, p, q] += 1.0
        if p != q:
            d[P, q, p] += 1.0
        num = fd(lambda s: float(loss(h0, L0 + s * d, C, "chol")))
        ana = float((L.grad * d).sum())
        assert abs(num - ana) < 1e-6 * max(1.0, abs(ana)), (P, p, q, num, ana)
        checked += 1
    assert checked == 50
    # coefficient gradient, at a point away from the eigenvectors (where it is not just the
    # residual), along a random unit direction per column
    noise = torch.from_numpy(rng.normal(size=C.shape)).cuda()
    Cp = C + 0.05 * noise / torch.linalg.vector_norm(noise, dim=0)
    cp = Cp.clone().requires_grad_(True)
    loss(h0, L0, cp, "chol").backward()
    dC = torch.from_numpy(rng.normal(size=C.shape)).cuda()
    dC = dC / torch.linalg.vector_norm(dC, dim=0)
    num = fd(lambda s: float(loss(h0, L0, Cp + s * dC, "chol")))
    ana = float((cp.grad * dC).sum())
    assert abs(ana) > 1e-3 and abs(num - ana) < 1e-6 * max(1.0, abs(ana)), (num, ana)
