"""Host-side logic of the Davidson drivers, on the CPU with dense stand-ins for sigma.

The FP64 sigma is a dense symmetric matrix; the low-precision sigma applies the matrix
rounded to FP32 to the vectors rounded to FP32 (what the FP32-storage kernel does), with
the products summed in FP64.  Both drivers must reach numpy's eigenvalues; the mixed one
must do so with only a few FP64 products.
"""
import numpy as np
import pytest
import torch

from paper_2501_18185_gb300.davidson import davidson, davidson_mixed


def _ci_like(n, seed):
    """Diagonally dominant symmetric matrix with a CI-like spectrum."""
    rng = np.random.default_rng(seed)
    A = rng.normal(scale=0.05, size=(n, n))
    A = 0.5 * (A + A.T)
    A[np.diag_indices(n)] = np.sort(rng.uniform(-5.0, 5.0, n)) + np.linspace(0, 1, n)
    return A


@pytest.mark.parametrize("nroots", [1, 4])
def test_davidson_fp64_matches_eigh(nroots):
    A = _ci_like(600, 1)
    ref = np.linalg.eigvalsh(A)[:nroots]
    At = torch.from_numpy(A)
    res = davidson(lambda X: At @ X, torch.from_numpy(np.diag(A).copy()), nroots=nroots, tol=1e-9)
    assert res.converged
    assert np.abs(res.energies.numpy() - ref).max() < 1e-10


@pytest.mark.parametrize("nroots", [1, 4])
def test_davidson_mixed_reaches_fp64_energies(nroots):
    A = _ci_like(600, 2)
    ref = np.linalg.eigvalsh(A)[:nroots]
    At = torch.from_numpy(A)
    A32 = torch.from_numpy(A.astype(np.float32).astype(np.float64))
    calls = {"lo": 0, "hi": 0}

    def lo(X):
        calls["lo"] += 1
        return A32 @ X.to(torch.float32).to(torch.float64)

    def hi(X):
        calls["hi"] += 1
        return At @ X

    res = davidson_mixed(lo, hi, torch.from_numpy(np.diag(A).copy()), nroots=nroots, tol=1e-8)
    assert res.converged
    # the low-precision products alone would stall near 1e-7 relative; FP64 refinement
    # carries the energies to the FP64 eigenvalues
    assert np.abs(res.energies.numpy() - ref).max() < 1e-10
    assert 1 <= calls["hi"] <= 12 and calls["lo"] > calls["hi"]
    # exact residual of the returned vectors
    X = res.vectors
    R = At @ X - X * res.energies
    assert float(torch.linalg.vector_norm(R, dim=0).max()) <= 1e-8


def test_kato_temple_bound_holds_and_sets_the_tolerance():
    """The bench's claim "residual sqrt(1e-8 * min gap) puts every energy within 1e-8 of
    the exact one" rests on |E_k - lambda_k| <= r_k^2 / gap_k (Kato-Temple).  Check the
    bound on loose Davidson runs against dense eigenvalues, and that running to the
    tolerance it derives (from a tight run with one extra root) meets the target."""
    import bench

    A = _ci_like(800, 5)
    lam = np.linalg.eigvalsh(A)
    At = torch.from_numpy(A)
    diag = torch.from_numpy(np.diag(A).copy())
    nroots = 4
    for tol in (1e-2, 1e-3, 1e-4):
        r = davidson(lambda X: At @ X, diag, nroots=nroots + 1, tol=tol)
        gaps, bounds, _ = bench.kato_temple(r.energies.numpy(), r.residual_norms.numpy(), nroots)
        err = np.abs(r.energies.numpy()[:nroots] - lam[:nroots])
        assert np.all(err <= bounds * (1 + 1e-6) + 1e-14), (tol, err, bounds)
    ref = davidson(lambda X: At @ X, diag, nroots=nroots + 1, tol=1e-10)
    _, _, tol_t = bench.kato_temple(ref.energies.numpy(), ref.residual_norms.numpy(), nroots, target=1e-8)
    run = davidson(lambda X: At @ X, diag, nroots=nroots, tol=tol_t)
    assert np.abs(run.energies.numpy() - lam[:nroots]).max() <= 1e-8


def test_kato_temple_gaps():
    import bench

    # delta_k = min_j (|e_k - e_j| - r_j): the other Ritz values' residuals shrink the gap
    gaps, bounds, t = bench.kato_temple([-3.0, -2.9, -1.0, 0.5], [1e-3, 2e-3, 1e-4, 5e-4], 3, target=1e-8)
    assert np.allclose(gaps, [0.1 - 2e-3, 0.1 - 1e-3, 1.5 - 5e-4])
    assert np.allclose(bounds, [1e-6 / 0.098, 4e-6 / 0.099, 1e-8 / 1.4995])
    assert abs(t - np.sqrt(1e-8 * 0.098)) < 1e-15
    # a gap eaten by a residual is clamped, not negative
    gaps, _, _ = bench.kato_temple([-1.0, -0.99], [1e-3, 0.5], 1)
    assert gaps[0] == 1e-12
