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
