"""Block Davidson eigensolver over sigma = H X (torch, FP64 host-side loop).

The paper diagonalises the variational space through matrix-vector products
sigma_i = H X_i whose elements are recomputed, never stored (Sec. 2.4, the
diagonalisation paragraph; MetaWave uses the iVI solver there).  This driver uses the
Davidson method with the diagonal preconditioner (E - H_II)^-1: every product with H
goes through libsci's sigma kernels; Gram-Schmidt, the subspace matrix, the small
Hermitian eigenproblem and the residual are FP64 torch operations on the GPU.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch


@dataclass
class DavidsonResult:
    energies: torch.Tensor          # [nroots] float64
    vectors: torch.Tensor           # [M, nroots]
    residual_norms: torch.Tensor    # [nroots]
    iterations: int
    sigma_calls: int
    converged: bool
    history: list = field(default_factory=list)


def _orthonormalize(V: torch.Tensor, T: torch.Tensor, drop: float = 1e-10) -> torch.Tensor:
    """Two passes of block classical Gram-Schmidt of T against V, then within T."""
    for _ in range(2):
        if V is not None and V.shape[1] > 0:
            T = T - V @ (V.conj().T @ T)
    cols = []
    for j in range(T.shape[1]):
        t = T[:, j]
        for _ in range(2):
            for c in cols:
                t = t - c * (c.conj() @ t)
            if V is not None and V.shape[1] > 0:
                t = t - V @ (V.conj().T @ t)
        nrm = torch.linalg.vector_norm(t)
        if nrm > drop:
            cols.append(t / nrm)
    if not cols:
        return T[:, :0]
    return torch.stack(cols, dim=1)


def davidson(sigma, diag: torch.Tensor, nroots: int = 1, tol: float = 1e-9, max_iter: int = 200,
             max_space: int | None = None, guess: torch.Tensor | None = None,
             dtype=torch.float64) -> DavidsonResult:
    """Lowest `nroots` eigenpairs of H.

    sigma(X [M,k]) -> H X (same dtype); diag: H_II (float64, [M]).  Convergence when every
    root's residual 2-norm ||H x - E x|| <= tol.
    """
    M = diag.shape[0]
    dev = diag.device
    k0 = min(M, max(nroots, 2 * nroots))
    max_space = max_space or min(M, max(8 * nroots, 24))
    if guess is None:
        idx = torch.argsort(diag)[:k0]
        V = torch.zeros((M, k0), dtype=dtype, device=dev)
        V[idx, torch.arange(k0, device=dev)] = 1.0
    else:
        V = _orthonormalize(None, guess.to(dtype))
    W = sigma(V)
    calls = 1
    hist = []
    theta = None
    X = None
    rn = None
    for it in range(1, max_iter + 1):
        G = V.conj().T @ W
        G = 0.5 * (G + G.conj().T)
        evals, evecs = torch.linalg.eigh(G)
        theta = evals[:nroots].real.to(torch.float64)
        Y = evecs[:, :nroots]
        X = V @ Y
        R = W @ Y - X * theta.to(dtype)
        rn = torch.linalg.vector_norm(R, dim=0).real
        hist.append((it, theta.clone().cpu(), rn.clone().cpu()))
        if bool((rn <= tol).all()):
            return DavidsonResult(theta, X, rn, it, calls, True, hist)
        active = [j for j in range(nroots) if rn[j] > tol]
        T = []
        for j in active:
            den = theta[j] - diag
            den = torch.where(den.abs() < 1e-8, torch.full_like(den, 1e-8), den)
            T.append(R[:, j] / den.to(dtype))
        T = torch.stack(T, dim=1)
        if V.shape[1] + T.shape[1] > max_space:
            # restart from the current Ritz vectors
            V = _orthonormalize(None, X)
            W = sigma(V)
            calls += 1
        T = _orthonormalize(V, T)
        if T.shape[1] == 0:
            break
        WT = sigma(T)
        calls += 1
        V = torch.cat([V, T], dim=1)
        W = torch.cat([W, WT], dim=1)
    return DavidsonResult(theta, X, rn, max_iter, calls, False, hist)
