"""Block Davidson eigensolvers over sigma = H X (torch, FP64 host-side loop).

The paper diagonalises the variational space through matrix-vector products
sigma_i = H X_i whose elements are recomputed, never stored (Sec. 2.4, the
diagonalisation paragraph; MetaWave uses the iVI solver there).  These drivers use the
Davidson method with the diagonal preconditioner (E - H_II)^-1: every product with H
goes through libsci's sigma kernels; Gram-Schmidt, the subspace matrix, the small
Hermitian eigenproblem and the residual are FP64 torch operations on the GPU.

The projected matrix G = V^+ H V is kept and extended by its new rows and columns only
(two thin products per iteration); a full V^+ W every iteration would dominate the
iteration time on GB300, whose FP64 rate is 1.2 TFLOP/s.  Restarts are thick: the
subspace collapses to the lowest `keep` Ritz vectors (2 x nroots by default).
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
    sigma_calls_lo: int = 0
    sigma_calls_hi: int = 0


def _orthonormalize(V: torch.Tensor | None, T: torch.Tensor, drop: float = 1e-10) -> torch.Tensor:
    """Orthonormalise the columns of T against V and among themselves: two passes of
    block classical Gram-Schmidt against V, then Cholesky QR of the block (twice),
    dropping directions that are numerically in span(V)."""
    for _ in range(2):
        if V is not None and V.shape[1] > 0:
            T = T - V @ (V.conj().T @ T)
    nrm = torch.linalg.vector_norm(T, dim=0)
    T = T[:, nrm > drop]
    if T.shape[1] == 0:
        return T
    T = T / torch.linalg.vector_norm(T, dim=0)
    for _ in range(2):
        G = T.conj().T @ T
        evals, evecs = torch.linalg.eigh(G)
        good = evals > 1e-12
        if not bool(good.all()):
            T = T @ evecs[:, good]
            G = T.conj().T @ T
        L = torch.linalg.cholesky(G)
        T = torch.linalg.solve_triangular(L.conj().T, T, upper=True, left=False)
        if V is not None and V.shape[1] > 0:
            T = T - V @ (V.conj().T @ T)
    return T


def _guess(diag, nvec, dtype, seed: int = 20250130, noise: float = 1e-3):
    """Unit vectors on the lowest diagonal entries plus a small seeded random part.
    Without the random part the start block can lie entirely in one symmetry sector of
    H (e.g. have exactly zero overlap with the ground state), which a symmetry-blind
    solver would then never leave."""
    M = diag.shape[0]
    k = min(M, nvec)
    idx = torch.argsort(diag)[:k]
    g = torch.Generator(device="cpu").manual_seed(seed)
    V = noise * torch.randn((M, k), generator=g, dtype=torch.float64).to(diag.device).to(dtype) / (M ** 0.5)
    V[idx, torch.arange(k, device=diag.device)] += 1.0
    return _orthonormalize(None, V)


def _corrections(R, theta, diag, active, dtype):
    T = []
    for j in active:
        den = theta[j] - diag
        den = torch.where(den.abs() < 1e-8, torch.full_like(den, 1e-8), den)
        T.append(R[:, j] / den.to(dtype))
    return torch.stack(T, dim=1)


def _herm(G):
    return 0.5 * (G + G.conj().T)


def davidson(sigma, diag: torch.Tensor, nroots: int = 1, tol: float = 1e-9, max_iter: int = 300,
             max_space: int | None = None, keep: int | None = None, guess: torch.Tensor | None = None,
             dtype=torch.float64) -> DavidsonResult:
    """Lowest `nroots` eigenpairs of H.

    sigma(X [M,k]) -> H X (same dtype); diag: H_II (float64, [M]).  Converged when every
    root's residual 2-norm ||H x - E x|| <= tol.
    """
    M = diag.shape[0]
    keep = min(M, keep or 2 * nroots)
    max_space = min(M, max_space or max(12 * nroots, keep + 2 * nroots, 24))
    # at least 8 start vectors
    V = _guess(diag, max(keep, 8), dtype) if guess is None else _orthonormalize(None, guess.to(dtype))
    W = sigma(V)
    G = _herm(V.conj().T @ W)
    calls = 1
    hist = []
    theta = X = rn = None
    for it in range(1, max_iter + 1):
        evals, evecs = torch.linalg.eigh(G)
        theta = evals[:nroots].real.to(torch.float64)
        Y = evecs[:, :nroots]
        X = V @ Y
        R = W @ Y - X * theta.to(dtype)
        rn = torch.linalg.vector_norm(R, dim=0).real
        hist.append((it, theta.clone().cpu(), rn.clone().cpu()))
        if bool((rn <= tol).all()):
            return DavidsonResult(theta, X, rn, it, calls, True, hist, 0, calls)
        active = [j for j in range(nroots) if rn[j] > tol]
        T = _corrections(R, theta, diag, active, dtype)
        if V.shape[1] + T.shape[1] > max_space:
            Yk = evecs[:, :min(keep, V.shape[1])]
            V, W = V @ Yk, W @ Yk
            G = torch.diag(evals[:Yk.shape[1]]).to(dtype)
        T = _orthonormalize(V, T)
        if T.shape[1] == 0:
            break
        WT = sigma(T)
        calls += 1
        B = V.conj().T @ WT                       # old x new block
        C = _herm(T.conj().T @ WT)                # new x new block
        G = torch.cat([torch.cat([G, B], dim=1), torch.cat([B.conj().T, C], dim=1)], dim=0)
        V = torch.cat([V, T], dim=1)
        W = torch.cat([W, WT], dim=1)
    return DavidsonResult(theta, X, rn, max_iter, calls, False, hist, 0, calls)


def davidson_mixed(sigma_lo, sigma_hi, diag: torch.Tensor, nroots: int = 1, tol: float = 1e-6,
                   max_iter: int = 400, max_space: int | None = None, keep: int | None = None,
                   guess: torch.Tensor | None = None, dtype=torch.float64) -> DavidsonResult:
    """Davidson with low-precision products for the correction vectors and FP64 refinement.

    sigma_lo(X) -> H X from the FP32-storage sigma (C rounded to FP32, exact products,
    FP64 accumulation); sigma_hi(X) -> H X in FP64.  Correction vectors take their
    products from sigma_lo.  When the estimated residuals claim convergence, stall, or
    the space is full, the subspace is refined: it collapses to the lowest `keep` Ritz
    vectors and their products are recomputed with sigma_hi, which makes the Rayleigh
    quotients and residuals of the Ritz vectors exact in FP64.  Convergence is declared
    only on those exact residuals (every root's ||H x - E x|| <= tol).

    In the subspace matrix an entry that couples a column with an exact product takes the
    exact side (v_i^+ (H v_j) or (H v_i)^+ v_j), so the FP32 error stays in the block of
    low-precision columns, whose coefficients in the Ritz vectors are of the size of the
    residual.  FP64 is kept for the Gram-Schmidt, the subspace matrix, the Rayleigh
    quotient and the final energies.
    """
    M = diag.shape[0]
    dev = diag.device
    keep = min(M, keep or 2 * nroots)
    max_space = min(M, max_space or max(12 * nroots, keep + 2 * nroots, 24))
    V = _guess(diag, max(keep, 8), dtype) if guess is None else _orthonormalize(None, guess.to(dtype))
    W = sigma_lo(V)
    G = _herm(0.5 * (V.conj().T @ W + W.conj().T @ V))
    ex = torch.zeros(V.shape[1], dtype=torch.bool, device=dev)   # columns of W from sigma_hi
    calls_lo, calls_hi = 1, 0
    best_est, stall = None, 0
    hist = []
    theta = X = rn = None

    def refine(Vn):
        nonlocal calls_hi
        Wn = sigma_hi(Vn)
        calls_hi += 1
        return Vn, Wn, _herm(Vn.conj().T @ Wn), torch.ones(Vn.shape[1], dtype=torch.bool, device=dev)

    for it in range(1, max_iter + 1):
        evals, evecs = torch.linalg.eigh(G)
        theta = evals[:nroots].real.to(torch.float64)
        Y = evecs[:, :nroots]
        X = V @ Y
        R = W @ Y - X * theta.to(dtype)
        rn = torch.linalg.vector_norm(R, dim=0).real
        rmax = float(rn.max())
        exact = bool(ex.all())
        hist.append((it, theta.clone().cpu(), rn.clone().cpu(), exact))
        if exact and rmax <= tol:
            return DavidsonResult(theta, X, rn, it, calls_lo + calls_hi, True, hist, calls_lo, calls_hi)
        if exact:
            best_est, stall = rmax, 0
        else:
            if best_est is None or rmax < 0.9 * best_est:
                best_est, stall = rmax, 0
            else:
                stall += 1
            if rmax <= tol or stall >= 6:
                V, W, G, ex = refine(V @ evecs[:, :min(keep, V.shape[1])])
                best_est, stall = None, 0
                continue
        active = [j for j in range(nroots) if rn[j] > tol]
        T = _corrections(R, theta, diag, active, dtype)
        if V.shape[1] + T.shape[1] > max_space:
            # a full space collapses with FP64 products: rotating the stored W would mix
            # the FP32 error into the exact block of the kept Ritz vectors
            V, W, G, ex = refine(V @ evecs[:, :min(keep, V.shape[1])])
            best_est, stall = None, 0
            continue
        T = _orthonormalize(V, T)
        if T.shape[1] == 0:
            V, W, G, ex = refine(V @ evecs[:, :min(keep, V.shape[1])])
            continue
        WT = sigma_lo(T)
        calls_lo += 1
        # old x new block: exact side when the old column's product is exact
        B1 = V.conj().T @ WT                      # v_i^+ (H_lo t_j)
        B2 = W.conj().T @ T                       # (H v_i)^+ t_j
        B = torch.where(ex[:, None], B2, 0.5 * (B1 + B2))
        C = _herm(0.5 * (T.conj().T @ WT + WT.conj().T @ T))
        G = torch.cat([torch.cat([G, B], dim=1), torch.cat([B.conj().T, C], dim=1)], dim=0)
        V = torch.cat([V, T], dim=1)
        W = torch.cat([W, WT], dim=1)
        ex = torch.cat([ex, torch.zeros(T.shape[1], dtype=torch.bool, device=dev)])
    return DavidsonResult(theta, X, rn, max_iter, calls_lo + calls_hi, False, hist, calls_lo, calls_hi)
