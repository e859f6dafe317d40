"""Differentiable Rayleigh quotients E_k = c_k^T H c_k / c_k^T c_k through libsci.

H is the Hamiltonian of Eq. Hamiltonian (Sec. 2.1) on the determinant list held by a
`sci.Hamiltonian`, built from h and either the dense (pq|rs) or Cholesky factors L^P with
(pq|rs) = sum_P L^P_pq L^P_rs (real spin-orbital mode).  Forward: one sigma = H C.
Backward, hand-written (the connections are recomputed by libsci's density-matrix walk,
never stored; the spin sums and the contraction with L run in libsci too, sci_rdm_grads),
with G_k = grad_output_k / (c_k^T c_k) and the spin-summed density matrices gamma (n x n)
and Gamma (n^4) of the weighted ensemble sum_k G_k |c_k><c_k|:
    dL/dh_pq        = gamma_pq                     (gamma_pq = sum_s g1[p s, q s])
    dL/d(pq|rs)     = 1/2 Gamma_pqrs               (Gamma_pqrs = sum_st g2[p s, q s, r t, s t])
    dL/dL^P_pq      = sum_rs Gamma_pqrs L^P_rs
    dL/dc_k         = 2 G_k (sigma_k - E_k c_k)
The factor 1/2 on (pq|rs) is that of Eq. Hamiltonian: E = sum h g1 + 1/2 sum (pq|rs) g2.
h, (pq|rs) and L^P are treated as free entries (no symmetrisation of the gradient); a
perturbation that keeps H Hermitian moves a whole symmetry orbit and picks up the sum of
the orbit's entries.
"""
from __future__ import annotations

import numpy as np
import torch


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, L, C, ham, kind):
        n = h.shape[0]
        # the integrals stay on the device: sci_set_integrals_ex reads them in place
        hd = h.detach().to(ham.device)
        Ld = L.detach().to(ham.device)
        if kind == "chol":
            ham.set_integrals("spin_orbitals", hd, chol=Ld)
        else:
            ham.set_integrals("spin_orbitals", hd, eri=Ld)
        Cd = C.detach().contiguous()
        S = ham.sigma(Cd)
        den = (Cd * Cd).sum(dim=0)
        E = (Cd * S).sum(dim=0) / den
        ctx.save_for_backward(L, Cd, S, E, den)
        ctx.ham, ctx.kind, ctx.n = ham, kind, n
        return E

    @staticmethod
    def backward(ctx, gE):
        L, C, S, E, den = ctx.saved_tensors
        ham, kind, n = ctx.ham, ctx.kind, ctx.n
        G = (gE / den).detach()
        need_h, need_L, need_C = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        gh = gL = gC = None
        if need_h or need_L:
            w = G.cpu().numpy()
            if need_L and kind == "chol":
                gamma, _, gL = ham.rdm_grads(C, weights=w, chol=L.detach().to(ham.device))
            else:
                gamma, Gamma, _ = ham.rdm_grads(C, weights=w, Gamma=need_L)
                if need_L:
                    gL = 0.5 * Gamma.to(L.device)
            if need_h:
                gh = gamma.to(L.device)
            if gL is not None:
                gL = gL.to(L.device)
        if need_C:
            gC = 2.0 * (S - C * E) * G
        return gh, gL, gC, None, None


def rayleigh_energy(h: torch.Tensor, L: torch.Tensor, C: torch.Tensor, ham, kind: str = "chol") -> torch.Tensor:
    """E_k = c_k^T H c_k / c_k^T c_k for the columns of C ([M, nroots], CUDA float64).

    h: [n, n]; L: Cholesky factors [naux, n, n] (kind "chol") or the dense (pq|rs) [n]^4
    (kind "eri").  `ham` is a sci.Hamiltonian holding the determinant list; its integrals
    are replaced by (h, L) on every forward.  Differentiable in h, L and C."""
    if kind not in ("chol", "eri"):
        raise ValueError("kind is 'chol' or 'eri'")
    if C.dim() == 1:
        C = C.reshape(-1, 1)
    return _Energy.apply(h, L, C, ham, kind)


def symmetry_orbit(p: int, q: int, r: int, s: int):
    """The entries (pq|rs) = (qp|rs) = (pq|sr) = (rs|pq) = ... of one real permutation
    orbit (8-fold), as a set of index tuples."""
    return {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
            (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}


def orbit_mask(n: int, idx) -> np.ndarray:
    m = np.zeros((n,) * 4)
    for t in symmetry_orbit(*idx):
        m[t] = 1.0
    return m
