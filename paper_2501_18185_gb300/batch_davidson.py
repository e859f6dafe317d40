"""Ground states of many small Hamiltonians at once: a Davidson iteration for every
instance, with one batched sigma launch per iteration.

The instances are the sci.Hamiltonian contexts of a sci.Batch (heterogeneous sizes).
Every iteration applies H to the new search vector of every instance in one persistent
launch, replayed from a CUDA graph captured once over fixed vector buffers (the batched
sigma of config 3b).  The subspace algebra runs batched over instances: the search spaces
are padded to the largest instance, [B, M_max, k], and the projections, Rayleigh-Ritz
problems ([B, k, k] eigh), residuals and Gram-Schmidt are batched tensor operations in
FP64.  All instances grow their space together (one column per iteration); an instance
whose space is exhausted (M_i <= k), or that has converged, takes a null column whose
diagonal in G is set above its lowest Ritz values, so it is never chosen.  Restarts are
thick (the space collapses to the `keep` lowest Ritz vectors of each instance).

The method per instance is that of davidson.davidson with one root: diagonal
preconditioner (theta - H_II)^-1, convergence when ||H x - theta x|| <= tol.  The start
block is the same as there: unit vectors on the lowest diagonal entries plus a small
seeded random part, so that no instance starts inside one symmetry sector of its H.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import sci

_PAD = 1e30   # diagonal of the padding rows: their preconditioned residual is zero


@dataclass
class BatchDavidsonResult:
    energies: np.ndarray        # [B]
    residual_norms: np.ndarray  # [B]
    converged: np.ndarray       # [B] bool
    iterations: int
    sigma_launches: int
    vectors: torch.Tensor       # concatenated [sum M_i], instance i at batch.offsets[i]


class _Padded:
    """Index maps between the concatenated vector of the batch ([sum M_i], instance i at
    its offset) and the padded block [B, M_max]; the diagonal and the valid-row mask."""

    def __init__(self, batch):
        dev = batch.device
        hams = batch.hams
        self.B = len(hams)
        Ms = torch.tensor([H.M for H in hams], device=dev)
        self.Mmax = int(Ms.max())
        self.Mtot = batch.M
        off = torch.tensor(batch.offsets, device=dev)
        inst = torch.repeat_interleave(torch.arange(self.B, device=dev), Ms)
        self.flat = inst * self.Mmax + (torch.arange(self.Mtot, device=dev) - off[inst])
        hd = torch.cat([H.diagonal() for H in hams])
        diag = torch.full((self.B * self.Mmax,), _PAD, dtype=torch.float64, device=dev)
        diag[self.flat] = hd
        self.diag = diag.view(self.B, self.Mmax)
        valid = torch.zeros(self.B * self.Mmax, dtype=torch.float64, device=dev)
        valid[self.flat] = 1.0
        self.valid = valid.view(self.B, self.Mmax)
        # G entry of a null column: above the lowest Ritz values (bounded by the diagonal),
        # small enough to keep eigh's absolute error at the level of the spectrum
        self.penalty = 10.0 * float(hd.abs().max()) + 10.0
        self.dev = dev

    def to_concat(self, T):
        return T.reshape(-1)[self.flat]

    def from_concat(self, x):
        out = torch.zeros(self.B * self.Mmax, dtype=torch.float64, device=self.dev)
        out[self.flat] = x
        return out.view(self.B, self.Mmax)

    def start_block(self, nstart, seed=20250130, noise=1e-3):
        """[B, Mmax, nstart]: unit vectors on the nstart lowest diagonal entries of each
        instance plus seeded noise of norm ~noise (valid rows only)."""
        g = torch.Generator(device="cpu").manual_seed(seed)
        T = noise * torch.randn((self.B, self.Mmax, nstart), generator=g, dtype=torch.float64).to(self.dev)
        T = T * self.valid[:, :, None] / max(1.0, self.Mmax ** 0.5)
        idx = torch.argsort(self.diag, dim=1)[:, :nstart]              # [B, nstart]
        unit = torch.eye(nstart, dtype=torch.float64, device=self.dev)[None].expand(self.B, nstart, nstart)
        T.scatter_add_(1, idx[:, :, None].expand(self.B, nstart, nstart).contiguous(), unit.contiguous())
        return T * self.valid[:, :, None]


def davidson_batched(batch: "sci.Batch", tol: float = 1e-8, max_iter: int = 300, max_space: int = 24,
                     keep: int = 2, nstart: int = 4, schedule: int = sci.SCI_SCHED_AUTO) -> BatchDavidsonResult:
    """Lowest eigenpair of every instance of `batch` (a sci.Batch of real spin-orbital
    Hamiltonians): converged when ||H x - theta x|| <= tol for every instance."""
    pd = _Padded(batch)
    B, Mmax, dev = pd.B, pd.Mmax, pd.dev
    Cbuf = torch.zeros(pd.Mtot, dtype=torch.float64, device=dev)
    Sbuf = torch.zeros(pd.Mtot, dtype=torch.float64, device=dev)
    batch.plan(schedule, Cbuf.normal_(), Sbuf)
    batch.capture(Cbuf, Sbuf)
    launches = 0
    V = torch.zeros((B, Mmax, max_space), dtype=torch.float64, device=dev)
    Wm = torch.zeros_like(V)
    G = torch.zeros((B, max_space, max_space), dtype=torch.float64, device=dev)
    k = 0

    def append(T):
        """Orthonormalise T [B, Mmax] against V[:, :, :k] (two passes), multiply it by H in
        one replay of the captured launch and append both; a direction with no remaining
        norm becomes a null column."""
        nonlocal k, launches
        T = T * pd.valid
        T = T / torch.linalg.vector_norm(T, dim=1, keepdim=True).clamp_min(1e-300)
        for _ in range(2):
            if k:
                Vk = V[:, :, :k]
                T = T - torch.bmm(Vk, torch.bmm(Vk.transpose(1, 2), T.unsqueeze(2))).squeeze(2)
        nrm = torch.linalg.vector_norm(T, dim=1, keepdim=True)
        null = nrm[:, 0] < 1e-8
        T = torch.where(null[:, None], torch.zeros_like(T), T / nrm.clamp_min(1e-300))
        Cbuf.copy_(pd.to_concat(T))
        batch.replay()
        launches += 1
        WT = pd.from_concat(Sbuf)
        V[:, :, k] = T
        Wm[:, :, k] = WT
        g = torch.bmm(V[:, :, :k + 1].transpose(1, 2), WT.unsqueeze(2)).squeeze(2)   # [B, k+1]
        G[:, :k + 1, k] = g
        G[:, k, :k + 1] = g
        G[null, k, k] = pd.penalty
        k += 1

    start = pd.start_block(max(1, min(nstart, max_space - 1)))
    for j in range(start.shape[2]):
        append(start[:, :, j])
    theta = rn = evecs = None
    it = 0
    for it in range(1, max_iter + 1):
        evals, evecs = torch.linalg.eigh(0.5 * (G[:, :k, :k] + G[:, :k, :k].transpose(1, 2)))
        theta, y = evals[:, 0], evecs[:, :, 0:1]
        x = torch.bmm(V[:, :, :k], y).squeeze(2)
        r = torch.bmm(Wm[:, :, :k], y).squeeze(2) - theta[:, None] * x
        rn = torch.linalg.vector_norm(r, dim=1)
        if bool((rn <= tol).all()):
            break
        if k == max_space:   # thick restart to the lowest `keep` Ritz vectors
            Y = evecs[:, :, :keep]
            V[:, :, :keep] = torch.bmm(V[:, :, :k], Y)
            Wm[:, :, :keep] = torch.bmm(Wm[:, :, :k], Y)
            G.zero_()
            G[:, :keep, :keep] = torch.diag_embed(evals[:, :keep])
            k = keep
        den = theta[:, None] - pd.diag
        den = torch.where(den.abs() < 1e-8, torch.full_like(den, 1e-8), den)
        append(torch.where(rn[:, None] > tol, r / den, torch.zeros_like(r)))
    evals, evecs = torch.linalg.eigh(0.5 * (G[:, :k, :k] + G[:, :k, :k].transpose(1, 2)))
    X = pd.to_concat(torch.bmm(V[:, :, :k], evecs[:, :, 0:1]).squeeze(2))
    rnh = rn.cpu().numpy()
    return BatchDavidsonResult(theta.cpu().numpy(), rnh, rnh <= tol, it, launches, X)
