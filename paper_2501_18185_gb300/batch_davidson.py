"""Ground states of many small Hamiltonians at once: a Davidson iteration for every
instance, with one batched sigma launch per iteration.

The instances are the sci.Hamiltonian contexts of a sci.Batch (heterogeneous sizes).
Every iteration applies H to the new search vector of every instance in one persistent
launch, replayed from a CUDA graph captured once over fixed vector buffers; instances
that have converged are switched off in that launch (sci_batch_set_active), so the late
iterations pay only for the instances still running.

The vectors of all instances lie end to end, as in the batch: the search space is one
column-major block V [k, sum M_i] (and W = H V), without padding.  Projections, norms,
Gram-Schmidt updates, residuals and the diagonal preconditioner are the segmented
products of libsci (sci_seg_tn / sci_seg_nn), one launch each for all instances.  The
projected matrices G_i = V_i^T H V_i stay on the device, [B, k, k], and their
eigenpairs come from one launch of libsci's batched Jacobi eigensolver
(sci_syev_batched); the only host read per iteration is the vector of residual norms.

All instances grow their space together (one column per iteration).  An instance that
has converged, or whose space is exhausted (M_i <= k), takes a null column: zero vector,
zero coupling, and a diagonal in G above its spectrum, so it is never chosen.  Restarts
are thick (the space collapses to the `keep` lowest Ritz vectors of each instance).

The method per instance is that of davidson.davidson with one root: diagonal
preconditioner (theta - H_II)^-1, convergence when ||H x - theta x|| <= tol.  The start
block is the same as there: unit vectors on the lowest diagonal entries plus a small
seeded random part, so that no instance starts inside one symmetry sector of its H.
"""
from __future__ import annotations

import contextlib
from dataclasses import dataclass

import numpy as np
import torch

from . import sci


@dataclass
class BatchDavidsonResult:
    energies: np.ndarray        # [B]
    residual_norms: np.ndarray  # [B]
    converged: np.ndarray       # [B] bool
    iterations: int
    sigma_launches: int
    vectors: torch.Tensor       # concatenated [sum M_i], instance i at batch.offsets[i]
    active_per_launch: list     # instances computed in each sigma launch


def start_block(offsets, diag: np.ndarray, nstart: int, seed: int = 20250130, noise: float = 1e-3) -> np.ndarray:
    """[nstart, sum M_i]: per instance, unit vectors on its nstart lowest diagonal entries
    (fewer if M_i < nstart) plus seeded N(0, noise^2 / M_i) entries."""
    M = int(offsets[-1])
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((nstart, M)) * noise
    for s in range(len(offsets) - 1):
        a, b = int(offsets[s]), int(offsets[s + 1])
        if b == a:
            continue
        T[:, a:b] /= np.sqrt(b - a)
        low = np.argsort(diag[a:b], kind="stable")[:nstart]
        T[np.arange(len(low)), a + low] += 1.0
    return T


def davidson_batched(batch: "sci.Batch", tol: float = 1e-8, max_iter: int = 300, max_space: int = 32,
                     keep: int = 4, nstart: int = 4, schedule: int = sci.SCI_SCHED_AUTO,
                     drop_converged: bool = True) -> BatchDavidsonResult:
    """Lowest eigenpair of every instance of `batch` (a sci.Batch of real spin-orbital
    Hamiltonians): converged when ||H x - theta x|| <= tol for every instance.

    max_space (<= 64) and keep: the search space of every instance and the Ritz vectors
    a restart keeps.  On the 64 FCI instances of 6-16 orbitals (tol 1e-8), (32, 4) took
    218 iterations and 1.99 s against 311 and 2.29 s for (24, 2), 200 and 2.09 s for
    (48, 6), 382 and 2.49 s for (16, 2): the slowest instance sets the count."""
    if not 2 <= max_space <= 64:
        raise ValueError("max_space must be in 2..64 (the batched eigensolver's limit)")
    dev = batch.device
    f64 = dict(dtype=torch.float64, device=dev)
    offsets = np.asarray(list(batch.offsets) + [batch.M], dtype=np.int64)
    B, M = len(offsets) - 1, int(batch.M)
    nstart = max(1, min(nstart, max_space - 1))
    keep = max(1, min(keep, max_space - 1))
    # the segment workspace is freed, and the batch's mask restored, on every exit
    with contextlib.ExitStack() as cleanup:
        seg = sci.Segments(offsets, kmax=max_space, device=dev.index)
        cleanup.callback(seg.close)
        diag = torch.cat([H.diagonal() for H in batch.hams]).to(**f64)
        penalty = 10.0 * float(diag.abs().max()) + 10.0 if M else 10.0
        V = torch.zeros((max_space + keep, M), **f64)   # rows >= max_space: restart scratch
        Wm = torch.zeros_like(V)
        T = torch.zeros(M, **f64)
        S = torch.zeros(M, **f64)
        batch.plan(schedule, T.normal_(), S)
        # on every exit the batch goes back to computing all instances
        cleanup.callback(batch.set_active, np.ones(B, dtype=bool))
        batch.capture(T, S)
        G = torch.zeros((B, max_space, max_space), **f64)
        ev_w = torch.empty((B, max_space), **f64)
        ev_V = torch.empty((B, max_space, max_space), **f64)

        def eig(k):
            """Eigenpairs of every G_s[:k, :k], ascending (one batched Jacobi launch)."""
            return sci.syev_batched(G, n=k, w=ev_w, V=ev_V)

        ones = torch.ones(B, **f64)
        act = np.ones(B, dtype=bool)          # instances not converged yet
        act_dev = ones.clone()
        launches, per_launch = 0, []
        k = 0

        def append():
            """T holds one direction per instance (zero for an instance that takes none):
            orthonormalise it against V[:k] (two Gram-Schmidt passes), multiply it by H in one
            replay, and append it to V, W and G."""
            nonlocal k, launches
            n0 = seg.tn(T, T)[:, 0].clone()
            for _ in range(2):
                if k:
                    seg.nn(T, ones, A1=V[:k], c1=seg.tn(V[:k], T), alpha1=-1.0)
            n1 = seg.tn(T, T)[:, 0]
            live = n1 > 1e-16 * n0                     # False also where T was zero
            scale = torch.where(live, torch.rsqrt(torch.where(live, n1, ones)), torch.zeros_like(n1))
            seg.nn(T, scale)
            batch.replay()
            launches += 1
            per_launch.append(int(act.sum()) if drop_converged else B)
            V[k].copy_(T)
            Wm[k].copy_(S)
            g = seg.tn(V[:k + 1], S)                    # [B, k+1]; zero for a null column
            G[:, :k + 1, k] = g
            G[:, k, :k + 1] = g
            G[:, k, k] = torch.where(live, g[:, k], torch.full_like(n1, penalty))
            k += 1

        st = start_block(offsets, diag.cpu().numpy(), nstart)
        for j in range(nstart):
            T.copy_(torch.from_numpy(st[j]))
            append()
        del st
        rn = np.zeros(B)
        theta_h = np.zeros(B)
        it = 0
        for it in range(1, max_iter + 1):
            evals, evecs = eig(k)
            theta, y = evals[:, 0].contiguous(), evecs[:, :, 0].contiguous()
            # residual H x - theta x = W y - theta V y of the running instances, into T
            yc = y * act_dev[:, None]
            seg.nn(T, None, A1=Wm[:k], c1=yc, A2=V[:k], c2=(theta[:, None] * yc).contiguous(), alpha2=-1.0)
            host = torch.stack([torch.sqrt(seg.tn(T, T)[:, 0]), theta]).cpu().numpy()   # the one host read
            rn = np.where(act, host[0], rn)
            theta_h = np.where(act, host[1], theta_h)
            done = act & (rn <= tol)
            if done.any():
                act &= ~done
                act_dev = torch.from_numpy(act.astype(np.float64)).to(dev)
                if drop_converged:
                    batch.set_active(act)
            if not act.any():
                break
            if k == max_space:   # thick restart to the lowest `keep` Ritz vectors
                Y = evecs[:, :, :keep]
                for j in range(keep):
                    cj = Y[:, :, j].contiguous()
                    seg.nn(V[max_space + j], None, A1=V[:k], c1=cj)
                    seg.nn(Wm[max_space + j], None, A1=Wm[:k], c1=cj)
                V[:keep].copy_(V[max_space:max_space + keep])
                Wm[:keep].copy_(Wm[max_space:max_space + keep])
                G.zero_()
                G[:, :keep, :keep] = torch.diag_embed(evals[:, :keep])
                k = keep
            # preconditioned residual of the running instances: T / (theta - H_II)
            seg.nn(T, act_dev, dg=diag, shift=theta)
            append()
        # Ritz vectors: unchanged for an instance since it converged (its later columns are
        # null and decoupled, and restarts keep its lowest Ritz vectors)
        evals, evecs = eig(k)
        X = torch.empty(M, **f64)
        seg.nn(X, None, A1=V[:k], c1=evecs[:, :, 0].contiguous())
        return BatchDavidsonResult(theta_h, rn, rn <= tol, it, launches, X, per_launch)
