"""Block Davidson eigensolvers over sigma = H X.

The paper diagonalises the variational space through matrix-vector products
sigma_i = H X_i whose elements are recomputed, never stored (Sec. 2.4, the
diagonalisation paragraph; MetaWave uses the iVI solver there).  These drivers use the
Davidson method with the diagonal preconditioner (E - H_II)^-1.  Every product with H goes
through libsci's sigma kernels; every tall-skinny product of the subspace algebra
(projections, Gram matrices, Ritz vectors, residuals) through libsci's block-vector
kernels (sci_bv_gemm_tn / sci_bv_gemm_nn); the small dense problems (the projected matrix
G = V^+ H V, its eigenpairs, the Gram eigenproblems of Gram-Schmidt) are solved in FP64
on the host.

Search space: V and W = H V live in preallocated [M, max_space] device buffers, so a new
block is orthonormalised, multiplied and appended in place; G is extended by its new
rows only.  Restarts are thick: the space collapses to the lowest `keep` Ritz vectors
(2 x nroots by default), V and W rotated in place.

Gram-Schmidt is block classical Gram-Schmidt, twice (more if the second pass still
removes a sizeable component), each pass followed by symmetric orthonormalisation of the
new block from its Gram matrix (directions whose remaining norm is below threshold are
dropped).  The Gram matrix of the projected block comes from the same pass as the
projection: for T' = T - V S with S = V^T T, T'^T T' = T^T T - S^T S.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
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


# ---------------------------------------------------------------- block operations
class TorchBlockOps:
    """Tall-skinny products through torch (CPU tensors, or complex data on the GPU)."""

    def tn(self, A, B) -> np.ndarray:
        """A^+ B as a host array."""
        return (A.conj().T @ B).cpu().numpy()

    def nn(self, C, a, A1=None, S1=None, A2=None, S2=None, beta=0.0, dg=None, shift=None, colsq=False):
        """C[:, :a] = A1 S1 + A2 S2 (+ beta C); optional residual norms and preconditioner
        (see sci_bv_gemm_nn).  Returns the column sums of squares when colsq."""
        acc = None
        for A, S in ((A1, S1), (A2, S2)):
            if A is None or S is None or A.shape[1] == 0:
                continue
            t = A @ torch.as_tensor(np.ascontiguousarray(S), dtype=A.dtype, device=A.device)
            acc = t if acc is None else acc + t
        if beta != 0.0:
            acc = acc + beta * C[:, :a]
        cs = (acc.abs() ** 2).sum(dim=0).real.cpu().numpy() if colsq else None
        if dg is not None:
            sh = torch.as_tensor(np.real(shift), dtype=torch.float64, device=C.device)
            den = sh[None, :] - dg[:, None]
            den = torch.where(den.abs() < 1e-8, torch.full_like(den, 1e-8), den)
            acc = acc / den.to(acc.dtype)
        C[:, :a] = acc
        return cs


class SciBlockOps:
    """Tall-skinny products through libsci's block-vector kernels (real FP64 CUDA tensors).

    arith "f64": FP64 FMA; "ds": paired FP32 on the FP32 pipes (48-bit significands,
    FP64 folds).  Work is queued on the torch stream current at construction."""

    def __init__(self, device, arith: str = "f64"):
        from . import sci

        self.sci = sci
        self.device = torch.device(device)
        idx = self.device.index if self.device.index is not None else torch.cuda.current_device()
        self.ctx = sci.sci_create(idx, torch.cuda.current_stream(self.device).cuda_stream)
        self.prec = {"f64": sci.SCI_PREC_F64, "ds": sci.SCI_PREC_F64_DS}[arith]

    def __del__(self):
        try:
            if getattr(self, "ctx", None) is not None:
                self.sci.sci_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    @staticmethod
    def _ld(x):
        assert x.dtype == torch.float64 and x.is_cuda and (x.shape[1] <= 1 or x.stride(1) == 1)
        return x.stride(0) if x.shape[0] > 1 else max(1, x.shape[1])

    def _dev(self, S):
        return torch.as_tensor(np.ascontiguousarray(S, dtype=np.float64), device=self.device)

    # one kernel call takes blocks of at most 16 columns, P = A^T B with at most
    # 8 * 256 / pow2(a) columns of A, and C = A1 S1 + A2 S2 with at most 256 columns in all;
    # larger products are cut into such calls here
    MAX_A, MAX_NN = 16, 256

    @staticmethod
    def _tn_kmax(a):
        p2 = 1
        while p2 < a:
            p2 <<= 1
        return 8 * (256 // p2)

    def tn(self, A, B) -> np.ndarray:
        M, k = A.shape
        a = B.shape[1]
        P = torch.empty((k, a), dtype=torch.float64, device=self.device)
        for j0 in range(0, a, self.MAX_A):
            j1 = min(a, j0 + self.MAX_A)
            kmax = self._tn_kmax(j1 - j0)
            for i0 in range(0, k, kmax):
                i1 = min(k, i0 + kmax)
                Pc = P[i0:i1, j0:j1] if (j0 == 0 and j1 == a) else torch.empty((i1 - i0, j1 - j0), dtype=torch.float64,
                                                                                 device=self.device)
                Ai, Bj = A[:, i0:i1], B[:, j0:j1]
                self.sci.sci_bv_gemm_tn(self.ctx, M, i1 - i0, j1 - j0, Ai, self._ld(Ai), Bj, self._ld(Bj), Pc, self.prec)
                if not (j0 == 0 and j1 == a):
                    P[i0:i1, j0:j1] = Pc
        return P.cpu().numpy()

    def nn(self, C, a, A1=None, S1=None, A2=None, S2=None, beta=0.0, dg=None, shift=None, colsq=False):
        """C[:, :a] = A1 S1 + A2 S2 (+ beta C), the epilogue as in sci_bv_gemm_nn.  One call
        is row-local, so C may alias A1 or A2 (in-place updates).  A product wider than one
        call is cut into calls over output columns and operand segments (beta = 1 after the
        first, the epilogue on the last) that write a temporary, copied to C at the end."""
        M = C.shape[0]
        segs = []  # (A, S) operand segments of at most MAX_NN columns
        for A, S in ((A1, S1), (A2, S2)):
            if A is None or A.shape[1] == 0:
                continue
            for i0 in range(0, A.shape[1], self.MAX_NN):
                i1 = min(A.shape[1], i0 + self.MAX_NN)
                segs.append((A[:, i0:i1], np.asarray(S)[i0:i1]))
        calls = [segs] if sum(x[0].shape[1] for x in segs) <= self.MAX_NN else [[sg] for sg in segs]
        chunked = a > self.MAX_A or len(calls) > 1
        out = C
        if chunked:
            out = C[:, :a].clone() if beta != 0.0 else torch.empty((M, a), dtype=torch.float64, device=self.device)
        cs_all = np.zeros(a) if colsq else None
        for j0 in range(0, a, self.MAX_A):
            j1 = min(a, j0 + self.MAX_A)
            for ci, ops in enumerate(calls):
                last = ci == len(calls) - 1
                A1c, S1c = (ops[0][0], ops[0][1][:, j0:j1]) if len(ops) > 0 else (None, None)
                A2c, S2c = (ops[1][0], ops[1][1][:, j0:j1]) if len(ops) > 1 else (None, None)
                k1 = 0 if A1c is None else A1c.shape[1]
                k2 = 0 if A2c is None else A2c.shape[1]
                s1 = self._dev(S1c) if k1 else None
                s2 = self._dev(S2c) if k2 else None
                use_epi = last and dg is not None
                sh = self._dev(np.real(np.asarray(shift))[j0:j1]) if use_epi else None
                cs = torch.zeros(j1 - j0, dtype=torch.float64, device=self.device) if (colsq and last) else None
                Cc = out[:, j0:]
                self.sci.sci_bv_gemm_nn(self.ctx, M, j1 - j0, A1c, self._ld(A1c) if k1 else 1, k1, s1, A2c,
                                        self._ld(A2c) if k2 else 1, k2, s2, beta if ci == 0 else 1.0, Cc, self._ld(Cc),
                                        dg if use_epi else None, sh, cs, self.prec)
                if cs is not None:
                    cs_all[j0:j1] = cs.cpu().numpy()
        if chunked:
            C[:, :a].copy_(out)
        return cs_all


def default_ops(diag: torch.Tensor, dtype, arith: str = "f64"):
    """libsci block kernels for real data on the GPU, torch otherwise."""
    if diag.is_cuda and dtype == torch.float64:
        return SciBlockOps(diag.device, arith)
    return TorchBlockOps()


# ---------------------------------------------------------------- search space
class _Space:
    """V, W = H V in [M, cap] buffers; G = V^+ H V on the host; ex marks the columns of W
    that come from the FP64 product (mixed solver)."""

    def __init__(self, ops, M, cap, dtype, device):
        self.ops = ops
        self.V = torch.zeros((M, cap), dtype=dtype, device=device)
        self.W = torch.zeros((M, cap), dtype=dtype, device=device)
        self.k = 0
        self.G = np.zeros((0, 0), dtype=np.complex128 if dtype.is_complex else np.float64)
        self.ex = np.zeros(0, dtype=bool)

    def orthonormalize_new(self, a: int) -> int:
        """Orthonormalise V[:, k:k+a] against V[:, :k] and among themselves, in place.
        Returns the number of directions kept (packed to the front of the block)."""
        V, k, ops = self.V, self.k, self.ops
        for p in range(4):
            if a == 0:
                return 0
            P = ops.tn(V[:, :k + a], V[:, k:k + a])
            S, Gm = P[:k], P[k:]
            Gm = 0.5 * (Gm + Gm.conj().T)
            d = np.sqrt(np.maximum(np.real(np.diag(Gm)), 1e-300))
            Gp = Gm - S.conj().T @ S
            Gn = Gp / d[:, None] / d[None, :]
            lam, U = np.linalg.eigh(0.5 * (Gn + Gn.conj().T))
            keep = lam > (1e-12 if p == 0 else 1e-10)
            Z = (U[:, keep] / np.sqrt(lam[keep])[None, :]) / d[:, None]
            if Z.shape[1] == 0:
                return 0
            ops.nn(V[:, k:], Z.shape[1], A1=V[:, :k] if k else None, S1=-(S @ Z) if k else None,
                   A2=V[:, k:k + a], S2=Z)
            a = Z.shape[1]
            # stop once a pass after the first removed only a rounding-level component
            if p >= 1 and (k == 0 or np.abs(S).max() < 1e-10 * d.max()) and np.abs(lam[keep] - 1).max(initial=0) < 1e-8:
                break
        return a

    def append(self, a: int, WT, exact: bool, mixed: bool):
        """W[:, k:k+a] = WT (= H V[:, k:k+a]); extend G by the new rows and columns."""
        V, W, k, ops = self.V, self.W, self.k, self.ops
        W[:, k:k + a].copy_(WT)
        P1 = ops.tn(V[:, :k + a], W[:, k:k + a])            # v_i^+ (H t_j)
        B, C = P1[:k].copy(), P1[k:]
        if mixed and not exact:
            # rows of columns with an exact product take the exact side (H v_i)^+ t_j; the
            # exact columns are a prefix (the refined block), so one narrow product serves
            nex = int(self.ex.sum())
            assert self.ex[:nex].all()
            if nex:
                B[:nex] = ops.tn(W[:, :nex], V[:, k:k + a])
        C = 0.5 * (C + C.conj().T)
        G = np.zeros((k + a, k + a), dtype=self.G.dtype)
        G[:k, :k], G[:k, k:], G[k:, :k], G[k:, k:] = self.G, B, B.conj().T, C
        self.G = G
        self.ex = np.concatenate([self.ex, np.full(a, exact)])
        self.k = k + a

    def rotate(self, Yk: np.ndarray, with_w: bool = True):
        """V <- V Yk (and W <- W Yk) in place (columns of Yk orthonormal)."""
        k, m = self.k, Yk.shape[1]
        self.ops.nn(self.V, m, A1=self.V[:, :k], S1=Yk)
        if with_w:
            self.ops.nn(self.W, m, A1=self.W[:, :k], S1=Yk)
        self.ex = np.full(m, bool(self.ex.all()))
        self.k = m

    def residual(self, Y, theta, diag, ops=None):
        """Preconditioned residuals (H x - theta x) / (theta - H_II) of the Ritz vectors
        x = V Y, written to V[:, k:k+r]; returns the residual 2-norms.  ops: the block
        backend for this product (default: the space's own)."""
        k, r = self.k, Y.shape[1]
        cs = (ops or self.ops).nn(self.V[:, k:], r, A1=self.W[:, :k], S1=Y, A2=self.V[:, :k],
                                  S2=-(Y * theta[None, :]), dg=diag, shift=theta, colsq=True)
        return np.sqrt(np.maximum(cs, 0.0))

    def ritz_vectors(self, Y):
        X = torch.empty((self.V.shape[0], Y.shape[1]), dtype=self.V.dtype, device=self.V.device)
        self.ops.nn(X, Y.shape[1], A1=self.V[:, :self.k], S1=Y)
        return X


def _guess_block(sp: _Space, diag, nvec, seed: int = 20250130, noise: float = 1e-3) -> int:
    """Unit vectors on the lowest diagonal entries plus a small seeded random part, into
    V[:, :nvec].  Without the random part the start block can lie entirely in one symmetry
    sector of H (e.g. have exactly zero overlap with the ground state), which a
    symmetry-blind solver would then never leave."""
    M = diag.shape[0]
    k = min(M, nvec)
    idx = torch.argsort(diag)[:k]
    g = torch.Generator(device="cpu").manual_seed(seed)
    B = noise * torch.randn((M, k), generator=g, dtype=torch.float64) / (M ** 0.5)
    sp.V[:, :k].copy_(B.to(sp.V.device).to(sp.V.dtype))
    sp.V[idx, torch.arange(k, device=sp.V.device)] += 1.0
    return sp.orthonormalize_new(k)


def _start(sigma, diag, nroots, max_space, keep, guess, dtype, ops, arith):
    M = diag.shape[0]
    keep = min(M, keep or 2 * nroots)
    max_space = min(M, max_space or max(12 * nroots, keep + 2 * nroots, 24))
    ops = ops or default_ops(diag, dtype, arith)
    sp = _Space(ops, M, max_space + 2 * nroots, dtype, diag.device)
    if guess is None:
        a = _guess_block(sp, diag, max(keep, 8))
    else:
        a = guess.shape[1]
        sp.V[:, :a].copy_(guess.to(dtype))
        a = sp.orthonormalize_new(a)
    return sp, a, keep, max_space


def _ritz(sp: _Space, nroots):
    evals, evecs = np.linalg.eigh(sp.G)
    return evals, evecs, evals[:nroots].real.copy(), evecs[:, :nroots]


def davidson(sigma, diag: torch.Tensor, nroots: int = 1, tol: float = 1e-9, max_iter: int = 300,
             max_space: int | None = None, keep: int | None = None, guess: torch.Tensor | None = None,
             dtype=torch.float64, ops=None, arith: str = "f64") -> DavidsonResult:
    """Lowest `nroots` eigenpairs of H.

    sigma(X [M,k]) -> H X (same dtype); diag: H_II (float64, [M]).  Converged when every
    root's residual 2-norm ||H x - E x|| <= tol.  ops: block-product backend (default:
    libsci block kernels for real CUDA data, arithmetic `arith`).
    """
    sp, a, keep, max_space = _start(sigma, diag, nroots, max_space, keep, guess, dtype, ops, arith)
    calls = 0
    hist = []
    theta = rn = Y = None
    for it in range(1, max_iter + 1):
        if a == 0:
            break
        WT = sigma(sp.V[:, sp.k:sp.k + a].contiguous())
        calls += 1
        sp.append(a, WT, True, False)
        evals, evecs, theta, Y = _ritz(sp, nroots)
        rn = sp.residual(Y, theta, diag)
        hist.append((it, theta.copy(), rn.copy()))
        if bool((rn <= tol).all()):
            return _result(sp, theta, Y, rn, it, calls, True, hist, 0, calls)
        active = np.nonzero(rn > tol)[0]
        if sp.k + len(active) > max_space:
            old_k = sp.k
            sp.rotate(evecs[:, :min(keep, sp.k)])
            sp.G = np.diag(evals[:sp.k]).astype(sp.G.dtype)
            # the Ritz vectors and their residuals are unchanged by the rotation
            sp.V[:, sp.k:sp.k + nroots] = sp.V[:, old_k:old_k + nroots].clone()
        _pack(sp, nroots, active)
        a = sp.orthonormalize_new(len(active))
    return _result(sp, theta, Y, rn, max_iter, calls, False, hist, 0, calls)


def _pack(sp: _Space, nroots, active):
    """Move the preconditioned residuals of the active roots to the front of the block."""
    k = sp.k
    if len(active) < nroots:
        sp.V[:, k:k + len(active)] = sp.V[:, k + torch.as_tensor(active, device=sp.V.device)]


def _result(sp, theta, Y, rn, it, calls, conv, hist, lo, hi):
    X = sp.ritz_vectors(Y) if Y is not None else None
    dev = sp.V.device
    return DavidsonResult(torch.as_tensor(theta, device=dev), X, torch.as_tensor(rn, device=dev), it, calls, conv, hist,
                          lo, hi)


def davidson_mixed(sigma_lo, sigma_hi, diag: torch.Tensor, nroots: int = 1, tol: float = 1e-6,
                   max_iter: int = 400, max_space: int | None = None, keep: int | None = None,
                   guess: torch.Tensor | None = None, dtype=torch.float64, ops=None,
                   arith: str = "f64", est_arith: str | None = "ds") -> DavidsonResult:
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
    quotient, the final energies and the exact residuals that decide convergence.

    est_arith: block arithmetic of the residual estimates of iterations whose space holds
    low-precision columns ("ds": paired FP32, the default; "f64" or None: the space's
    own).  Those residuals carry the FP32-storage error of sigma_lo; the paired-FP32
    product adds ~2^-47 of its operands, far below it, at ~5x the FP64 rate.

    max_space defaults to 16 x nroots (12 x nroots in `davidson`): every collapse of a full
    space costs this solver an FP64 product of the kept vectors, so a larger space, with
    fewer collapses, pays here (8 roots, 2M space, 1e-8 Eh: 4.71 s at 128 columns against
    4.82 s at 96; plain FP64 is fastest at 96).
    """
    if max_space is None:
        max_space = max(16 * nroots, 24)
    sp, a, keep, max_space = _start(sigma_lo, diag, nroots, max_space, keep, guess, dtype, ops, arith)
    est_ops = None
    if est_arith == "ds" and isinstance(sp.ops, SciBlockOps) and arith == "f64":
        est_ops = SciBlockOps(diag.device, "ds")
    calls_lo, calls_hi = 0, 0
    best_est, stall = None, 0
    hist = []
    theta = rn = Y = None
    exact_next = False
    for it in range(1, max_iter + 1):
        if a == 0:
            break
        X = sp.V[:, sp.k:sp.k + a].contiguous()
        if exact_next:
            WT = sigma_hi(X)
            calls_hi += 1
        else:
            WT = sigma_lo(X)
            calls_lo += 1
        sp.append(a, WT, exact_next, True)
        exact_next = False
        evals, evecs, theta, Y = _ritz(sp, nroots)
        exact = bool(sp.ex.all())
        rn = sp.residual(Y, theta, diag, ops=None if exact else est_ops)
        rmax = float(rn.max())
        hist.append((it, theta.copy(), rn.copy(), exact))
        if exact and rmax <= tol:
            return _result(sp, theta, Y, rn, it, calls_lo + calls_hi, True, hist, calls_lo, calls_hi)
        refine = False
        if exact:
            best_est, stall = rmax, 0
        else:
            if best_est is None or rmax < 0.9 * best_est:
                best_est, stall = rmax, 0
            else:
                stall += 1
            refine = rmax <= tol or stall >= 6
        active = np.nonzero(rn > tol)[0]
        # a full space also collapses with FP64 products: rotating the stored W would mix
        # the FP32 error into the exact block of the kept Ritz vectors
        if refine or sp.k + len(active) > max_space:
            m = min(keep, sp.k)
            sp.rotate(evecs[:, :m], with_w=False)
            # the kept Ritz vectors become the next block, multiplied in FP64
            sp.k, a = 0, m
            sp.G = sp.G[:0, :0]
            sp.ex = sp.ex[:0]
            exact_next = True
            best_est, stall = None, 0
            continue
        _pack(sp, nroots, active)
        a = sp.orthonormalize_new(len(active))
    return _result(sp, theta, Y, rn, max_iter, calls_lo + calls_hi, False, hist, calls_lo, calls_hi)
