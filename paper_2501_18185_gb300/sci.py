"""Python binding of libsci (include/sci.h): argument marshalling only.

Every step of the sigma path runs in the CUDA kernels of libsci.so; this module passes
pointers and sizes.  PyTorch supplies device memory and the stream.  There is no CPU
fallback: if libsci.so is missing or no GPU is visible, the calls raise.

The functions named sci_* mirror the C entry points one to one; ``Hamiltonian`` is a
small convenience class over them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

SCI_OK = 0
SCI_ERR_ARG = -1
SCI_ERR_UNSORTED = -2
SCI_ERR_DUPLICATE = -3
SCI_ERR_POPCOUNT = -4
SCI_ERR_NOMEM = -5
SCI_ERR_CUDA = -6
SCI_ERR_STATE = -7
SCI_ERR_OVERFLOW = -8
SCI_ERR_TIMEOUT = -9
SCI_REAL64, SCI_COMPLEX128 = 1, 2
SCI_SPIN_ORBITALS, SCI_SPINORS = 1, 2
SCI_PREC_F64, SCI_PREC_F32_STORE_F64_ACC, SCI_PREC_F64_DS = 1, 2, 3

# every entry point declared in include/sci.h, with (restype, argtypes)
_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
SIGNATURES = {
    "sci_create": (_i32, [ctypes.POINTER(_vp), _i32, _vp]),
    "sci_destroy": (_i32, [_vp]),
    "sci_set_stream": (_i32, [_vp, _vp]),
    "sci_set_integrals": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _i32, _vp]),
    "sci_set_integrals_ex": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _i32, _vp, _i32]),
    "sci_set_determinants": (_i32, [_vp, _vp, _i64, _i32, _i32, _i32]),
    "sci_set_determinants_w": (_i32, [_vp, _vp, _i32, _i64, _i32, _i32, _i32]),
    "sci_diagonal": (_i32, [_vp, _vp]),
    "sci_sigma": (_i32, [_vp, _vp, _vp, _i32, _i32]),
    "sci_set_row_range": (_i32, [_vp, _i64, _i64]),
    "sci_set_tile_threshold": (_i32, [_vp, _i32]),
    "sci_row_costs": (_i32, [_vp, _vp]),
    "sci_set_deterministic": (_i32, [_vp, _i32]),
    "sci_connections": (_i32, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _i64]),
    "sci_connections_noalloc": (_i32, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _i64]),
    "sci_count_pairs": (_i32, [_vp, _vp]),
    "sci_sigma_host": (_i32, [_vp, _vp, _vp, _i32, _i32]),
    "sci_info": (_i32, [_vp, _vp, _i32]),
    "sci_profile": (_i32, [_vp, _i32]),
    "sci_kernel_times": (_i32, [_vp, _vp, _i32]),
    "sci_rdm12": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp]),
    "sci_rdm_grads": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _i32, _vp, _vp]),
    "sci_enpt2": (_i32, [_vp, _vp, _i32, _vp, ctypes.c_double, ctypes.c_size_t, _vp, _vp]),
    "sci_batch_create": (_i32, [ctypes.POINTER(_vp), _i32, _vp]),
    "sci_batch_destroy": (_i32, [_vp]),
    "sci_batch_add": (_i32, [_vp, _vp]),
    "sci_batch_plan": (_i32, [_vp, _i32, _vp, _vp]),
    "sci_batch_sigma": (_i32, [_vp, _vp, _vp]),
    "sci_batch_capture": (_i32, [_vp, _vp, _vp]),
    "sci_batch_replay": (_i32, [_vp]),
    "sci_batch_set_active": (_i32, [_vp, _vp, _i32]),
    "sci_batch_info": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "sci_batch_items": (_i32, [_vp, _vp, _i32]),
    "sci_batch_last_error": (ctypes.c_char_p, [_vp]),
    "sci_seg_create": (_i32, [ctypes.POINTER(_vp), _i32, _i32, _vp, _i32, _vp]),
    "sci_seg_destroy": (_i32, [_vp]),
    "sci_seg_tn": (_i32, [_vp, _i32, _vp, _i64, _vp, _vp]),
    "sci_seg_nn": (_i32, [_vp, _vp, _vp, _i32, _vp, _i64, _vp, ctypes.c_double, _i32, _vp, _i64, _vp,
                          ctypes.c_double, _vp, _vp]),
    "sci_seg_last_error": (ctypes.c_char_p, [_vp]),
    "sci_syev_batched": (_i32, [_i32, _i32, _i32, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _i64, _i32, _vp, _vp]),
    "sci_bv_gemm_tn": (_i32, [_vp, _i64, _i32, _i32, _vp, _i64, _vp, _i64, _vp, _i32]),
    "sci_bv_gemm_nn": (_i32, [_vp, _i64, _i32, _vp, _i64, _i32, _vp, _vp, _i64, _i32, _vp, ctypes.c_double, _vp,
                              _i64, _vp, _vp, _vp, _i32]),
    "sci_peak_fma": (_i32, [_i32, _i32, _i32, _vp, _vp]),
    "sci_sync_status": (_i32, [_vp]),
    "sci_last_error": (ctypes.c_char_p, [_vp]),
}

_lib = None


class SciError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libsci error {code}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Load libsci.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is not built: run paper_2501_18185_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = L
    return L


def _check(ctx, rc):
    if rc != SCI_OK:
        msg = load().sci_last_error(ctx) if ctx else b""
        raise SciError(rc, (msg or b"").decode())
    return rc


def _p(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


# ---------------------------------------------------------------- thin C mirrors
def sci_create(device: int = 0, stream: int | None = None):
    ctx = ctypes.c_void_p()
    rc = load().sci_create(ctypes.byref(ctx), device, ctypes.c_void_p(stream or 0))
    if rc != SCI_OK:
        raise SciError(rc, "sci_create failed")
    return ctx


def sci_destroy(ctx):
    return load().sci_destroy(ctx)


def sci_set_stream(ctx, stream: int | None):
    return _check(ctx, load().sci_set_stream(ctx, ctypes.c_void_p(stream or 0)))


def sci_set_integrals(ctx, scalar, mode, n, h, eri=None, naux=0, chol=None):
    return _check(ctx, load().sci_set_integrals(ctx, scalar, mode, n, _p(h), _p(eri), naux, _p(chol)))


def sci_set_integrals_ex(ctx, scalar, mode, n, h, eri=None, naux=0, chol=None, on_device=0):
    return _check(ctx, load().sci_set_integrals_ex(ctx, scalar, mode, n, _p(h), _p(eri), naux, _p(chol),
                                                   int(on_device)))


def sci_set_determinants(ctx, keys, M, n_alpha, n_beta, keys_on_device):
    return _check(ctx, load().sci_set_determinants(ctx, _p(keys), M, n_alpha, n_beta, keys_on_device))


def sci_set_determinants_w(ctx, keys, nwords, M, n_alpha, n_beta, keys_on_device):
    return _check(ctx, load().sci_set_determinants_w(ctx, _p(keys), nwords, M, n_alpha, n_beta, keys_on_device))


def sci_diagonal(ctx, hdiag):
    return _check(ctx, load().sci_diagonal(ctx, _p(hdiag)))


def sci_sigma(ctx, C, S, nvec, prec):
    return _check(ctx, load().sci_sigma(ctx, _p(C), _p(S), nvec, prec))


def sci_set_row_range(ctx, row_begin, row_end):
    return _check(ctx, load().sci_set_row_range(ctx, int(row_begin), int(row_end)))


def sci_set_tile_threshold(ctx, members):
    return _check(ctx, load().sci_set_tile_threshold(ctx, int(members)))


def sci_set_deterministic(ctx, max_nvec: int):
    return _check(ctx, load().sci_set_deterministic(ctx, int(max_nvec)))


def sci_row_costs(ctx, cost):
    return _check(ctx, load().sci_row_costs(ctx, _p(cost)))


def sci_connections(ctx, row_begin, row_end, cap):
    cnt = np.zeros(1, dtype=np.int64)
    rows = np.zeros(max(cap, 1), dtype=np.int64)
    J = np.zeros(max(cap, 1), dtype=np.int64)
    deg = np.zeros(max(cap, 1), dtype=np.int8)
    ph = np.zeros(max(cap, 1), dtype=np.int8)
    rc = load().sci_connections(ctx, row_begin, row_end, _p(cnt), _p(rows), _p(J), _p(deg), _p(ph), cap)
    if rc == SCI_ERR_OVERFLOW:
        return int(cnt[0]), None
    _check(ctx, rc)
    n = int(cnt[0])
    return n, (rows[:n], J[:n], deg[:n], ph[:n])


def sci_connections_noalloc(ctx, row_begin, row_end, cap):
    """The connection export for callers that cannot allocate device memory: the
    library uses a fixed device scratch array instead (see include/sci.h)."""
    cnt = np.zeros(1, dtype=np.int64)
    rows = np.zeros(max(cap, 1), dtype=np.int64)
    J = np.zeros(max(cap, 1), dtype=np.int64)
    deg = np.zeros(max(cap, 1), dtype=np.int8)
    ph = np.zeros(max(cap, 1), dtype=np.int8)
    rc = load().sci_connections_noalloc(ctx, row_begin, row_end, _p(cnt), _p(rows), _p(J), _p(deg), _p(ph), cap)
    if rc == SCI_ERR_OVERFLOW:
        return int(cnt[0]), None
    _check(ctx, rc)
    n = int(cnt[0])
    return n, (rows[:n], J[:n], deg[:n], ph[:n])


def sci_count_pairs(ctx) -> int:
    out = np.zeros(1, dtype=np.int64)
    _check(ctx, load().sci_count_pairs(ctx, _p(out)))
    return int(out[0])


def sci_sigma_host(ctx, C, S, nvec, prec):
    return _check(ctx, load().sci_sigma_host(ctx, _p(C), _p(S), nvec, prec))


def sci_info(ctx) -> dict:
    out = np.zeros(10, dtype=np.int64)
    _check(ctx, load().sci_info(ctx, _p(out), 10))
    keys = ["M", "pairs", "b2_entries", "b2_buckets", "b1_entries", "b1_buckets", "max_bucket", "device_bytes",
            "pairs_doubles", "pairs_singles"]
    return dict(zip(keys, (int(v) for v in out)))


def sci_profile(ctx, enable: bool):
    return _check(ctx, load().sci_profile(ctx, int(enable)))


def sci_kernel_times(ctx, n: int = 3) -> list:
    ms = np.zeros(n, dtype=np.float32)
    _check(ctx, load().sci_kernel_times(ctx, _p(ms), n))
    return [float(x) for x in ms]


def sci_rdm12(ctx, C, nvec, weights, rdm1, rdm2):
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    return _check(ctx, load().sci_rdm12(ctx, _p(C), nvec, _p(w), _p(rdm1), _p(rdm2)))


def sci_rdm_grads(ctx, C, nvec, weights, gamma, Gamma, naux, chol, gchol):
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    return _check(ctx, load().sci_rdm_grads(ctx, _p(C), nvec, _p(w), _p(gamma), _p(Gamma), int(naux), _p(chol),
                                            _p(gchol)))


def sci_enpt2(ctx, C, nroots, E0, eps=0.0, table_bytes=1 << 30):
    """(E2[W], E2[P], E2[Q]) as three arrays of nroots, and the stats dict."""
    e0 = np.ascontiguousarray(E0, dtype=np.float64).reshape(-1)
    out = np.zeros(3 * nroots, dtype=np.float64)
    st = np.zeros(8, dtype=np.int64)
    _check(ctx, load().sci_enpt2(ctx, _p(C), nroots, _p(e0), float(eps), int(table_bytes), _p(out), _p(st)))
    stats = dict(zip(["batches", "distinct_W", "passes", "table_capacity", "clear_us", "generate_us", "evaluate_us",
                      "sample_distinct"], (int(v) for v in st)))
    return out[:nroots], out[nroots:2 * nroots], out[2 * nroots:], stats


SCI_SCHED_AUTO, SCI_SCHED_TILE, SCI_SCHED_WARP = 0, 1, 2


def _bcheck(b, rc):
    if rc < 0:
        msg = load().sci_batch_last_error(b) if b else b""
        raise SciError(rc, (msg or b"").decode())
    return rc


def sci_batch_create(device: int = 0, stream: int | None = None):
    b = ctypes.c_void_p()
    rc = load().sci_batch_create(ctypes.byref(b), device, ctypes.c_void_p(stream or 0))
    if rc != SCI_OK:
        raise SciError(rc, "sci_batch_create failed")
    return b


def sci_batch_destroy(b):
    return load().sci_batch_destroy(b)


def sci_batch_add(b, ctx) -> int:
    return _bcheck(b, load().sci_batch_add(b, ctx))


def sci_batch_plan(b, schedule, C=None, S=None):
    return _bcheck(b, load().sci_batch_plan(b, schedule, _p(C), _p(S)))


def sci_batch_sigma(b, C, S):
    return _bcheck(b, load().sci_batch_sigma(b, _p(C), _p(S)))


def sci_batch_capture(b, C, S):
    return _bcheck(b, load().sci_batch_capture(b, _p(C), _p(S)))


def sci_batch_replay(b):
    return _bcheck(b, load().sci_batch_replay(b))


def sci_batch_set_active(b, active):
    a = np.ascontiguousarray(active, dtype=np.int32)
    return _bcheck(b, load().sci_batch_set_active(b, _p(a), int(a.size)))


def sci_batch_info(b, i) -> dict:
    sch = ctypes.c_int()
    mt, mw = ctypes.c_float(), ctypes.c_float()
    off = ctypes.c_int64()
    _bcheck(b, load().sci_batch_info(b, i, ctypes.byref(sch), ctypes.byref(mt), ctypes.byref(mw), ctypes.byref(off)))
    return {"schedule": {0: "auto", 1: "tile", 2: "warp"}[sch.value], "ms_tile": mt.value, "ms_warp": mw.value,
            "offset": off.value}


def sci_batch_items(b) -> dict:
    out = np.zeros(4, dtype=np.int64)
    _bcheck(b, load().sci_batch_items(b, _p(out), 4))
    return dict(zip(["items", "ctas", "M", "pairs"], (int(v) for v in out)))


def _scheck(sg, rc):
    if rc < 0:
        msg = load().sci_seg_last_error(sg) if sg else b""
        raise SciError(rc, (msg or b"").decode())
    return rc


def sci_seg_create(device, offsets, kmax, stream=None):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    sg = ctypes.c_void_p()
    rc = load().sci_seg_create(ctypes.byref(sg), device, int(off.size) - 1, _p(off), int(kmax), ctypes.c_void_p(stream or 0))
    if rc != SCI_OK:
        raise SciError(rc, "sci_seg_create failed")
    return sg


def sci_seg_destroy(sg):
    return load().sci_seg_destroy(sg)


def sci_seg_tn(sg, k, A, lda, t, out):
    return _scheck(sg, load().sci_seg_tn(sg, k, _p(A), lda, _p(t), _p(out)))


def sci_seg_nn(sg, y, beta, k1, A1, lda1, c1, alpha1, k2, A2, lda2, c2, alpha2, dg=None, shift=None):
    return _scheck(sg, load().sci_seg_nn(sg, _p(y), _p(beta), k1, _p(A1), lda1, _p(c1), float(alpha1), k2, _p(A2), lda2,
                                         _p(c2), float(alpha2), _p(dg), _p(shift)))


def sci_syev_batched(device, nb, n, A, lda, strideA, w, stridew, V, ldv, strideV, max_sweeps=30, not_converged=None,
                     stream=None):
    rc = load().sci_syev_batched(device, nb, n, _p(A), lda, strideA, _p(w), stridew, _p(V), ldv, strideV, max_sweeps,
                                 _p(not_converged), ctypes.c_void_p(stream or 0))
    if rc != SCI_OK:
        raise SciError(rc, "sci_syev_batched failed")
    return rc


def syev_batched(G, n=None, w=None, V=None, max_sweeps=30):
    """Eigenvalues (ascending) and eigenvectors (columns) of the leading n x n blocks of
    the symmetric float64 CUDA matrices G [nb, >= n, >= n] (row-major inner dims).
    Returns (w [nb, n], V [nb, n, n]) as views of the given or new buffers."""
    import torch

    nb = G.shape[0]
    n = G.shape[1] if n is None else n
    assert G.dtype == torch.float64 and G.is_cuda and G.stride(2) == 1
    if w is None:
        w = torch.empty((nb, n), dtype=torch.float64, device=G.device)
    if V is None:
        V = torch.empty((nb, n, n), dtype=torch.float64, device=G.device)
    assert w.stride(1) == 1 and V.stride(2) == 1 and w.shape[1] >= n and V.shape[1] >= n and V.shape[2] >= n
    stream = torch.cuda.current_stream(G.device).cuda_stream
    sci_syev_batched(G.device.index or 0, nb, n, G, G.stride(1), G.stride(0), w, w.stride(0), V, V.stride(1),
                     V.stride(0), max_sweeps, None, stream)
    return w[:, :n], V[:, :n, :n]


def sci_bv_gemm_tn(ctx, M, k, a, A, lda, B, ldb, P, prec):
    return _check(ctx, load().sci_bv_gemm_tn(ctx, M, k, a, _p(A), lda, _p(B), ldb, _p(P), prec))


def sci_bv_gemm_nn(ctx, M, a, A1, lda1, k1, S1, A2, lda2, k2, S2, beta, C, ldc, dg, shift, colsq, prec):
    return _check(ctx, load().sci_bv_gemm_nn(ctx, M, a, _p(A1), lda1, k1, _p(S1), _p(A2), lda2, k2, _p(S2), float(beta),
                                             _p(C), ldc, _p(dg), _p(shift), _p(colsq), prec))


def sci_peak_fma(device: int, prec: int, iters: int, stream: int | None = None) -> float:
    """Measured FMAs per second of the FP64 (SCI_PREC_F64) or FP32
    (SCI_PREC_F32_STORE_F64_ACC) pipes -- see sci_peak_fma in include/sci.h."""
    out = np.zeros(1, dtype=np.float64)
    rc = load().sci_peak_fma(device, prec, iters, ctypes.c_void_p(stream or 0), _p(out))
    if rc != SCI_OK:
        raise SciError(rc, "sci_peak_fma failed")
    return float(out[0])


def sci_sync_status(ctx):
    return _check(ctx, load().sci_sync_status(ctx))


def sci_last_error(ctx) -> str:
    return (load().sci_last_error(ctx) or b"").decode()


# ---------------------------------------------------------------- convenience class
class Hamiltonian:
    """One libsci context: integrals + a sorted determinant list on one GPU.

    mode "spin_orbitals" (n <= 32 spatial orbitals, real) or "spinors" (n <= 64 spinors,
    complex).  Tensors are torch CUDA tensors on the context's device; work is queued on
    the torch stream that is current when the context is created (or set_stream()).
    """

    def __init__(self, device: int = 0, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libsci needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.device = torch.device("cuda", device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = s
        self.ctx = sci_create(device, s.cuda_stream)
        self.mode = None
        self.M = 0
        self.complex = False

    def close(self):
        if getattr(self, "ctx", None) is not None:
            sci_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        sci_set_stream(self.ctx, stream.cuda_stream)

    def set_integrals(self, mode: str, h, eri=None, chol=None):
        """h, and eri or chol, as numpy arrays (host) or CUDA tensors of this device, which
        are read in place (sci_set_integrals_ex with on_device = 1)."""
        torch = self.torch
        n = h.shape[0]
        if isinstance(h, torch.Tensor) and h.is_cuda:
            self.complex = bool(h.is_complex())
            dt = torch.complex128 if self.complex else torch.float64
            hh = h.detach().to(dt).contiguous()
            e = None if eri is None else eri.detach().to(dt).contiguous()
            L = None if chol is None else chol.detach().to(dt).contiguous()
            for t in (e, L):
                if t is not None and not (t.is_cuda and t.device == hh.device):
                    raise ValueError("h, eri and chol must be on the same CUDA device")
            # the copies above ran on torch's current stream; the library reads on its own
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            sci_set_integrals_ex(self.ctx, SCI_COMPLEX128 if self.complex else SCI_REAL64,
                                 SCI_SPINORS if mode == "spinors" else SCI_SPIN_ORBITALS, n, hh, e,
                                 0 if L is None else L.shape[0], L, 1)
        else:
            self.complex = bool(np.iscomplexobj(h))
            dt = np.complex128 if self.complex else np.float64
            hh = np.ascontiguousarray(h, dtype=dt)
            e = None if eri is None else np.ascontiguousarray(eri, dtype=dt)
            L = None if chol is None else np.ascontiguousarray(chol, dtype=dt)
            sci_set_integrals(self.ctx, SCI_COMPLEX128 if self.complex else SCI_REAL64,
                              SCI_SPINORS if mode == "spinors" else SCI_SPIN_ORBITALS, n, hh, e,
                              0 if L is None else L.shape[0], L)
        self.mode = mode
        self.n = n

    def set_determinants(self, keys, n_alpha: int, n_beta: int):
        torch = self.torch
        if isinstance(keys, torch.Tensor):
            k = keys.contiguous()
            on_dev = int(k.is_cuda)
            M = k.shape[0] if k.dim() else 0
        else:
            k = np.ascontiguousarray(keys, dtype=np.uint64)
            on_dev = 0
            M = len(k)
        nwords = 1 if k.ndim == 1 else k.shape[1]      # [M] strings or [M, 2] words
        sci_set_determinants_w(self.ctx, k, nwords, M, n_alpha, n_beta if self.mode != "spinors" else -1, on_dev)
        self.M = M
        self.n_alpha, self.n_beta = int(n_alpha), int(n_beta)
        self.row_range = (0, M)

    @property
    def n_electrons(self) -> int:
        return self.n_alpha + (self.n_beta if self.mode != "spinors" else 0)

    @classmethod
    def from_workload(cls, w, device: int = 0, use_chol: bool = True):
        H = cls(device)
        if use_chol:
            H.set_integrals(w.mode, w.ints.h, chol=w.ints.chol)
        else:
            H.set_integrals(w.mode, w.ints.h, eri=w.ints.eri())
        H.set_determinants(w.keys, w.n_alpha, w.n_beta)
        return H

    def set_row_range(self, row_begin: int, row_end: int):
        """Later sigma calls compute rows [row_begin, row_end) of S only (the other rows
        of S are left as they were); (0, M) returns to the whole list."""
        sci_set_row_range(self.ctx, row_begin, row_end)
        self.row_range = (int(row_begin), int(row_end))

    def set_tile_threshold(self, members: int):
        """(N-2) buckets of more than `members` members go through the tiled sigma kernel
        (0 = the default: 512, or 384 for launches of 8 real vectors)."""
        sci_set_tile_threshold(self.ctx, members)

    def set_deterministic(self, max_nvec: int):
        """Later sigma calls with up to max_nvec vectors accumulate row sums in a fixed
        order (bitwise reproducible S); 0 returns to FP64 atomics."""
        sci_set_deterministic(self.ctx, max_nvec)

    def row_costs(self):
        """Per-row count of connected determinants (torch int64 on the device)."""
        c = self.torch.empty(self.M, dtype=self.torch.int64, device=self.device)
        sci_row_costs(self.ctx, c)
        return c

    def diagonal(self):
        d = self.torch.empty(self.M, dtype=self.torch.float64, device=self.device)
        sci_diagonal(self.ctx, d)
        return d

    def sigma(self, C, out=None, prec: int = SCI_PREC_F64):
        """S = H C for C of shape [M] or [M, nvec] (torch CUDA, contiguous)."""
        torch = self.torch
        squeeze = C.dim() == 1
        C2 = (C.reshape(-1, 1) if squeeze else C).contiguous()
        nvec = C2.shape[1]
        if self.M and C2.shape[0] != self.M:
            raise ValueError(f"C has {C2.shape[0]} rows, the determinant list {self.M}")
        odt = torch.complex128 if self.complex else torch.float64
        S = out if out is not None else torch.empty((C2.shape[0], nvec), dtype=odt, device=self.device)
        sci_sigma(self.ctx, C2, S, nvec, prec)
        return S.reshape(-1) if squeeze and out is None else S

    @property
    def norb(self) -> int:
        """Bits of a key: 2n spin-orbitals or n spinors."""
        return self.n if self.mode == "spinors" else 2 * self.n

    def rdm12(self, C, weights=None, rdm2: bool = True):
        """(g1 [norb, norb], g2 [norb]^4 or None): sum_k w_k of the unnormalised density
        matrices of the columns of C ([M] or [M, nvec], torch CUDA) -- see sci_rdm12."""
        torch = self.torch
        C2 = (C.reshape(-1, 1) if C.dim() == 1 else C).contiguous()
        if self.M and C2.shape[0] != self.M:
            raise ValueError(f"C has {C2.shape[0]} rows, the determinant list {self.M}")
        dt = torch.complex128 if self.complex else torch.float64
        if C2.dtype != dt:
            raise ValueError(f"C must be {dt} for this Hamiltonian")
        no = self.norb
        g1 = torch.empty((no, no), dtype=dt, device=self.device)
        g2 = torch.empty((no, no, no, no), dtype=dt, device=self.device) if rdm2 else None
        sci_rdm12(self.ctx, C2, C2.shape[1], weights, g1, g2)
        return g1, g2

    def rdm_grads(self, C, weights=None, chol=None, Gamma: bool = False):
        """(gamma [n, n], Gamma [n]^4 or None, gchol [naux, n, n] or None): the spin-summed
        1-RDM, optionally the spin-summed 2-RDM, and sum_rs Gamma_pqrs chol[P, r, s] for
        Cholesky factors `chol` (float64 CUDA) -- see sci_rdm_grads."""
        torch = self.torch
        C2 = (C.reshape(-1, 1) if C.dim() == 1 else C).contiguous()
        if C2.dtype != torch.float64 or self.complex:
            raise ValueError("rdm_grads: real spin-orbital Hamiltonians, float64 C")
        n = self.n
        gam = torch.empty((n, n), dtype=torch.float64, device=self.device)
        G = torch.empty((n, n, n, n), dtype=torch.float64, device=self.device) if Gamma else None
        gL = None
        if chol is not None:
            chol = chol.contiguous()
            gL = torch.empty_like(chol)
        sci_rdm_grads(self.ctx, C2, C2.shape[1], weights, gam, G, 0 if chol is None else chol.shape[0], chol, gL)
        return gam, G, gL

    def enpt2(self, C, E0, eps: float = 0.0, table_bytes: int = 1 << 30):
        """Epstein-Nesbet second-order energies of the columns of C ([M, nroots] CUDA,
        float64 for a real spin-orbital Hamiltonian, complex128 for a complex spinor one)
        with zeroth-order energies E0: (E2[W], E2[P], E2[Q], stats) -- see sci_enpt2."""
        C2 = (C.reshape(-1, 1) if C.dim() == 1 else C).contiguous()
        want = self.torch.complex128 if self.complex else self.torch.float64
        if C2.dtype != want or not C2.is_cuda or (self.M and C2.shape[0] != self.M):
            raise ValueError(f"C must be a [M, nroots] {want} CUDA tensor for this Hamiltonian")
        return sci_enpt2(self.ctx, C2, C2.shape[1], E0, eps, table_bytes)

    def connections(self, row_begin: int = 0, row_end: int | None = None):
        row_end = self.M if row_end is None else row_end
        n, _ = sci_connections(self.ctx, row_begin, row_end, 0)
        n2, arrs = sci_connections(self.ctx, row_begin, row_end, n)
        return arrs

    def count_pairs(self) -> int:
        return sci_count_pairs(self.ctx)

    def sigma_host(self, C: np.ndarray, out: np.ndarray | None = None, prec: int = SCI_PREC_F64):
        """S = H C with host (numpy or pinned torch CPU) buffers; synchronous."""
        nvec = 1 if C.ndim == 1 else C.shape[1]
        if out is None:
            out = np.empty((self.M, nvec), dtype=np.complex128 if self.complex else np.float64)
        sci_sigma_host(self.ctx, C, out, nvec, prec)
        return out

    def info(self) -> dict:
        return sci_info(self.ctx)

    def sync_status(self):
        return sci_sync_status(self.ctx)


class Batch:
    """Heterogeneous instances (sci.Hamiltonian, real spin-orbital mode) applied to their
    vectors in one persistent launch.  Vectors are concatenated: instance i occupies
    rows offsets[i] : offsets[i] + M_i of one [sum M] float64 CUDA tensor."""

    def __init__(self, hams, device: int = 0, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.b = sci_batch_create(device, s.cuda_stream)
        self.hams = list(hams)          # the batch points into their tables: keep them alive
        self.offsets = []
        off = 0
        for H in self.hams:
            sci_batch_add(self.b, H.ctx)
            self.offsets.append(off)
            off += H.M
        self.M = off

    def close(self):
        if getattr(self, "b", None) is not None:
            sci_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, schedule: int = SCI_SCHED_AUTO, C=None, S=None):
        if schedule == SCI_SCHED_AUTO and C is None:
            C = self.torch.ones(self.M, dtype=self.torch.float64, device=self.device)
        if schedule == SCI_SCHED_AUTO and S is None:
            S = self.torch.empty(self.M, dtype=self.torch.float64, device=self.device)
        sci_batch_plan(self.b, schedule, C, S)

    def sigma(self, C, out=None):
        S = out if out is not None else self.torch.empty_like(C)
        sci_batch_sigma(self.b, C.contiguous(), S)
        return S

    def capture(self, C, S):
        sci_batch_capture(self.b, C, S)

    def replay(self):
        sci_batch_replay(self.b)

    def set_active(self, active):
        """Per-instance flags (nonzero = computed) for later launches and replays."""
        sci_batch_set_active(self.b, active)

    def info(self, i: int) -> dict:
        return sci_batch_info(self.b, i)

    def items(self) -> dict:
        return sci_batch_items(self.b)


class Segments:
    """Segmented block-vector products over vectors stored end to end (instance s on rows
    offsets[s] : offsets[s+1] of one float64 CUDA array); blocks are column-major
    [k, total rows] tensors whose rows are the columns of the block."""

    def __init__(self, offsets, kmax: int, device: int = 0, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.nseg, self.M, self.kmax = len(self.offsets) - 1, int(self.offsets[-1]), int(kmax)
        self.sg = sci_seg_create(device, self.offsets, kmax, s.cuda_stream)

    def close(self):
        if getattr(self, "sg", None) is not None:
            sci_seg_destroy(self.sg)
            self.sg = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _ld(A):
        return int(A.stride(0)) if A.dim() == 2 else 0

    def tn(self, A, t, out=None):
        """[nseg, k]: per instance, the dot products of the k rows of A [k, M] with t [M]."""
        A2 = A if A.dim() == 2 else A.view(1, -1)
        k = A2.shape[0]
        assert A2.stride(1) == 1 and t.stride(0) == 1 and A2.shape[1] == self.M and t.shape[0] == self.M
        if out is None:
            out = self.torch.empty((self.nseg, k), dtype=self.torch.float64, device=self.device)
        sci_seg_tn(self.sg, k, A2, self._ld(A2), t, out)
        return out

    def nn(self, y, beta=None, A1=None, c1=None, alpha1=1.0, A2=None, c2=None, alpha2=1.0, dg=None, shift=None):
        """y = beta_s y + alpha1 A1^T c1_s + alpha2 A2^T c2_s per instance, then / (shift_s - dg)
        if dg is given (A: [k, M] row blocks, c: [nseg, k], beta and shift: [nseg])."""
        def op(A, c):
            if A is None or A.shape[0] == 0:
                return 0, None, 0, None
            assert A.stride(1) == 1 and A.shape[1] == self.M and c.shape == (self.nseg, A.shape[0]) and c.is_contiguous()
            return A.shape[0], A, int(A.stride(0)), c
        k1, A1, l1, c1 = op(A1, c1)
        k2, A2, l2, c2 = op(A2, c2)
        assert y.stride(0) == 1 and y.shape[0] == self.M
        sci_seg_nn(self.sg, y, beta, k1, A1, l1, c1, alpha1, k2, A2, l2, c2, alpha2, dg, shift)
        return y
