"""CPU oracle for sigma = H c over a sorted determinant list.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline leg of the
benchmark may import this package.  It shares no code with the CUDA path: the C library
``sciref.c`` evaluates Slater-Condon elements by explicit operator application
(paper Sec. 2.1, Eq. Hamiltonian) and finds connections by generation + binary search;
``fock_route`` assembles H literally from the second-quantised operators.

Parity status: every function here is pinned by tests/test_oracle_pins.py (closed forms,
textbook limits, invariances, an independent NumPy route and brute force).  The paper's
own molecular energies need its Br and Cr2 integrals, which are not available, so
parity against real molecules is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sciref.c")
_LIB_PATH = os.path.join(_HERE, "libsciref.so")
_lock = threading.Lock()
_lib = None

SCIREF_OK = 0
SCIREF_ERR_CAP = -8


def build(force: bool = False) -> str:
    """Compile sciref.c into oracle/libsciref.so (plain gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.sciref_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, vp, vp]
            L.sciref_destroy.argtypes = [vp]
            L.sciref_destroy.restype = None
            L.sciref_set_determinants.argtypes = [vp, vp, i64]
            L.sciref_set_determinants_w.argtypes = [vp, vp, i32, i64]
            L.sciref_diagonal.argtypes = [vp, vp]
            L.sciref_hij.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, vp]
            L.sciref_connections.argtypes = [vp, i64, vp, vp, vp, vp, i64]
            L.sciref_row_elements.argtypes = [vp, i64, vp, vp, vp, i64]
            L.sciref_count_pairs.argtypes = [vp, i64, i64, vp]
            L.sciref_sigma_rows.argtypes = [vp, vp, i64, vp, i32, vp]
            L.sciref_sigma_brute_rows.argtypes = [vp, vp, i64, vp, i32, vp]
            L.sciref_sigma_abs_rows.argtypes = [vp, vp, i64, vp, i32, vp]
            L.sciref_rdm12.argtypes = [vp, vp, vp, vp]
            L.sciref_enpt2.argtypes = [vp, vp, i32, vp, ctypes.c_double, i32, vp, vp]
            L.sciref_set_threads.argtypes = [i32]
            L.sciref_set_threads.restype = i32
            _lib = L
    return _lib


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's parallel loops (n <= 0: the OpenMP default).
    Returns the number in force afterwards."""
    return int(_load().sciref_set_threads(int(n)))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Oracle:
    """One Hamiltonian (h, dense (pq|rs)) plus one sorted determinant list.

    mode: "spin_orbitals" (n spatial orbitals, real) or "spinors" (n spinors, complex).
    h: n x n; eri: n x n x n x n in Mulliken order [p,q,r,s] = (pq|rs).
    """

    def __init__(self, mode: str, n: int, h: np.ndarray, eri: np.ndarray, keys=None):
        self.L = _load()
        self.mode = mode
        self.is_complex = bool(np.iscomplexobj(h) or np.iscomplexobj(eri))
        self.dtype = np.complex128 if self.is_complex else np.float64
        hh = np.ascontiguousarray(h, dtype=self.dtype)
        ee = np.ascontiguousarray(eri, dtype=self.dtype)
        self._h, self._eri = hh, ee
        self.ctx = ctypes.c_void_p()
        rc = self.L.sciref_create(ctypes.byref(self.ctx), int(self.is_complex),
                                  int(mode == "spinors"), int(n), _ptr(hh), _ptr(ee))
        if rc != SCIREF_OK:
            raise ValueError(f"sciref_create failed ({rc})")
        self.M = 0
        if keys is not None:
            self.set_determinants(keys)

    @classmethod
    def from_workload(cls, w):
        return cls(w.mode, w.n, w.ints.h, w.ints.eri(), w.keys)

    def __del__(self):
        if getattr(self, "ctx", None):
            self.L.sciref_destroy(self.ctx)
            self.ctx = None

    def set_determinants(self, keys):
        """keys: [M] uint64 strings, or [M, 2] uint64 words (word 0 = orbitals 0..63) for
        more than 64 spin-orbitals (spinors)."""
        self.keys = np.ascontiguousarray(keys, dtype=np.uint64)
        nwords = 1 if self.keys.ndim == 1 else self.keys.shape[1]
        rc = self.L.sciref_set_determinants_w(self.ctx, _ptr(self.keys), nwords, len(self.keys))
        if rc != SCIREF_OK:
            raise ValueError(f"sciref_set_determinants failed ({rc})")
        self.M = len(self.keys)

    def diagonal(self) -> np.ndarray:
        out = np.zeros(self.M, dtype=self.dtype)
        self.L.sciref_diagonal(self.ctx, _ptr(out))
        return out

    def hij(self, bra: int, ket: int):
        out = np.zeros(1, dtype=self.dtype)
        self.L.sciref_hij(self.ctx, ctypes.c_uint64(int(bra)), ctypes.c_uint64(int(ket)), _ptr(out))
        return out[0]

    def connections(self, row: int):
        cnt = np.zeros(1, dtype=np.int64)
        cap = 1 << 12
        while True:
            J = np.zeros(cap, dtype=np.int64)
            deg = np.zeros(cap, dtype=np.int8)
            ph = np.zeros(cap, dtype=np.int8)
            rc = self.L.sciref_connections(self.ctx, int(row), _ptr(cnt), _ptr(J), _ptr(deg), _ptr(ph), cap)
            if rc == SCIREF_ERR_CAP:
                cap = int(cnt[0])
                continue
            if rc != SCIREF_OK:
                raise ValueError(rc)
            n = int(cnt[0])
            return J[:n], deg[:n], ph[:n]

    def row_elements(self, row: int):
        cnt = np.zeros(1, dtype=np.int64)
        cap = 1 << 12
        while True:
            J = np.zeros(cap, dtype=np.int64)
            hv = np.zeros(cap, dtype=self.dtype)
            rc = self.L.sciref_row_elements(self.ctx, int(row), _ptr(cnt), _ptr(J), _ptr(hv), cap)
            if rc == SCIREF_ERR_CAP:
                cap = int(cnt[0])
                continue
            if rc != SCIREF_OK:
                raise ValueError(rc)
            n = int(cnt[0])
            return J[:n], hv[:n]

    def count_pairs(self, row_begin: int = 0, row_end: int | None = None) -> int:
        row_end = self.M if row_end is None else row_end
        out = np.zeros(1, dtype=np.int64)
        rc = self.L.sciref_count_pairs(self.ctx, int(row_begin), int(row_end), _ptr(out))
        if rc != SCIREF_OK:
            raise ValueError(rc)
        return int(out[0])

    def _sigma(self, fn, rows, C):
        C = np.ascontiguousarray(C, dtype=self.dtype)
        if C.ndim == 1:
            C = C[:, None]
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        S = np.zeros((len(rows), C.shape[1]), dtype=self.dtype)
        rc = fn(self.ctx, _ptr(rows), len(rows), _ptr(C), C.shape[1], _ptr(S))
        if rc != SCIREF_OK:
            raise ValueError(rc)
        return S

    def sigma_rows(self, rows, C) -> np.ndarray:
        """sigma restricted to `rows` (generation + lookup route)."""
        return self._sigma(self.L.sciref_sigma_rows, rows, C)

    def sigma_brute_rows(self, rows, C) -> np.ndarray:
        """sigma restricted to `rows` (all-pairs route)."""
        return self._sigma(self.L.sciref_sigma_brute_rows, rows, C)

    def sigma(self, C) -> np.ndarray:
        return self.sigma_rows(np.arange(self.M), C)

    def sigma_abs_rows(self, rows, C) -> np.ndarray:
        """A[r, v] = |H_II| |C_Iv| + sum_J |H_IJ| |C_Jv| for I = rows[r] (real): the scale
        of the rounding errors of row I of sigma (sciref_sigma_abs_rows)."""
        C = np.ascontiguousarray(C, dtype=self.dtype)
        if C.ndim == 1:
            C = C[:, None]
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        A = np.zeros((len(rows), C.shape[1]), dtype=np.float64)
        rc = self.L.sciref_sigma_abs_rows(self.ctx, _ptr(rows), len(rows), _ptr(C), C.shape[1], _ptr(A))
        if rc != SCIREF_OK:
            raise ValueError(rc)
        return A

    def rdm12(self, c):
        """Unnormalised 1- and 2-RDM of vector c over spin-orbitals (spinors):
        g1[p,q] = <c|a+_p a_q|c>, g2[p,q,r,s] = <c|a+_p a+_r a_s a_q|c>."""
        c = np.ascontiguousarray(np.asarray(c).reshape(-1), dtype=self.dtype)
        norb = self._h.shape[0] * (1 if self.mode == "spinors" else 2)
        g1 = np.zeros((norb, norb), dtype=self.dtype)
        g2 = np.zeros((norb,) * 4, dtype=self.dtype)
        rc = self.L.sciref_rdm12(self.ctx, _ptr(c), _ptr(g1), _ptr(g2))
        if rc != SCIREF_OK:
            raise ValueError(rc)
        return g1, g2

    def enpt2(self, C, E0, eps: float = 0.0, over_w: bool = False):
        """Epstein-Nesbet E2_k (Eq. ENPT2E) of the columns of C on this list with
        zeroth-order energies E0, summed over the single and double excitations of the
        list that are outside it (sciref_enpt2); with eps > 0 a contribution H_IJ C_J with
        |H_IJ| max_k |C_Jk| < eps is left out; over_w sums over W (the list's excitations,
        members included: E2[W] of Eq. EW1) instead of Q.  Returns (E2 [nroots], number of
        distinct determinants summed)."""
        C = np.ascontiguousarray(np.asarray(C).reshape(self.M, -1), dtype=self.dtype)
        e0 = np.ascontiguousarray(np.asarray(E0, dtype=np.float64).reshape(-1))
        assert e0.size == C.shape[1]
        E2 = np.zeros(C.shape[1], dtype=np.float64)
        nx = np.zeros(1, dtype=np.int64)
        rc = self.L.sciref_enpt2(self.ctx, _ptr(C), C.shape[1], _ptr(e0), float(eps), int(over_w), _ptr(E2),
                                 _ptr(nx))
        if rc != SCIREF_OK:
            raise ValueError(rc)
        return E2, int(nx[0])

    def dense(self) -> np.ndarray:
        """Dense H on the list (small spaces only)."""
        H = np.zeros((self.M, self.M), dtype=self.dtype)
        H[np.arange(self.M), np.arange(self.M)] = self.diagonal()
        for r in range(self.M):
            J, hv = self.row_elements(r)
            H[r, J] = hv
        return H
