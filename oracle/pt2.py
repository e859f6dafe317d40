"""Epstein-Nesbet second-order energy by its definition (Sec. 2.4, Eq. ENPT2E).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

    E2_k = sum_{I in Q} (sum_{J in P} H_IJ c_Jk)^2 / (E0_k - H_II),

Q = every determinant with the electron counts of P that is not in P.  The full space is
enumerated, so this is for tiny spaces only.  H_IJ are the oracle's row elements
(operator application, sciref.c) and H_II its diagonal.  Unlike the GPU route, no
W - P rewriting (Eq. PT2final) is used, and no excitation generation either.

Parity: pinned by tests/test_oracle_pt2_pins.py against the dense matrix of the literal
operator route (fock_route.hamiltonian), and by E2 = 0 when P is the full space.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import Oracle


def full_space_keys(mode: str, n: int, na: int, nb: int) -> np.ndarray:
    """Every determinant of the space, ascending: spin-orbital mode (bit p alpha p, bit
    n+p beta p) with na alpha and nb beta electrons, or spinor mode with na electrons."""
    def strings(m, k):
        return [sum(1 << p for p in c) for c in itertools.combinations(range(m), k)]

    if mode == "spinors":
        keys = strings(n, na)
    else:
        keys = [a | (b << n) for a in strings(n, na) for b in strings(n, nb)]
    return np.array(sorted(keys), dtype=np.uint64)


def enpt2(mode: str, n: int, na: int, nb: int, h, eri, P_keys, C, E0) -> np.ndarray:
    """E2_k of Eq. ENPT2E for the columns of C (coefficients on the sorted P_keys) with
    zeroth-order energies E0 (one per column)."""
    full = full_space_keys(mode, n, na, nb)
    P_keys = np.asarray(P_keys, dtype=np.uint64)
    C = np.asarray(C).reshape(len(P_keys), -1)
    E0 = np.asarray(E0, dtype=np.float64).reshape(-1)
    o = Oracle(mode, n, h, eri, full)
    d = o.diagonal().real
    pos = np.searchsorted(full, P_keys)
    assert np.array_equal(full[pos], P_keys), "P must be a subset of the space"
    in_p = np.zeros(len(full), dtype=bool)
    in_p[pos] = True
    Cf = np.zeros((len(full), C.shape[1]), dtype=C.dtype)
    Cf[pos] = C
    E2 = np.zeros(C.shape[1])
    for I in np.nonzero(~in_p)[0]:
        J, hv = o.row_elements(int(I))
        v = hv @ Cf[J]
        E2 += np.abs(v) ** 2 / (E0 - d[I])
    return E2
