"""Closed forms of sigma on one- and two-electron spinor spaces, written from the
second-quantised Hamiltonian (Eq. 1) with no bit logic: for N = 1, sigma = h c; for N = 2
on the pairs p < q, with A the antisymmetric extension of c (A_rs = c_rs for r < s,
A_sr = -c_rs), sigma_pq = (h A + A h^T + sum_P L^P A L^P^T)_pq, where
(pr|qs) = sum_P L^P_pr L^P_qs.  Test infrastructure only."""
import numpy as np


def spinor_pair_sigma(h, chol, pairs, c):
    """sigma on the two-electron determinants pairs[i] = (p, q), p < q, for coefficients c
    ([M] or [M, k])."""
    c = np.asarray(c)
    cols = c.reshape(len(pairs), -1)
    n = h.shape[0]
    p, q = pairs[:, 0], pairs[:, 1]
    out = np.empty(cols.shape, dtype=np.result_type(h, chol, c))
    for k in range(cols.shape[1]):
        A = np.zeros((n, n), dtype=out.dtype)
        A[p, q] = cols[:, k]
        A[q, p] = -cols[:, k]
        S = h @ A + A @ h.T + np.einsum("Ppr,rs,Pqs->pq", chol, A, chol, optimize=True)
        out[:, k] = S[p, q]
    return out.reshape(c.shape)
