"""Single-step pivoted Cholesky decomposition (Eq. 21).

Test infrastructure (see ``oracle/__init__``).

The two-electron integral matrix over orbital pairs is Hermitian positive
semidefinite when its columns are indexed as M[(pq), (rs)] = (pq|sr); with
complex Cholesky vectors that is M = sum_P l_P l_P^H, l_P[(pq)] = L^P_pq.
The single-step algorithm forms one vector per step from the column of the
largest remaining diagonal element and stops when that element falls below
the threshold tau, which also bounds the error: the remainder
M - sum_P l_P l_P^H is positive semidefinite with every diagonal element
below tau, so every element is below tau in magnitude.

Here the matrix is given by a generator B (N x r), M = B B^H, whose columns
stand in for integrals computed on demand: column p of M is B conj(B[p]).
"""
from __future__ import annotations

import numpy as np


def column(B, p):
    """Column p of M = B B^H, from the generator."""
    return B @ np.conj(B[p])


def pivoted_cholesky(B, tau, max_vec=None):
    """Cholesky vectors of M = B B^H by the single-step algorithm.

    Step k: p = argmax of the remaining diagonal d; stop if d[p] < tau;
    l_k = (M[:, p] - sum_{j<k} l_j conj(l_j[p])) / sqrt(d[p]);
    d <- d - |l_k|^2. Returns (L [n_vec][N], pivots).
    """
    N = B.shape[0]
    if max_vec is None:
        max_vec = N
    d = np.einsum("ps,ps->p", B, np.conj(B)).real.copy()
    vecs, piv = [], []
    while len(vecs) < max_vec:
        p = int(np.argmax(d))
        if d[p] < tau:
            break
        col = column(B, p)
        for lj in vecs:
            col = col - lj * np.conj(lj[p])
        lk = col / np.sqrt(d[p])
        d = d - np.abs(lk) ** 2
        vecs.append(lk)
        piv.append(p)
    L = np.array(vecs, dtype=np.complex128).reshape(len(vecs), N)
    return L, np.array(piv, dtype=np.int64)
