"""Plain non-Hermitian block Davidson for the lowest IP-EOM roots.

Test infrastructure (see ``oracle/__init__``).

The paper solves the EOM eigenproblem (Eq. 18) with Davidson's method in
the non-Hermitian form of Hirao and Nakatsuji (its EOM section). Steps per
iteration: orthonormal basis V; S = sigma(V); projected G = V^H S;
eigenpairs of G, the n_roots of smallest real part; Ritz vectors x = V y;
residuals r = S y - omega x; stop when every ||r|| < tol (unit x); else add
the preconditioned residuals r / (omega - diag) after orthogonalisation;
restart from the Ritz vectors when the basis exceeds ``max_space``.
"""
from __future__ import annotations

import numpy as np


def _orthonormalise(V, X, drop=1e-10):
    """Append the columns of X to V after two Gram-Schmidt passes."""
    cols = [V[:, k] for k in range(V.shape[1])] if V is not None else []
    for k in range(X.shape[1]):
        x = X[:, k].copy()
        for _ in range(2):
            for c in cols:
                x -= np.vdot(c, x) * c
        nrm = np.linalg.norm(x)
        if nrm > drop:
            cols.append(x / nrm)
    return np.stack(cols, axis=1)


def davidson(apply_sigma, diag, n_roots, tol=1e-7, max_iter=200,
             max_space=None, guesses=None):
    """Return (omega[n_roots], X[:, n_roots], n_iter, converged)."""
    n = diag.shape[0]
    if max_space is None:
        max_space = max(8 * n_roots, 40)
    if guesses is None:
        idx = np.argsort(diag.real, kind="stable")[:n_roots]
        guesses = np.zeros((n, n_roots), dtype=np.complex128)
        guesses[idx, np.arange(n_roots)] = 1.0
    V = _orthonormalise(None, guesses)
    S = np.stack([apply_sigma(V[:, k]) for k in range(V.shape[1])], axis=1)
    omega = None
    for it in range(1, max_iter + 1):
        G = V.conj().T @ S
        w, Y = np.linalg.eig(G)
        order = np.argsort(w.real, kind="stable")[:n_roots]
        w = w[order]
        Y = Y[:, order]
        X = V @ Y
        norms = np.linalg.norm(X, axis=0)
        X /= norms
        Y /= norms
        R = S @ Y - X * w[None, :]
        rn = np.linalg.norm(R, axis=0)
        omega = w
        if np.all(rn < tol):
            return omega, X, it, True
        if V.shape[1] + n_roots > max_space:
            V = _orthonormalise(None, X)
            S = np.stack([apply_sigma(V[:, k]) for k in range(V.shape[1])],
                         axis=1)
            continue
        corr = []
        for k in range(n_roots):
            if rn[k] >= tol:
                den = w[k] - diag
                den = np.where(np.abs(den) < 1e-8, 1e-8, den)
                corr.append(R[:, k] / den)
        m0 = V.shape[1]
        V = _orthonormalise(V, np.stack(corr, axis=1))
        new = [apply_sigma(V[:, k]) for k in range(m0, V.shape[1])]
        if not new:
            return omega, X, it, False
        S = np.concatenate([S, np.stack(new, axis=1)], axis=1)
    return omega, X, max_iter, False
