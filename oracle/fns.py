"""Frozen natural spinors (Eqs. 24-28), step by step.

Test infrastructure (see ``oracle/__init__``).

Steps, in the paper's order:

1. Eq. 24: the virtual-virtual block of the MP2 one-body density,
   D_ab = 1/2 sum_{c,i,j} <ac||ij> <ij||bc> / (eps_ij^ac eps_ij^bc),
   with eps_ij^ac = eps_i + eps_j - eps_a - eps_c and the sums unrestricted.
2. Eq. 25: D V = V n; natural virtual spinors V, occupations n.
3. Truncation: keep the natural spinors with n_k >= threshold (sorted by
   decreasing occupation); their columns form V~.
4. Eq. 26: F^NS = V~^H F_vv V~ with F_vv = diag(eps_virt).
5. Eq. 27: F^NS Z~ = Z~ eps~ (eps~ ascending).
6. Eq. 28: the virtual-space transformation. The printed product "Z~ V~" is
   dimensionally invalid for a truncated V~ (v x v~) and Z~ (v~ x v~); the
   reading used here is U = V~ Z~ (v x v~), which maps canonical virtual
   spinors onto semicanonical natural ones.

The occupied spinors stay canonical ("frozen"); only virtual indices of the
Cholesky vectors rotate, in the form of Eq. 22:
L^P_{i a~} = sum_a L^P_{ia} U_{a a~}, L^P_{a~ i} = sum_a U*_{a a~} L^P_{ai},
L^P_{a~ b~} = (U^H L^P_vv U)_{a~ b~}; L^P_ij is unchanged.
"""
from __future__ import annotations

import numpy as np


def vv_density(L, eps, n_occ):
    """Eq. 24, summed one occupied index i at a time to bound memory."""
    L = np.asarray(L, dtype=np.complex128)
    n = L.shape[1]
    o = slice(0, n_occ)
    v = slice(n_occ, n)
    ev = eps[n_occ:]
    eo = eps[:n_occ]
    nv = n - n_occ
    D = np.zeros((nv, nv), dtype=np.complex128)
    Lvo = L[:, v, o]
    Lov = L[:, o, v]
    for i in range(n_occ):
        # <ac||ij> = sum_P (L_ai L_cj - L_aj L_ci), indices [a, c, j]
        ket = (np.einsum("Pa,Pcj->acj", Lvo[:, :, i], Lvo, optimize=True)
               - np.einsum("Paj,Pc->acj", Lvo, Lvo[:, :, i], optimize=True))
        # <ij||bc> = sum_P (L_ib L_jc - L_ic L_jb), indices [j, b, c]
        bra = (np.einsum("Pb,Pjc->jbc", Lov[:, i, :], Lov, optimize=True)
               - np.einsum("Pc,Pjb->jbc", Lov[:, i, :], Lov, optimize=True))
        # eps_ij^ac, indices [a, c, j]
        den = eo[i] + eo[None, None, :] - ev[:, None, None] - ev[None, :, None]
        num_l = ket / den                       # [a, c, j]
        num_r = bra / den.transpose(2, 0, 1)    # [j, b, c] / eps_ij^bc
        D += 0.5 * np.einsum("acj,jbc->ab", num_l, num_r, optimize=True)
    return D


def natural_spinors(D):
    """Eq. 25: eigenpairs of the Hermitian D, occupations sorted descending."""
    n, V = np.linalg.eigh(0.5 * (D + D.conj().T))
    order = np.argsort(-n, kind="stable")
    return n[order], V[:, order]


def semicanonical(V_kept, eps_virt):
    """Eqs. 26-27: F^NS = V~^H diag(eps_v) V~, diagonalised; returns eps~, Z~."""
    F_ns = V_kept.conj().T @ (eps_virt[:, None] * V_kept)
    F_ns = 0.5 * (F_ns + F_ns.conj().T)
    eps_t, Z = np.linalg.eigh(F_ns)
    return eps_t, Z, F_ns


def rotate_cholesky(L, U, n_occ):
    """Apply the virtual transformation U (v x v~) to L in the form of Eq. 22."""
    L = np.asarray(L, dtype=np.complex128)
    n_aux, n, _ = L.shape
    nvt = U.shape[1]
    m = n_occ + nvt
    out = np.empty((n_aux, m, m), dtype=np.complex128)
    o = slice(0, n_occ)
    v = slice(n_occ, n)
    out[:, :n_occ, :n_occ] = L[:, o, o]
    out[:, :n_occ, n_occ:] = L[:, o, v] @ U
    out[:, n_occ:, :n_occ] = U.conj().T @ L[:, v, o]
    out[:, n_occ:, n_occ:] = U.conj().T @ L[:, v, v] @ U
    return out


def frozen_natural_spinors(L, eps, n_occ, threshold=None, n_keep=None):
    """Eqs. 24-28. Keep n_k >= threshold, or the n_keep largest occupations.

    Returns a dict with the new eps, rotated L, U, occupations, the number
    kept and the intermediate matrices.
    """
    if (threshold is None) == (n_keep is None):
        raise ValueError("give exactly one of threshold, n_keep")
    D = vv_density(L, eps, n_occ)
    occ, V = natural_spinors(D)
    if n_keep is None:
        n_keep = int(np.count_nonzero(occ >= threshold))
    V_kept = V[:, :n_keep]
    eps_t, Z, F_ns = semicanonical(V_kept, eps[n_occ:])
    U = V_kept @ Z
    L_new = rotate_cholesky(L, U, n_occ)
    eps_new = np.concatenate([eps[:n_occ], eps_t])
    return {
        "eps": eps_new, "L": L_new, "U": U, "occupations": occ,
        "n_keep": n_keep, "D": D, "F_ns": F_ns, "eps_virt": eps_t,
    }
