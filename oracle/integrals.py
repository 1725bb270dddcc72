"""Antisymmetrised two-electron integrals from Cholesky vectors.

Test infrastructure (see ``oracle/__init__``). Conventions:

* Chemists' integrals (pq|rs) = sum_P L^P_pq L^P_rs  (Eq. 21 in the MO
  basis of Eq. 22).
* Physicists' integrals <pq|rs> = (pr|qs).
* <pq||rs> = <pq|rs> - <pq|sr> = sum_P (L^P_pr L^P_qs - L^P_ps L^P_qr),
  which is Eq. 23 term by term.

Spinor index p in [0, n), occupied spinors first.
"""
from __future__ import annotations

import numpy as np


def antisym_full(L):
    """Full <pq||rs> tensor [n, n, n, n] straight from Eq. 23."""
    L = np.asarray(L, dtype=np.complex128)
    direct = np.einsum("Ppr,Pqs->pqrs", L, L, optimize=True)
    exchange = np.einsum("Pps,Pqr->pqrs", L, L, optimize=True)
    return direct - exchange


def antisym_block(L, p, q, r, s):
    """<pq||rs> restricted to index ranges p, q, r, s (slices), Eq. 23."""
    L = np.asarray(L, dtype=np.complex128)
    direct = np.einsum("Ppr,Pqs->pqrs", L[:, p, r], L[:, q, s], optimize=True)
    exchange = np.einsum("Pps,Pqr->pqrs", L[:, p, s], L[:, q, r],
                         optimize=True)
    return direct - exchange


class Blocks:
    """Occupied/virtual blocks of <pq||rs> cut from the full tensor.

    Attribute names list the o/v class of p, q, r, s, e.g. ``oovv[i,j,a,b]``
    = <ij||ab>.
    """

    NAMES = ("oooo", "ooov", "oovo", "oovv", "ovoo", "ovov", "ovvo", "ovvv",
             "vooo", "vovv", "vvoo", "vvvo", "vvvv")

    def __init__(self, g, n_occ):
        o = slice(0, n_occ)
        v = slice(n_occ, g.shape[0])
        sl = {"o": o, "v": v}
        for name in self.NAMES:
            setattr(self, name, g[tuple(sl[c] for c in name)])
        self.n_occ = n_occ
        self.n_virt = g.shape[0] - n_occ


def blocks_from_cholesky(L, n_occ):
    return Blocks(antisym_full(L), n_occ)


def antisym_fixed_order(L, p, q, r, s):
    """Eq. 23 for index ranges p, q, r, s (slices), in one fixed order.

    The sum over P runs in ascending order; each complex product is formed
    as (ar*br - ai*bi, ar*bi + ai*br) with every multiply and add rounded
    separately (no fused multiply-add), the term is direct - exchange, and
    it is added to the running sum. Any evaluation that follows the same
    order gives the same bits.
    """
    L = np.asarray(L, dtype=np.complex128)
    Lpr = L[:, p, r]
    Lqs = L[:, q, s]
    Lps = L[:, p, s]
    Lqr = L[:, q, r]
    shape = (Lpr.shape[1], Lqs.shape[1], Lpr.shape[2], Lqs.shape[2])
    acc_r = np.zeros(shape)
    acc_i = np.zeros(shape)
    for P in range(L.shape[0]):
        a = Lpr[P][:, None, :, None]
        b = Lqs[P][None, :, None, :]
        c = Lps[P][:, None, None, :]
        d = Lqr[P][None, :, :, None]
        d1r = a.real * b.real - a.imag * b.imag
        d1i = a.real * b.imag + a.imag * b.real
        d2r = c.real * d.real - c.imag * d.imag
        d2i = c.real * d.imag + c.imag * d.real
        acc_r = acc_r + (d1r - d2r)
        acc_i = acc_i + (d1i - d2i)
    return acc_r + 1j * acc_i
