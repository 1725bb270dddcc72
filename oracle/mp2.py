"""First-order (MP2) doubles and the MP2 correlation energy.

Test infrastructure (see ``oracle/__init__``).

With the Fock operator diagonal, f = diag(eps) (the semicanonical basis the
paper's natural-spinor step ends in, Eqs. 26-27), the first-order doubles are

    t_ij^ab = <ab||ij> / D_ij^ab,   D_ij^ab = eps_i + eps_j - eps_a - eps_b,

the same denominators that appear in Eq. 24, and

    E_MP2 = 1/4 sum_ijab <ij||ab> t_ij^ab.
"""
from __future__ import annotations

import numpy as np


def denom2(eps, n_occ):
    """D_ij^ab = eps_i + eps_j - eps_a - eps_b as an [o, o, v, v] array."""
    eo = eps[:n_occ]
    ev = eps[n_occ:]
    return (eo[:, None, None, None] + eo[None, :, None, None]
            - ev[None, None, :, None] - ev[None, None, None, :])


def denom1(eps, n_occ):
    """D_i^a = eps_i - eps_a as an [o, v] array."""
    return eps[:n_occ, None] - eps[None, n_occ:]


def amplitudes(blocks, eps):
    """t_ij^ab = <ab||ij> / D_ij^ab, stored [i, j, a, b]."""
    vvoo = blocks.vvoo  # [a, b, i, j] = <ab||ij>
    return vvoo.transpose(2, 3, 0, 1) / denom2(eps, blocks.n_occ)


def energy(blocks, t2):
    """E_MP2 = 1/4 sum <ij||ab> t_ij^ab."""
    return 0.25 * np.einsum("ijab,ijab->", blocks.oovv, t2)
