"""Spin-orbital CCSD (Eqs. 12-15) with Jacobi updates and DIIS.

Test infrastructure (see ``oracle/__init__``).

The paper states the CCSD conditions (Eqs. 13-14: singles and doubles
projections of H-bar = e^{-T} H e^{T} vanish) and the energy (Eq. 15) and
defers the working equations to the coupled-cluster literature it cites.
This module writes them in the spin-orbital intermediate form of Stanton,
Gauss, Watts and Bartlett (J. Chem. Phys. 94, 4334 (1991)), with every
integral in "creation indices first" order, <pq||rs> with p, q created and
r, s annihilated, which is the form that holds for complex spinors (for
example the doubles driver is <ab||ij>, not <ij||ab>). The Fock operator is
diagonal, f = diag(eps), so f_ia = 0 and every off-diagonal f term drops.
The brute-force module ``oracle.fci`` pins these equations.

Amplitudes: t1[i, a], t2[i, j, a, b] antisymmetric in (i, j) and in (a, b).

Convergence reading: ||dt||_2 over unique amplitudes (all t1, t2 with i<j,
a<b) below tol and |dE| below tol. DIIS: Pulay extrapolation over the last
``diis_size`` amplitude vectors from iteration ``diis_start`` on, error
vector = Jacobi step, complex Hermitian B matrix, solved in FP64.
"""
from __future__ import annotations

import numpy as np

from .mp2 import denom1, denom2


def tau_tilde(t1, t2):
    x = np.einsum("ia,jb->ijab", t1, t1)
    return t2 + 0.5 * (x - x.transpose(0, 1, 3, 2))


def tau(t1, t2):
    x = np.einsum("ia,jb->ijab", t1, t1)
    return t2 + x - x.transpose(0, 1, 3, 2)


def p_ij(x):
    """P(ij) X = X - X with i, j (axes 0, 1) exchanged."""
    return x - x.transpose(1, 0, 2, 3)


def p_ab(x):
    """P(ab) X = X - X with a, b (axes 2, 3) exchanged."""
    return x - x.transpose(0, 1, 3, 2)


def intermediates(g, t1, t2):
    """F_ae, F_mi, F_me, W_mnij, W_abef, W_mbej of the CCSD equations."""
    tt = tau_tilde(t1, t2)
    ta = tau(t1, t2)
    Fae = (np.einsum("mf,mafe->ae", t1, g.ovvv)
           - 0.5 * np.einsum("mnaf,mnef->ae", tt, g.oovv))
    Fmi = (np.einsum("ne,mnie->mi", t1, g.ooov)
           + 0.5 * np.einsum("inef,mnef->mi", tt, g.oovv))
    Fme = np.einsum("nf,mnef->me", t1, g.oovv)
    x = np.einsum("je,mnie->mnij", t1, g.ooov)
    Wmnij = (g.oooo + x - x.transpose(0, 1, 3, 2)
             + 0.25 * np.einsum("ijef,mnef->mnij", ta, g.oovv))
    y = np.einsum("mb,amef->abef", t1, g.vovv)
    Wabef = (g.vvvv - y + y.transpose(1, 0, 2, 3)
             + 0.25 * np.einsum("mnab,mnef->abef", ta, g.oovv))
    z = 0.5 * t2 + np.einsum("jf,nb->jnfb", t1, t1)
    Wmbej = (g.ovvo + np.einsum("jf,mbef->mbej", t1, g.ovvv)
             - np.einsum("nb,mnej->mbej", t1, g.oovo)
             - np.einsum("jnfb,mnef->mbej", z, g.oovv))
    return Fae, Fmi, Fme, Wmnij, Wabef, Wmbej


def ladder_term(g_vvvv, tau_amp):
    """Particle-particle ladder 1/2 sum_cd <ab||cd> tau_ij^cd, [i, j, a, b]."""
    return 0.5 * np.einsum("ijcd,abcd->ijab", tau_amp, g_vvvv, optimize=True)


def residuals(g, eps, t1, t2):
    """Right-hand sides of the singles and doubles equations.

    Returns (R1, R2) such that the Jacobi update is t1 = R1 / D1,
    t2 = R2 / D2 (the diagonal Fock part sits in the denominators).
    """
    Fae, Fmi, Fme, Wmnij, Wabef, Wmbej = intermediates(g, t1, t2)
    ta = tau(t1, t2)

    # singles (Eq. 13)
    R1 = (np.einsum("ie,ae->ia", t1, Fae)
          - np.einsum("ma,mi->ia", t1, Fmi)
          + np.einsum("imae,me->ia", t2, Fme)
          - np.einsum("nf,naif->ia", t1, g.ovov)
          - 0.5 * np.einsum("imef,maef->ia", t2, g.ovvv)
          - 0.5 * np.einsum("mnae,nmei->ia", t2, g.oovo))

    # doubles (Eq. 14)
    R2 = g.vvoo.transpose(2, 3, 0, 1).copy()
    Fbe = Fae - 0.5 * np.einsum("mb,me->be", t1, Fme)
    R2 += p_ab(np.einsum("ijae,be->ijab", t2, Fbe))
    Fmj = Fmi + 0.5 * np.einsum("je,me->mj", t1, Fme)
    R2 -= p_ij(np.einsum("imab,mj->ijab", t2, Fmj))
    R2 += 0.5 * np.einsum("mnab,mnij->ijab", ta, Wmnij)
    R2 += 0.5 * np.einsum("ijef,abef->ijab", ta, Wabef)
    ring = (np.einsum("imae,mbej->ijab", t2, Wmbej)
            - np.einsum("ie,ma,mbej->ijab", t1, t1, g.ovvo))
    R2 += p_ij(p_ab(ring))
    R2 += p_ij(np.einsum("ie,abej->ijab", t1, g.vvvo))
    R2 -= p_ab(np.einsum("ma,mbij->ijab", t1, g.ovoo))
    return R1, R2


def energy(g, t1, t2):
    """Eq. 15 with f_ia = 0: 1/4 <ij||ab> t_ij^ab + 1/2 <ij||ab> t_i^a t_j^b."""
    return (0.25 * np.einsum("ijab,ijab->", g.oovv, t2)
            + 0.5 * np.einsum("ijab,ia,jb->", g.oovv, t1, t1))


def pack(t1, t2):
    """Unique amplitudes: all of t1, then t2 with i<j and a<b."""
    o, v = t1.shape
    io, jo = np.triu_indices(o, 1)
    av, bv = np.triu_indices(v, 1)
    return np.concatenate([t1.ravel(), t2[io, jo][:, av, bv].ravel()])


def unpack(vec, o, v):
    t1 = vec[:o * v].reshape(o, v).copy()
    io, jo = np.triu_indices(o, 1)
    av, bv = np.triu_indices(v, 1)
    u = vec[o * v:].reshape(len(io), len(av))
    t2 = np.zeros((o, o, v, v), dtype=np.complex128)
    for k in range(len(io)):
        blk = np.zeros((v, v), dtype=np.complex128)
        blk[av, bv] = u[k]
        blk -= blk.T
        t2[io[k], jo[k]] = blk
        t2[jo[k], io[k]] = -blk
    return t1, t2


class Diis:
    """Pulay DIIS over complex vectors with a Hermitian B matrix."""

    def __init__(self, size=8):
        self.size = size
        self.vecs = []
        self.errs = []

    def push(self, vec, err):
        self.vecs.append(vec.copy())
        self.errs.append(err.copy())
        if len(self.vecs) > self.size:
            self.vecs.pop(0)
            self.errs.pop(0)

    def extrapolate(self):
        m = len(self.vecs)
        B = np.empty((m + 1, m + 1), dtype=np.complex128)
        for i in range(m):
            for j in range(m):
                B[i, j] = np.vdot(self.errs[i], self.errs[j])
        B[m, :m] = -1.0
        B[:m, m] = -1.0
        B[m, m] = 0.0
        rhs = np.zeros(m + 1, dtype=np.complex128)
        rhs[m] = -1.0
        c = np.linalg.solve(B, rhs)[:m]
        out = np.zeros_like(self.vecs[0])
        for ci, vi in zip(c, self.vecs):
            out += ci * vi
        return out


def solve(g, eps, tol=1e-8, max_iter=100, diis_size=8, diis_start=3,
          t1=None, t2=None, verbose=False):
    """Iterate the CCSD equations to convergence.

    Start: t1 = 0 and t2 = MP2 (or the given amplitudes).
    Returns dict(e_corr, t1, t2, n_iter, converged, history).
    """
    o = g.n_occ
    v = g.n_virt
    D1 = denom1(eps, o)
    D2 = denom2(eps, o)
    if t1 is None:
        t1 = np.zeros((o, v), dtype=np.complex128)
    if t2 is None:
        t2 = g.vvoo.transpose(2, 3, 0, 1) / D2
    e_old = energy(g, t1, t2)
    diis = Diis(diis_size)
    hist = []
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        R1, R2 = residuals(g, eps, t1, t2)
        t1n = R1 / D1
        t2n = R2 / D2
        old = pack(t1, t2)
        new = pack(t1n, t2n)
        step = new - old
        dnorm = float(np.linalg.norm(step))
        e_new = energy(g, t1n, t2n)
        de = abs(e_new - e_old)
        hist.append((it, e_new, dnorm))
        if verbose:
            print(f"ccsd it {it:3d} E={e_new.real:+.12f}{e_new.imag:+.2e}j "
                  f"|dt|={dnorm:.3e} |dE|={de:.3e}")
        if dnorm < tol and de < tol:
            t1, t2 = t1n, t2n
            e_old = e_new
            converged = True
            break
        if it >= diis_start:
            diis.push(new, step)
            if len(diis.vecs) >= 2:
                new = diis.extrapolate()
        t1, t2 = unpack(new, o, v)
        e_old = energy(g, t1, t2)
    return {"e_corr": energy(g, t1, t2), "t1": t1, "t2": t2, "n_iter": it,
            "converged": converged, "history": hist}
