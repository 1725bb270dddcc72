"""IP-EOM-CCSD (Eqs. 16-20): H-bar intermediates, sigma, dense eigenproblem,
left vectors.

Test infrastructure (see ``oracle/__init__``).

The ionisation operator is Eq. 17 truncated at 2h1p:
R = sum_i r_i a_i + sum_{i<j,b} r_ij^b a+_b a_j a_i, with r_ji^b = -r_ij^b.
Eq. 18, [H-bar, R]|0> = omega R|0>, projected on {|i>, |ij^b>}, gives the
non-Hermitian eigenproblem sigma(r) = omega r. omega = E(N-1) - E(N) is the
ionisation potential (positive for bound electrons).

H-bar elements are those with at most two virtual indices, built once from
converged amplitudes (as the paper's implementation section describes), in
the spin-orbital form of Stanton and Gauss (J. Chem. Phys. 101, 8938 (1994))
with creation indices first in every <pq||rs>. The three-body part of H-bar
enters through <mn||ef> and t2 directly. The brute-force module
``oracle.fci`` pins every element.

Vector layout: [r_i for i in range(o)] + [r_ij^b for (i<j) in
numpy.triu_indices order, b fastest]. Left vectors (Eq. 20) use the same
layout for l^i and l^ij_b; Eq. 19 pairs them with right vectors bilinearly
over these unique elements.
"""
from __future__ import annotations

import numpy as np

from .ccsd import tau


def hbar(g, eps, t1, t2):
    """H-bar one- and two-body elements with at most two virtual indices."""
    o = g.n_occ
    eo = eps[:o]
    ev = eps[o:]
    ta = tau(t1, t2)
    Hov = np.einsum("nf,mnef->me", t1, g.oovv)
    Hoo = (np.diag(eo).astype(complex)
           + np.einsum("ne,mnie->mi", t1, g.ooov)
           + 0.5 * np.einsum("inef,mnef->mi", ta, g.oovv))
    Hvv = (np.diag(ev).astype(complex)
           + np.einsum("mf,amef->ae", t1, g.vovv)
           - 0.5 * np.einsum("mnaf,mnef->ae", ta, g.oovv))
    x = np.einsum("je,mnie->mnij", t1, g.ooov)
    Hoooo = (g.oooo + x - x.transpose(0, 1, 3, 2)
             + 0.5 * np.einsum("ijef,mnef->mnij", ta, g.oovv))
    Hooov = g.ooov + np.einsum("if,mnfe->mnie", t1, g.oovv)
    z = t2 + np.einsum("jf,nb->jnfb", t1, t1)
    Hovvo = (g.ovvo + np.einsum("jf,mbef->mbej", t1, g.ovvv)
             - np.einsum("nb,mnej->mbej", t1, g.oovo)
             - np.einsum("jnfb,mnef->mbej", z, g.oovv))
    # W_mbij (ovoo)
    y = (np.einsum("mnie,jnbe->mbij", g.ooov, t2)
         + np.einsum("ie,mbej->mbij", t1,
                     g.ovvo - np.einsum("njbf,mnef->mbej", t2, g.oovv)))
    Hovoo = (g.ovoo
             - np.einsum("me,ijbe->mbij", Hov, t2)
             - np.einsum("nb,mnij->mbij", t1, Hoooo)
             + 0.5 * np.einsum("mbef,ijef->mbij", g.ovvv, ta)
             + y - y.transpose(0, 1, 3, 2))
    return {"ov": Hov, "oo": Hoo, "vv": Hvv, "oooo": Hoooo, "ooov": Hooov,
            "ovvo": Hovvo, "ovoo": Hovoo, "oovv": g.oovv, "t2": t2}


def dim(o, v):
    return o + o * (o - 1) // 2 * v


def unpack_r(vec, o, v):
    r1 = vec[:o]
    io, jo = np.triu_indices(o, 1)
    r2 = np.zeros((o, o, v), dtype=np.complex128)
    u = vec[o:].reshape(len(io), v)
    r2[io, jo] = u
    r2[jo, io] = -u
    return r1, r2


def pack_r(r1, r2):
    o = r1.shape[0]
    io, jo = np.triu_indices(o, 1)
    return np.concatenate([r1, r2[io, jo].ravel()])


def sigma(H, vec, o, v):
    """(H-bar R)_connected projected on 1h and 2h1p (Eq. 18 left side)."""
    r1, r2 = unpack_r(vec, o, v)
    s1 = (-np.einsum("mi,m->i", H["oo"], r1)
          + np.einsum("me,ime->i", H["ov"], r2)
          - 0.5 * np.einsum("mnie,mne->i", H["ooov"], r2))
    s2 = (-np.einsum("mbij,m->ijb", H["ovoo"], r1)
          + np.einsum("be,ije->ijb", H["vv"], r2))
    x = np.einsum("mi,mjb->ijb", H["oo"], r2)
    s2 -= x - x.transpose(1, 0, 2)
    s2 += 0.5 * np.einsum("mnij,mnb->ijb", H["oooo"], r2)
    y = np.einsum("mbej,ime->ijb", H["ovvo"], r2)
    s2 += y - y.transpose(1, 0, 2)
    xe = 0.5 * np.einsum("mnef,mnf->e", H["oovv"], r2)
    s2 -= np.einsum("e,ijeb->ijb", xe, H["t2"])
    return pack_r(s1, s2)


def left_sigma(H, lvec, o, v):
    """l^T H-bar_IP for a left vector in the same packed layout.

    Eqs. 19-20 pair a left vector with a right one bilinearly over the unique
    elements, <L|R> = sum_i l^i r_i + sum_{i<j,b} l^ij_b r_ij^b, so the left
    eigenproblem is l^T M = omega l^T for the matrix M of ``sigma``. Each
    term of ``sigma`` is read here with input and output exchanged: with
    l_ij^b antisymmetric, a term s_ijb <- f(r) contributes
    (1/2) sum l_ijb f(r) to <L|sigma(R)>, written as sum G_pqb r_pqb, and the
    packed derivative with respect to r_{p<q}^b is G_pqb - G_qpb.
    """
    l1, l2 = unpack_r(lvec, o, v)
    s1 = (-np.einsum("mi,i->m", H["oo"], l1)
          - 0.5 * np.einsum("mbij,ijb->m", H["ovoo"], l2))
    # G[p, q, b], from the terms of sigma in the order written there
    g = np.einsum("i,me->ime", l1, H["ov"])
    g -= 0.5 * np.einsum("i,mnie->mne", l1, H["ooov"])
    g += 0.5 * np.einsum("ijb,be->ije", l2, H["vv"])
    g -= np.einsum("ijb,mi->mjb", l2, H["oo"])
    g += 0.25 * np.einsum("ijb,mnij->mnb", l2, H["oooo"])
    g += np.einsum("ijb,mbej->ime", l2, H["ovvo"])
    ye = 0.5 * np.einsum("ijb,ijeb->e", l2, H["t2"])
    g -= 0.5 * np.einsum("e,mnef->mnf", ye, H["oovv"])
    return pack_r(s1, g - g.transpose(1, 0, 2))


def dense_left_right(H, o, v, n_roots):
    """The n_roots eigenvalues of smallest real part with right vectors R
    (unit 2-norm) and left vectors L scaled so that L^T R = 1 (Eq. 19).

    Left vectors are the right eigenvectors of M^T, M from ``dense_matrix``;
    they are matched to the right ones by the largest |l^T r| and the whole
    selected set is made biorthonormal by L <- L (L^T R)^-T, which also
    separates degenerate roots.
    """
    M = dense_matrix(H, o, v)
    w, R = np.linalg.eig(M)
    order = np.argsort(w.real, kind="stable")[:n_roots]
    w, R = w[order], R[:, order]
    wl, Lall = np.linalg.eig(M.T)
    L = np.empty_like(R)
    used = np.zeros(len(wl), bool)
    for k in range(n_roots):
        d = np.abs(wl - w[k])
        d[used] = np.inf
        # candidates at this eigenvalue; keep the one overlapping r_k most
        cand = np.flatnonzero(d <= 1e-8 * max(1.0, abs(w[k])) + d.min())
        j = cand[np.argmax(np.abs(Lall[:, cand].T @ R[:, k]))]
        used[j] = True
        L[:, k] = Lall[:, j]
    S = L.T @ R
    L = L @ np.linalg.inv(S).T
    return w, R, L


def pole_strength(lvec, rvec, o):
    """The 1h part of the biorthonormal pair's overlap, sum_i l^i r_i
    (equal to 1 for a Koopmans root at zero coupling, 0 for a 2h1p one;
    summed over all roots it is o)."""
    return complex(np.dot(lvec[:o], rvec[:o]))


def diagonal(H, o, v):
    """Diagonal of the sigma matrix from its one-body parts (preconditioner)."""
    hoo = np.diag(H["oo"])
    hvv = np.diag(H["vv"])
    io, jo = np.triu_indices(o, 1)
    d2 = (hvv[None, :] - hoo[io][:, None] - hoo[jo][:, None]).ravel()
    return np.concatenate([-hoo, d2])


def first_order_guess(H, o, v, i):
    """Starting vector of a Davidson root seeded at the 1h element i: r_i = 1
    and the 2h1p elements of first-order (Rayleigh-Schroedinger) perturbation
    theory about the diagonal, r_nu = M_nu,i / (M_ii - M_nu,nu), with
    M_nu,i the 2h1p <- 1h coupling (the sigma of the unit vector e_i) and the
    diagonal of ``diagonal``. The Davidson iterations converge to the same
    roots from any start; this one only shortens them."""
    d = diagonal(H, o, v)
    e = np.zeros(dim(o, v), dtype=np.complex128)
    e[i] = 1.0
    col = sigma(H, e, o, v)
    g = e.copy()
    g[o:] = col[o:] / (d[i] - d[o:])
    return g


def dense_matrix(H, o, v):
    """H-bar_IP by applying sigma to unit vectors (small sizes only)."""
    n = dim(o, v)
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[k] = 1.0
        M[:, k] = sigma(H, e, o, v)
        e[k] = 0.0
    return M


def dense_roots(H, o, v, n_roots):
    """The n_roots eigenvalues of smallest real part, with right vectors."""
    M = dense_matrix(H, o, v)
    w, V = np.linalg.eig(M)
    order = np.argsort(w.real, kind="stable")[:n_roots]
    return w[order], V[:, order]


def r1_weight(vec, o):
    """||r1||^2 / ||r||^2 for a right eigenvector."""
    return float(np.vdot(vec[:o], vec[:o]).real / np.vdot(vec, vec).real)
