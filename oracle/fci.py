"""Brute-force second quantisation on determinant bitstrings (tiny systems).

Test infrastructure (see ``oracle/__init__``). It shares nothing with the
working equations in ``ccsd`` and ``ipeom``: operators are built from their
definitions on occupation-number vectors, so it pins signs and factors.

Conventions. A determinant with occupied spinors p1 < p2 < ... < pk is
a+_{p1} a+_{p2} ... a+_{pk} |vac>. Then
a_p |det> = (-1)^{#occupied q < p} |det without p> if p is occupied, else 0;
a+_p is the transpose of a_p (real matrices).

Hamiltonian (Eq. 10 with the integrals of Eq. 23):
H = sum_pq h_pq a+_p a_q + 1/4 sum_pqrs <pq||rs> a+_p a+_q a_s a_r,
with bare h chosen so that the Fock operator of the reference (first n_occ
spinors occupied) is f = diag(eps):  h_pq = f_pq - sum_i <pi||qi>.

Cluster operators: T1 = sum t_i^a a+_a a_i, T2 = 1/4 sum t_ij^ab
a+_a a+_b a_j a_i. Excited determinants: |i^a> = a+_a a_i |0>,
|ij^ab> = a+_a a+_b a_j a_i |0>, and for ionisation |i> = a_i |0>,
|ij^b> = a+_b a_j a_i |0> (the operator string of Eq. 17).
"""
from __future__ import annotations

from itertools import combinations

import numpy as np
import scipy.linalg


class Sector:
    """All determinants of k electrons in n spinors, as integer bitmasks."""

    def __init__(self, n, k):
        self.n = n
        self.k = k
        self.dets = [sum(1 << p for p in occ)
                     for occ in combinations(range(n), k)] if k >= 0 else []
        self.index = {d: i for i, d in enumerate(self.dets)}

    def __len__(self):
        return len(self.dets)


def _sign_below(det, p):
    return -1.0 if bin(det & ((1 << p) - 1)).count("1") % 2 else 1.0


def annihilator(n, k, p):
    """Matrix of a_p from the k-electron sector to the (k-1)-electron one."""
    src = Sector(n, k)
    dst = Sector(n, k - 1)
    A = np.zeros((len(dst), len(src)))
    for col, det in enumerate(src.dets):
        if det >> p & 1:
            A[dst.index[det ^ (1 << p)], col] = _sign_below(det, p)
    return A


class Fock:
    """Annihilators a_p for every spinor between adjacent sectors."""

    def __init__(self, n):
        self.n = n
        self._cache = {}

    def a(self, p, k):
        """a_p : sector k -> sector k-1."""
        key = (p, k)
        if key not in self._cache:
            self._cache[key] = annihilator(self.n, k, p)
        return self._cache[key]

    def ad(self, p, k):
        """a+_p : sector k -> sector k+1."""
        return self.a(p, k + 1).T

    def pair_ann(self, k):
        """A[r, s] = a_s a_r : sector k -> k-2, as array [n, n, d(k-2), d(k)]."""
        n = self.n
        d2 = len(Sector(n, k - 2))
        dk = len(Sector(n, k))
        A = np.zeros((n, n, d2, dk))
        for r in range(n):
            ar = self.a(r, k)
            for s in range(n):
                A[r, s] = self.a(s, k - 1) @ ar
        return A

    def one_body(self, x, k):
        """sum_pq x_pq a+_p a_q in sector k."""
        n = self.n
        B = np.stack([self.a(q, k) for q in range(n)])  # [q, d(k-1), d(k)]
        return np.einsum("pq,pab,qac->bc", x, B, B, optimize=True)

    def two_body(self, w, k):
        """1/4 sum_pqrs w_pqrs a+_p a+_q a_s a_r in sector k.

        a+_p a+_q = (a_q a_p)^T, so the operator is
        1/4 sum A[p,q]^T w_pqrs A[r,s] with A[r,s] = a_s a_r.
        """
        if k < 2:
            d = len(Sector(self.n, k))
            return np.zeros((d, d), dtype=complex)
        A = self.pair_ann(k)
        M = np.einsum("pqrs,rsac->pqac", w, A, optimize=True)
        return 0.25 * np.einsum("pqab,pqac->bc", A, M, optimize=True)


def bare_one_body(eps, g, n_occ):
    """h_pq = f_pq - sum_i <pi||qi> with f = diag(eps)."""
    return np.diag(eps).astype(complex) - np.einsum(
        "piqi->pq", g[:, :n_occ, :, :n_occ])


def reference_energy(eps, g, n_occ):
    """E_ref = <0|H|0> = sum_i h_ii + 1/2 sum_ij <ij||ij>."""
    h = bare_one_body(eps, g, n_occ)
    o = slice(0, n_occ)
    return (np.trace(h[o, o])
            + 0.5 * np.einsum("ijij->", g[o, o, o, o]))


def hamiltonian(fock, eps, g, n_occ, k):
    h = bare_one_body(eps, g, n_occ)
    return fock.one_body(h, k) + fock.two_body(g, k)


def reference_vector(n, n_occ):
    sec = Sector(n, n_occ)
    v = np.zeros(len(sec), dtype=complex)
    v[sec.index[(1 << n_occ) - 1]] = 1.0
    return v


def cluster_operator(fock, t1, t2, n_occ, k):
    """T1 + T2 (Eq. 12 truncated to singles and doubles) in sector k."""
    o, v = t1.shape
    d = len(Sector(fock.n, k))
    T = np.zeros((d, d), dtype=complex)
    for i in range(o):
        for a in range(v):
            if t1[i, a] != 0:
                T += t1[i, a] * (fock.ad(o + a, k - 1) @ fock.a(i, k))
    if k >= 2:
        for i in range(o):
            for j in range(o):
                aji = fock.a(j, k - 1) @ fock.a(i, k)
                for a in range(v):
                    for b in range(v):
                        c = t2[i, j, a, b]
                        if c != 0:
                            T += 0.25 * c * (fock.ad(o + a, k - 1)
                                             @ fock.ad(o + b, k - 2) @ aji)
    return T


def similarity_transform(H, T):
    """H-bar = e^{-T} H e^{T} (dense; T is nilpotent on these sectors)."""
    E = scipy.linalg.expm(T)
    Ei = scipy.linalg.expm(-T)
    return Ei @ H @ E


def fci_energies(eps, L_or_g, n_occ, k, g_given=False):
    """All eigenvalues of H in the k-electron sector (ascending real part)."""
    from .integrals import antisym_full
    g = L_or_g if g_given else antisym_full(L_or_g)
    n = g.shape[0]
    H = hamiltonian(Fock(n), eps, g, n_occ, k)
    w = np.linalg.eigvals(H)
    return w[np.argsort(w.real)]


class BruteForce:
    """Everything needed to pin CCSD and IP-EOM-CCSD on one tiny system."""

    def __init__(self, eps, g, n_occ):
        self.eps = np.asarray(eps, dtype=float)
        self.g = g
        self.n = g.shape[0]
        self.o = n_occ
        self.v = self.n - n_occ
        self.fock = Fock(self.n)
        self.H_N = hamiltonian(self.fock, self.eps, g, n_occ, n_occ)
        self.H_Nm1 = hamiltonian(self.fock, self.eps, g, n_occ, n_occ - 1)
        self.ref = reference_vector(self.n, n_occ)
        self.e_ref = reference_energy(self.eps, g, n_occ)

    # excited determinants as vectors --------------------------------------
    def single(self, i, a):
        k = self.o
        return self.fock.ad(self.o + a, k - 1) @ (self.fock.a(i, k) @ self.ref)

    def double(self, i, j, a, b):
        k = self.o
        x = self.fock.a(j, k - 1) @ (self.fock.a(i, k) @ self.ref)
        return self.fock.ad(self.o + a, k - 1) @ (
            self.fock.ad(self.o + b, k - 2) @ x)

    def hole(self, i):
        return self.fock.a(i, self.o) @ self.ref

    def two_hole_particle(self, i, j, b):
        k = self.o
        x = self.fock.a(j, k - 1) @ (self.fock.a(i, k) @ self.ref)
        return self.fock.ad(self.o + b, k - 2) @ x

    # CC projections --------------------------------------------------------
    def hbar_N(self, t1, t2):
        T = cluster_operator(self.fock, t1, t2, self.o, self.o)
        return similarity_transform(self.H_N, T)

    def projections(self, t1, t2):
        """(E_total, <i^a|Hbar|0>, <ij^ab|Hbar|0>) for any amplitudes."""
        Hb = self.hbar_N(t1, t2)
        c = Hb @ self.ref
        e = np.vdot(self.ref, c)
        o, v = self.o, self.v
        P1 = np.array([[np.vdot(self.single(i, a), c) for a in range(v)]
                       for i in range(o)])
        P2 = np.zeros((o, o, v, v), dtype=complex)
        for i in range(o):
            for j in range(o):
                if i == j:
                    continue
                for a in range(v):
                    for b in range(v):
                        if a != b:
                            P2[i, j, a, b] = np.vdot(self.double(i, j, a, b), c)
        return e, P1, P2

    def ip_matrix(self, t1, t2):
        """<mu| Hbar - E_cc |nu> over {|i>, |ij^b> (i<j)} in the N-1 sector."""
        o, v = self.o, self.v
        T = cluster_operator(self.fock, t1, t2, self.o, self.o - 1)
        Hb = similarity_transform(self.H_Nm1, T)
        e_cc = np.vdot(self.ref, self.hbar_N(t1, t2) @ self.ref)
        basis = [self.hole(i) for i in range(o)]
        for i, j in zip(*np.triu_indices(o, 1)):
            for b in range(v):
                basis.append(self.two_hole_particle(i, j, b))
        Bm = np.stack(basis, axis=1)
        M = Bm.conj().T @ Hb @ Bm
        return M - e_cc * np.eye(M.shape[0])

    def mp2_energy(self):
        """Second-order Rayleigh-Schroedinger energy, Moller-Plesset H0.

        H0 = E_ref + sum_p eps_p {a+_p a_p} is diagonal on determinants, so
        E2 = - sum_{D != 0} |<D|H|0>|^2 / (E0(D) - E0(0)).
        """
        sec = Sector(self.n, self.o)
        c = self.H_N @ self.ref
        e0_ref = self.eps[:self.o].sum()
        e2 = 0.0
        ref_det = (1 << self.o) - 1
        for idx, det in enumerate(sec.dets):
            if det == ref_det:
                continue
            e0 = sum(self.eps[p] for p in range(self.n) if det >> p & 1)
            e2 -= abs(c[idx]) ** 2 / (e0 - e0_ref)
        return e2
