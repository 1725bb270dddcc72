"""Pins of the CPU oracle against facts fixed by theory (no GPU).

Each test checks the oracle against something other than itself: the
brute-force Fock-space module (exact e^{-T} H e^{T}, FCI, Rayleigh-
Schroedinger MP2), closed forms (Koopmans' theorem at zero coupling),
invariances (spinor phases, virtual rotations), symmetries (Kramers pairs,
real inputs) and scaling limits. A dropped term, wrong sign, wrong index or
transposed operand in the working equations fails at least one of them.
"""
import numpy as np
import pytest

from paper_2506_06805_gb300 import synth
from oracle import ccsd, cholesky, davidson, fci, fns, integrals, ipeom, mp2


def _system(o, v, X, seed=1, scale=1.0, kramers=False):
    rng = np.random.default_rng(seed)
    eps = synth.make_eps(rng, o, v, kramers)
    L = synth.make_cholesky(rng, o + v, X, kramers) * scale
    return eps, L


def _random_amplitudes(rng, o, v, s=0.05):
    t1 = s * (rng.standard_normal((o, v)) + 1j * rng.standard_normal((o, v)))
    t2 = s * (rng.standard_normal((o, o, v, v))
              + 1j * rng.standard_normal((o, o, v, v)))
    t2 = t2 - t2.transpose(1, 0, 2, 3)
    t2 = 0.5 * (t2 - t2.transpose(0, 1, 3, 2))
    return t1, t2


def _offdiag_mask(o, v):
    m = np.ones((o, o, v, v), bool)
    for i in range(o):
        m[i, i] = False
    for a in range(v):
        m[:, :, a, a] = False
    return m


# --- integrals (Eq. 23) ------------------------------------------------------

def test_integral_symmetries():
    eps, L = _system(3, 6, 15, scale=5.0)
    g = integrals.antisym_full(L)
    scale = np.abs(g).max()
    assert np.abs(g + g.transpose(1, 0, 2, 3)).max() <= 1e-15 * scale
    assert np.abs(g + g.transpose(0, 1, 3, 2)).max() <= 1e-15 * scale
    # Hermitian L^P  =>  <pq||rs> = <rs||pq>*
    assert np.abs(g - g.transpose(2, 3, 0, 1).conj()).max() <= 1e-15 * scale


def test_integrals_against_scalar_loop():
    """Eq. 23 evaluated element by element in plain Python."""
    eps, L = _system(2, 3, 4, scale=3.0)
    g = integrals.antisym_full(L)
    n = L.shape[1]
    rng = np.random.default_rng(0)
    for _ in range(40):
        p, q, r, s = rng.integers(0, n, size=4)
        ref = 0j
        for P in range(L.shape[0]):
            ref += L[P, p, r] * L[P, q, s] - L[P, p, s] * L[P, q, r]
        assert abs(g[p, q, r, s] - ref) <= 1e-15


def _fixed_order_scalar(L, p, q, r, s):
    """One element of Eq. 23 in plain Python floats: P ascending, each
    complex product as (ar*br - ai*bi, ar*bi + ai*br), term = direct -
    exchange added to the running sum (Python rounds every operation to
    nearest, with no fused multiply-add)."""
    acc_r = 0.0
    acc_i = 0.0
    for P in range(L.shape[0]):
        ar, ai = float(L[P, p, r].real), float(L[P, p, r].imag)
        br, bi = float(L[P, q, s].real), float(L[P, q, s].imag)
        cr, ci = float(L[P, p, s].real), float(L[P, p, s].imag)
        dr, di = float(L[P, q, r].real), float(L[P, q, r].imag)
        d1r = ar * br - ai * bi
        d1i = ar * bi + ai * br
        d2r = cr * dr - ci * di
        d2i = cr * di + ci * dr
        acc_r = acc_r + (d1r - d2r)
        acc_i = acc_i + (d1i - d2i)
    return acc_r, acc_i


def test_fixed_order_integrals_equal_scalar_loop_bit_for_bit():
    """antisym_fixed_order (the comparator of the bit-exact integral dump)
    equals the element-by-element scalar loop bit for bit on random blocks,
    and the unordered einsum form within 1e-15 relative."""
    o, v = 3, 7
    eps, L = _system(o, v, 11, seed=4, scale=5.0)
    n = o + v
    rng = np.random.default_rng(2)
    for _ in range(4):
        lo = rng.integers(0, n - 2, size=4)
        hi = [int(x) + int(rng.integers(1, 3)) for x in lo]
        sl = [slice(int(a), b) for a, b in zip(lo, hi)]
        got = integrals.antisym_fixed_order(L, *sl)
        ref = integrals.antisym_full(L)[tuple(sl)]
        assert np.abs(got - ref).max() <= 1e-15 * np.abs(ref).max()
        for idx in np.ndindex(got.shape):
            pqrs = [s_.start + k for s_, k in zip(sl, idx)]
            er, ei = _fixed_order_scalar(L, *pqrs)
            assert got[idx].real == er and got[idx].imag == ei, (idx, got[idx], er, ei)


def test_fixed_order_integrals_exact_on_integer_vectors():
    """With small-integer Cholesky vectors every product and partial sum is
    an integer below 2^53, so FP64 evaluation in any order is exact: the
    result must equal Eq. 23 in exact integer arithmetic, and swapping p, q
    (or r, s) must negate it bit for bit."""
    rng = np.random.default_rng(8)
    X, n = 6, 5
    L = (rng.integers(-40, 41, size=(X, n, n))
         + 1j * rng.integers(-40, 41, size=(X, n, n))).astype(np.complex128)
    full = slice(0, n)
    got = integrals.antisym_fixed_order(L, full, full, full, full)
    Li = [[[complex(L[P, a, b]) for b in range(n)] for a in range(n)] for P in range(X)]
    for p, q, r, s in np.ndindex(n, n, n, n):
        re = im = 0
        for P in range(X):
            d1 = Li[P][p][r] * Li[P][q][s]
            d2 = Li[P][p][s] * Li[P][q][r]
            re += int(d1.real) - int(d2.real)
            im += int(d1.imag) - int(d2.imag)
        assert got[p, q, r, s] == complex(re, im)
    assert np.array_equal(got, -got.transpose(1, 0, 2, 3))
    assert np.array_equal(got, -got.transpose(0, 1, 3, 2))


# --- MP2 ---------------------------------------------------------------------

def test_mp2_equals_rayleigh_schroedinger_second_order():
    eps, L = _system(3, 5, 12, scale=8.0)
    G = integrals.antisym_full(L)
    g = integrals.Blocks(G, 3)
    bf = fci.BruteForce(eps, G, 3)
    e_bf = bf.mp2_energy()
    e_or = mp2.energy(g, mp2.amplitudes(g, eps))
    assert abs(e_or - e_bf) <= 1e-13 * abs(e_bf)
    assert abs(e_or.imag) <= 1e-15


def test_ccsd_energy_at_mp2_amplitudes_is_mp2():
    eps, L = _system(3, 5, 12, scale=8.0)
    g = integrals.blocks_from_cholesky(L, 3)
    t2 = mp2.amplitudes(g, eps)
    t1 = np.zeros((3, 5), complex)
    assert ccsd.energy(g, t1, t2) == mp2.energy(g, t2)


# --- CCSD working equations vs exact similarity transform --------------------

@pytest.mark.parametrize("o,v,X,seed", [(3, 5, 12, 1), (2, 6, 10, 2),
                                        (4, 4, 9, 3)])
def test_ccsd_residual_equals_bruteforce_projection(o, v, X, seed):
    """<mu| e^{-T} H e^{T} |0> = R - D t for ANY amplitudes (Eqs. 13-15)."""
    eps, L = _system(o, v, X, seed=seed, scale=10.0)
    G = integrals.antisym_full(L)
    g = integrals.Blocks(G, o)
    bf = fci.BruteForce(eps, G, o)
    rng = np.random.default_rng(seed)
    t1, t2 = _random_amplitudes(rng, o, v)
    e_tot, P1, P2 = bf.projections(t1, t2)
    R1, R2 = ccsd.residuals(g, eps, t1, t2)
    D1 = mp2.denom1(eps, o)
    D2 = mp2.denom2(eps, o)
    assert abs((e_tot - bf.e_ref) - ccsd.energy(g, t1, t2)) <= 1e-13
    assert np.abs(P1 - (R1 - D1 * t1)).max() <= 1e-13
    m = _offdiag_mask(o, v)
    assert np.abs((P2 - (R2 - D2 * t2))[m]).max() <= 1e-13


def test_ladder_term_alone_equals_bruteforce():
    """With only virtual-virtual Cholesky blocks and eps = 0, every integral
    but <ab||cd> vanishes and the doubles projection at t1 = 0 is the ladder
    1/2 sum_cd <ab||cd> t_ij^cd alone."""
    o, v, X = 2, 5, 8
    eps, L = _system(o, v, X, scale=10.0)
    L[:, :o, :] = 0.0
    L[:, :, :o] = 0.0
    eps = np.zeros_like(eps)
    G = integrals.antisym_full(L)
    bf = fci.BruteForce(eps, G, o)
    rng = np.random.default_rng(5)
    _, t2 = _random_amplitudes(rng, o, v)
    t1 = np.zeros((o, v), complex)
    _, _, P2 = bf.projections(t1, t2)
    lad = ccsd.ladder_term(G[o:, o:, o:, o:], t2)
    m = _offdiag_mask(o, v)
    assert np.abs((P2 - lad)[m]).max() <= 1e-14
    assert np.abs(lad).max() > 1e-3


def test_diis_does_not_move_the_fixed_point():
    """DIIS (from iteration 2 or 3, any depth) only accelerates: the
    converged amplitudes solve the same equations as plain Jacobi."""
    o, v, X = 4, 9, 20
    eps, L = _system(o, v, X, seed=8, scale=4.0)
    g = integrals.blocks_from_cholesky(L, o)
    plain = ccsd.solve(g, eps, tol=1e-12, max_iter=500, diis_start=10 ** 9)
    assert plain["converged"]
    for size, start in ((8, 2), (8, 3), (3, 2)):
        res = ccsd.solve(g, eps, tol=1e-12, max_iter=200, diis_size=size, diis_start=start)
        assert res["converged"] and res["n_iter"] <= plain["n_iter"]
        assert abs(res["e_corr"] - plain["e_corr"]) < 1e-11
        assert np.abs(res["t2"] - plain["t2"]).max() < 1e-10


def test_ccsd_two_electrons_is_fci():
    """n_occ = 2: CCSD is exact; 1h + 2h1p spans the whole one-electron
    sector, so the IP-EOM roots are FCI(N-1) - FCI(N)."""
    o, v, X = 2, 6, 14
    eps, L = _system(o, v, X, seed=4, scale=8.0)
    G = integrals.antisym_full(L)
    g = integrals.Blocks(G, o)
    res = ccsd.solve(g, eps, tol=1e-12, max_iter=300)
    assert res["converged"]
    bf = fci.BruteForce(eps, G, o)
    e_fci = np.linalg.eigvals(bf.H_N)
    # the CC root is the FCI root closest to the CC energy (the ground state)
    e_cc = bf.e_ref + res["e_corr"]
    e0 = e_fci[np.argmin(np.abs(e_fci - e_cc))]
    assert e0.real == pytest.approx(np.min(e_fci.real), abs=1e-12)
    assert abs(e_cc - e0) <= 1e-10
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    w = np.sort_complex(np.linalg.eigvals(ipeom.dense_matrix(H, o, v)))
    w_fci = np.sort_complex(np.linalg.eigvals(bf.H_Nm1) - e0)
    assert np.abs(w - w_fci).max() <= 1e-9


@pytest.mark.parametrize("o,v,X,seed", [(3, 5, 12, 1), (4, 3, 10, 6)])
def test_ip_matrix_equals_bruteforce(o, v, X, seed):
    """H-bar_IP from the sigma equations equals <mu|Hbar - E|nu> exactly
    (n_occ >= 3 is where the truncation matters)."""
    eps, L = _system(o, v, X, seed=seed, scale=10.0)
    G = integrals.antisym_full(L)
    g = integrals.Blocks(G, o)
    res = ccsd.solve(g, eps, tol=1e-13, max_iter=400)
    assert res["converged"]
    bf = fci.BruteForce(eps, G, o)
    e_tot, P1, P2 = bf.projections(res["t1"], res["t2"])
    assert np.abs(P1).max() < 1e-11 and np.abs(P2).max() < 1e-11
    M_bf = bf.ip_matrix(res["t1"], res["t2"])
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    M = ipeom.dense_matrix(H, o, v)
    assert np.abs(M - M_bf).max() <= 1e-10 * max(1.0, np.abs(M_bf).max())


@pytest.mark.parametrize("o,v,X,seed", [(3, 5, 12, 1), (4, 3, 10, 6)])
def test_left_vectors_against_bruteforce(o, v, X, seed):
    """Eqs. 19-20: left_sigma is the transpose of the brute-force H-bar_IP
    (every sign and factor of the exchanged terms), and the oracle's left and
    right vectors are eigenvectors of that matrix, biorthonormal over all
    roots, with 1h overlaps summing to o (completeness)."""
    eps, L = _system(o, v, X, seed=seed, scale=10.0)
    G = integrals.antisym_full(L)
    g = integrals.Blocks(G, o)
    res = ccsd.solve(g, eps, tol=1e-13, max_iter=400)
    assert res["converged"]
    M_bf = fci.BruteForce(eps, G, o).ip_matrix(res["t1"], res["t2"])
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    n = ipeom.dim(o, v)
    scale = max(1.0, np.abs(M_bf).max())
    rng = np.random.default_rng(seed)
    for _ in range(3):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        assert np.abs(ipeom.left_sigma(H, x, o, v) - M_bf.T @ x).max() <= 1e-12 * scale * n
    w, R, Lv = ipeom.dense_left_right(H, o, v, n)
    for k in range(n):
        assert np.abs(Lv[:, k] @ M_bf - w[k] * Lv[:, k]).max() <= 1e-10 * scale * np.abs(Lv[:, k]).max()
        assert np.abs(M_bf @ R[:, k] - w[k] * R[:, k]).max() <= 1e-10 * scale
    assert np.abs(Lv.T @ R - np.eye(n)).max() <= 1e-10
    total = sum(ipeom.pole_strength(Lv[:, k], R[:, k], o) for k in range(n))
    assert abs(total - o) <= 1e-9


def test_pole_strengths_at_zero_coupling():
    """L = 0: H-bar_IP is the diagonal Koopmans matrix; each 1h root has
    1h overlap 1 and each 2h1p root 0."""
    o, v = 4, 5
    eps, L = _system(o, v, 8)
    L = 0 * L
    g = integrals.blocks_from_cholesky(L, o)
    z1 = np.zeros((o, v), complex)
    z2 = np.zeros((o, o, v, v), complex)
    H = ipeom.hbar(g, eps, z1, z2)
    n = ipeom.dim(o, v)
    w, R, Lv = ipeom.dense_left_right(H, o, v, n)
    p = np.array([ipeom.pole_strength(Lv[:, k], R[:, k], o) for k in range(n)])
    is_1h = np.abs(R[:o, :]).max(axis=0) > 0.5
    assert is_1h.sum() == o
    assert np.abs(p[is_1h] - 1).max() <= 1e-12
    assert np.abs(p[~is_1h]).max() <= 1e-12


def test_r1_weight_limits():
    """r1_weight = ||r1||^2 / ||r||^2: exactly 1 for the 1h roots and 0 for
    the 2h1p roots at zero coupling; unchanged by a complex scale of the
    vector; and at weak coupling the 2h1p admixture of a 1h root follows
    first-order perturbation theory, 1 - w -> sum_nu |M_nu,i|^2 /
    |omega_i - M_nu,nu|^2 (the relative deviation shrinks with lam)."""
    o, v = 3, 4
    eps, L0 = _system(o, v, 9, seed=5, scale=6.0)
    g = integrals.blocks_from_cholesky(0 * L0, o)
    z1, z2 = np.zeros((o, v), complex), np.zeros((o, o, v, v), complex)
    H = ipeom.hbar(g, eps, z1, z2)
    n = ipeom.dim(o, v)
    w, V = ipeom.dense_roots(H, o, v, n)
    wts = np.array([ipeom.r1_weight(V[:, k], o) for k in range(n)])
    assert np.sum(wts == 1.0) == o and np.sum(wts == 0.0) == n - o
    x = np.random.default_rng(0).standard_normal(n) + 1j
    assert ipeom.r1_weight((2.5 - 1.5j) * x, o) == pytest.approx(ipeom.r1_weight(x, o), rel=1e-14)
    devs = []
    for lam in (0.2, 0.1):
        L = lam * L0
        gb = integrals.blocks_from_cholesky(L, o)
        res = ccsd.solve(gb, eps, tol=1e-13, max_iter=300)
        Hb = ipeom.hbar(gb, eps, res["t1"], res["t2"])
        M = ipeom.dense_matrix(Hb, o, v)
        w, V = ipeom.dense_roots(Hb, o, v, n)
        k = int(np.argmax([ipeom.r1_weight(V[:, j], o) for j in range(n)]))
        i = int(np.argmax(np.abs(V[:o, k])))
        pt = sum(abs(M[nu, i]) ** 2 / abs(w[k] - M[nu, nu]) ** 2 for nu in range(o, n))
        devs.append(abs((1.0 - ipeom.r1_weight(V[:, k], o)) / pt - 1.0))
    assert devs[1] < 0.6 * devs[0] and devs[1] < 1e-3


def test_first_order_guess_is_perturbation_theory():
    """The first-order Davidson start of a 1h-dominated root against the
    exact eigenvector x (dense H-bar_IP), by the overlap deficit
    1 - |<g|x>|^2 / (|g|^2 |x|^2). With L -> lam L the couplings scale as
    lam^2, so the unit vector e_i misses a 2h1p part of order lam^2 (deficit
    ~ lam^4, a factor 16 per halving) while the first-order vector leaves
    only the second-order part (deficit ~ lam^8, a factor 256)."""
    o, v = 3, 5
    eps, L0 = _system(o, v, 10, seed=7, scale=5.0)
    n = ipeom.dim(o, v)

    def deficits(lam):
        L = lam * L0
        g = integrals.blocks_from_cholesky(L, o)
        res = ccsd.solve(g, eps, tol=1e-13, max_iter=300)
        H = ipeom.hbar(g, eps, res["t1"], res["t2"])
        w, V = ipeom.dense_roots(H, o, v, n)
        k = int(np.argmax([ipeom.r1_weight(V[:, j], o) for j in range(n)]))
        x = V[:, k]
        i = int(np.argmax(np.abs(x[:o])))
        e = np.zeros(n, complex)
        e[i] = 1.0
        gfo = ipeom.first_order_guess(H, o, v, i)

        def deficit(y):
            return 1.0 - abs(np.vdot(y, x)) ** 2 / (np.vdot(y, y).real * np.vdot(x, x).real)
        return deficit(gfo), deficit(e)

    f1, u1 = deficits(0.4)
    f2, u2 = deficits(0.2)
    assert f1 < 1e-3 * u1 and f2 < 1e-3 * u2
    assert 10.0 < u1 / u2 < 25.0         # deficit of e_i ~ lam^4
    assert 150.0 < f1 / f2 < 400.0       # first-order deficit ~ lam^8


# --- closed forms and invariances ---------------------------------------------

def test_koopmans_at_zero_coupling():
    o, v = 4, 6
    eps, L = _system(o, v, 5)
    L[:] = 0.0
    g = integrals.blocks_from_cholesky(L, o)
    res = ccsd.solve(g, eps, tol=1e-12)
    assert res["e_corr"] == 0.0
    assert np.all(res["t1"] == 0) and np.all(res["t2"] == 0)
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    w = np.sort(np.linalg.eigvals(ipeom.dense_matrix(H, o, v)).real)
    eo, ev = eps[:o], eps[o:]
    exact = [-e for e in eo]
    for i in range(o):
        for j in range(i + 1, o):
            exact += [b - eo[i] - eo[j] for b in ev]
    assert np.array_equal(w, np.sort(exact)) or np.abs(
        w - np.sort(exact)).max() <= 1e-15


def test_weak_coupling_limits():
    """L -> lam L: E_CCSD / E_MP2 -> 1 and IP - Koopmans = O(lam^4)."""
    o, v, X = 4, 8, 16
    eps, L0 = _system(o, v, X, seed=3, scale=6.0)
    ratios, shifts = [], []
    for lam in (1.0, 0.5, 0.25):
        g = integrals.blocks_from_cholesky(L0 * lam, o)
        res = ccsd.solve(g, eps, tol=1e-13, max_iter=200)
        ratios.append((res["e_corr"] / mp2.energy(
            g, mp2.amplitudes(g, eps))).real)
        H = ipeom.hbar(g, eps, res["t1"], res["t2"])
        w, _ = ipeom.dense_roots(H, o, v, 1)
        shifts.append(abs(w[0] - (-eps[o - 1])))
    assert abs(ratios[2] - 1) < abs(ratios[1] - 1) < abs(ratios[0] - 1)
    assert abs(ratios[2] - 1) < 1e-2
    # halving lam divides the shift by ~16
    assert 12.0 < shifts[1] / shifts[2] < 20.0


def test_gauge_invariance():
    """Spinor phases change amplitudes but not E or the IPs. Catches
    conjugation mistakes that real tests cannot see."""
    o, v, X = 4, 8, 16
    eps, L = _system(o, v, X, seed=7, scale=6.0)
    theta = np.random.default_rng(9).uniform(0, 2 * np.pi, o + v)
    out = []
    for LL in (L, synth.gauge_transform(L, theta)):
        g = integrals.blocks_from_cholesky(LL, o)
        res = ccsd.solve(g, eps, tol=1e-13, max_iter=200)
        H = ipeom.hbar(g, eps, res["t1"], res["t2"])
        w, _ = ipeom.dense_roots(H, o, v, 5)
        out.append((res["e_corr"], w))
    assert abs(out[0][0] - out[1][0]) <= 1e-13
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-11


def test_real_inputs_give_real_results():
    o, v, X = 4, 6, 12
    eps, L = _system(o, v, X, seed=8, scale=6.0)
    L = L.real.astype(complex)
    g = integrals.blocks_from_cholesky(L, o)
    res = ccsd.solve(g, eps, tol=1e-13, max_iter=200)
    assert np.abs(res["t2"].imag).max() == 0.0
    assert res["e_corr"].imag == 0.0


def test_kramers_pairs_are_degenerate():
    o, v, X = 4, 8, 16
    eps, L = _system(o, v, X, seed=2, scale=6.0, kramers=True)
    g = integrals.blocks_from_cholesky(L, o)
    res = ccsd.solve(g, eps, tol=1e-13, max_iter=200)
    assert abs(res["e_corr"].imag) <= 1e-14
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    w, _ = ipeom.dense_roots(H, o, v, 8)
    w = np.sort(w.real)
    assert np.abs(w[0::2] - w[1::2]).max() <= 1e-10
    assert np.min(np.diff(w[0::2])) > 1e-4


# --- frozen natural spinors (Eqs. 24-28) ---------------------------------------

def test_fns_density_properties():
    o, v, X = 4, 10, 20
    eps, L = _system(o, v, X, seed=5, scale=6.0)
    D = fns.vv_density(L, eps, o)
    assert np.abs(D - D.conj().T).max() <= 1e-15 * np.abs(D).max()
    n = np.linalg.eigvalsh(D)
    assert n.min() >= -1e-15
    g = integrals.blocks_from_cholesky(L, o)
    t2 = mp2.amplitudes(g, eps)
    assert abs(np.trace(D) - 0.5 * np.sum(np.abs(t2) ** 2)) <= 1e-14
    # Eq. 24 element against a plain loop
    G = integrals.antisym_full(L)
    ev, eo = eps[o:], eps[:o]
    a, b = 2, 7
    ref = 0j
    for c in range(v):
        for i in range(o):
            for j in range(o):
                ref += (G[o + a, o + c, i, j] * G[i, j, o + b, o + c]
                        / ((eo[i] + eo[j] - ev[a] - ev[c])
                           * (eo[i] + eo[j] - ev[b] - ev[c])))
    assert abs(D[a, b] - 0.5 * ref) <= 1e-15


def test_fns_keep_all_is_invariant():
    """Threshold 0 keeps every virtual: CCSD and IP-EOM are invariant under
    the unitary virtual rotation U (Eq. 28)."""
    o, v, X = 4, 8, 16
    eps, L = _system(o, v, X, seed=6, scale=6.0)
    out = fns.frozen_natural_spinors(L, eps, o, n_keep=v)
    U = out["U"]
    assert np.abs(U.conj().T @ U - np.eye(v)).max() <= 1e-13
    assert np.abs(np.linalg.eigvalsh(out["F_ns"]) - out["eps_virt"]).max() \
        <= 1e-13
    res = []
    for ee, LL in ((eps, L), (out["eps"], out["L"])):
        # the Fock matrix in the rotated basis is diag(eps~): semicanonical
        g = integrals.blocks_from_cholesky(LL, o)
        r = ccsd.solve(g, ee, tol=1e-13, max_iter=200)
        H = ipeom.hbar(g, ee, r["t1"], r["t2"])
        w, _ = ipeom.dense_roots(H, o, v, 4)
        res.append((r["e_corr"], w))
    assert abs(res[0][0] - res[1][0]) <= 1e-10
    assert np.abs(res[0][1] - res[1][1]).max() <= 1e-10


def test_fns_truncation_keeps_largest_occupations():
    o, v, X = 4, 12, 24
    eps, L = _system(o, v, X, seed=6, scale=6.0)
    occ = fns.natural_spinors(fns.vv_density(L, eps, o))[0]
    thr = 0.5 * (occ[5] + occ[6])
    out = fns.frozen_natural_spinors(L, eps, o, threshold=thr)
    assert out["n_keep"] == 6
    assert out["L"].shape == (X, o + 6, o + 6)
    Lr = out["L"]
    assert np.abs(Lr - Lr.conj().transpose(0, 2, 1)).max() <= 1e-15
    # truncated CCSD recovers most of the correlation energy
    e_full = ccsd.solve(integrals.blocks_from_cholesky(L, o), eps,
                        tol=1e-10)["e_corr"].real
    e_fns = ccsd.solve(integrals.blocks_from_cholesky(Lr, o), out["eps"],
                       tol=1e-10)["e_corr"].real
    assert 0.5 * e_full > e_fns > 1.05 * e_full or e_full < e_fns < 0


# --- pivoted Cholesky (Eq. 21) -----------------------------------------------------

def _generator(N, r, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))) / np.sqrt(2 * r)


def test_cholesky_error_bound_and_rank():
    """The remainder is PSD with diagonal below tau, so no element of
    M - L^T conj(L) exceeds tau; at a tau far below the spectrum the count
    equals the rank of M and M is recovered to rounding."""
    N, r = 60, 25
    B = _generator(N, r, 2)
    M = B @ B.conj().T
    prev = 0
    for tau in (1e-1, 1e-2, 1e-5):
        L, piv = cholesky.pivoted_cholesky(B, tau)
        E = M - L.T @ L.conj()
        assert np.abs(E).max() < tau
        assert len(piv) == len(set(piv.tolist())) and len(piv) >= prev
        prev = len(piv)
    L, _ = cholesky.pivoted_cholesky(B, 1e-12)
    assert L.shape[0] == r
    assert np.abs(M - L.T @ L.conj()).max() < 1e-12


def test_cholesky_full_rank_equals_lapack():
    """Full rank with tau = 0: in pivot order the vectors are the lower
    triangular Cholesky factor of the permuted matrix (LAPACK's, unique with
    a positive diagonal)."""
    N = 30
    B = _generator(N, 50, 3)
    M = B @ B.conj().T
    L, piv = cholesky.pivoted_cholesky(B, 0.0, max_vec=N)
    assert sorted(piv.tolist()) == list(range(N))
    C = np.linalg.cholesky(M[np.ix_(piv, piv)])
    assert np.abs(L[:, piv].T - C).max() < 1e-12


def test_cholesky_recovers_coulomb_integrals():
    """Generator B[(pq), P] = L^P_pq from Hermitian Cholesky vectors: the
    new vectors reproduce (pr|qs) = sum_P L^P_pr L^P_qs (Eq. 21 in the
    pair-matrix form M[(pr), (sq)] = (pr|qs)) and their count is X."""
    n, X = 7, 12
    L_in = synth.make_cholesky(np.random.default_rng(4), n, X)
    B = L_in.reshape(X, n * n).T.copy()
    Lc, _ = cholesky.pivoted_cholesky(B, 1e-13)
    assert Lc.shape[0] == X
    eri = np.einsum("Ppr,Pqs->prqs", L_in, L_in)
    Mc = Lc.T @ Lc.conj()  # [(pr), (sq)]
    eri_c = Mc.reshape(n, n, n, n).transpose(0, 1, 3, 2)  # (pr|qs) at [p][r][q][s]
    assert np.abs(eri_c - eri).max() < 1e-12


# --- Davidson -------------------------------------------------------------------

def test_davidson_matches_dense():
    o, v, X = 5, 8, 16
    eps, L = _system(o, v, X, seed=11, scale=6.0)
    g = integrals.blocks_from_cholesky(L, o)
    res = ccsd.solve(g, eps, tol=1e-12, max_iter=200)
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    w_dense, _ = ipeom.dense_roots(H, o, v, 6)
    w, X_, it, conv = davidson.davidson(
        lambda x: ipeom.sigma(H, x, o, v), ipeom.diagonal(H, o, v), 6,
        tol=1e-9)
    assert conv
    assert np.abs(w - w_dense).max() <= 1e-9
    # the same Davidson on the transposed sigma: the left problem has the
    # same eigenvalues, and its vectors are left eigenvectors of the matrix
    wl, Xl, _, conv = davidson.davidson(
        lambda x: ipeom.left_sigma(H, x, o, v), ipeom.diagonal(H, o, v), 6,
        tol=1e-9)
    assert conv
    assert np.abs(wl - w_dense).max() <= 1e-9
    M = ipeom.dense_matrix(H, o, v)
    for k in range(6):
        assert np.linalg.norm(Xl[:, k] @ M - wl[k] * Xl[:, k]) <= 1e-8


# --- warm-start network (oracle side) ------------------------------------------

def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.N_PARAMS) * 0.3
    X = rng.standard_normal((17, mlp.F))
    Y = np.column_stack([rng.standard_normal((17, 2)), rng.uniform(0.5, 2, 17)])
    loss, g = mlp.loss_grad(p, X, Y)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    for k in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss_grad(pp, X, Y)[0] - mlp.loss_grad(pm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_mlp_features_are_gauge_invariant():
    from oracle import mlp
    o, v, X = 3, 6, 10
    eps, L = _system(o, v, X, seed=3, scale=5.0)
    theta = np.random.default_rng(1).uniform(0, 2 * np.pi, o + v)
    f1 = mlp.features(L, eps, o, 20)
    f2 = mlp.features(synth.gauge_transform(L, theta), eps, o, 20)
    assert np.abs(f1 - f2).max() <= 1e-10


def test_guess_features_are_gauge_invariant_and_first_order_consistent():
    """The Davidson-start features do not change under spinor phase changes
    (each is a magnitude, a diagonal element or an indicator), and the first
    feature is log10 of the first-order component the start is built from."""
    from oracle import mlp
    o, v, X = 3, 5, 10
    eps, L = _system(o, v, X, seed=3, scale=5.0)
    theta = np.random.default_rng(2).uniform(0, 2 * np.pi, o + v)
    out = []
    for Lx in (L, synth.gauge_transform(L, theta)):
        g = integrals.blocks_from_cholesky(Lx, o)
        res = ccsd.solve(g, eps, tol=1e-12, max_iter=300)
        H = ipeom.hbar(g, eps, res["t1"], res["t2"])
        out.append((mlp.guess_features(H, g, eps, o, 1, 15), ipeom.first_order_guess(H, o, v, 1)))
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-8
    c = out[0][1][o:o + 15]
    assert np.abs(out[0][0][:, 0] - np.log10(np.abs(c) + 1e-30)).max() <= 1e-12
