"""Left IP-EOM vectors (Eqs. 19-20) through the C ABI against the oracle.

The left sigma (ipeom_left_sigma_dev) is compared element by element with
oracle.ipeom.left_sigma, whose terms are pinned against the transpose of the
brute-force H-bar_IP. The biorthonormal pairs of ipeom_solve_lr are compared
through quantities that do not depend on how a pair is scaled (r -> c r,
l -> l / c): the IPs, the 1h overlaps sum_i l^i r_i, the residuals of both
eigen-equations with the oracle's dense matrix, and L R^T = 1.
"""
import numpy as np
import pytest

from paper_2506_06805_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = {"fp64": 1e-11, "fp16": 4e-3, "fp16x3": 2e-6, "tf32x3": 2e-6}


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_06805_gb300 as P
    P.lib()
    return P


def _system(o, v, X, seed=1, scale=1.0):
    rng = np.random.default_rng(seed)
    eps = synth.make_eps(rng, o, v, False)
    L = synth.make_cholesky(rng, o + v, X, False) * scale
    return eps, L


def _oracle(eps, L, o):
    from oracle import ccsd, integrals, ipeom
    g = integrals.blocks_from_cholesky(L, o)
    res = ccsd.solve(g, eps, tol=1e-12, max_iter=200)
    assert res["converged"]
    return res, ipeom.hbar(g, eps, res["t1"], res["t2"])


@pytest.mark.parametrize("tier", ["fp64", "fp16", "fp16x3"])
def test_left_sigma_matches_oracle(tier):
    """Same shapes as the right sigma's parity test: several tiles and ragged
    tails in every contraction."""
    P = _gpu()
    from oracle import ipeom
    o, v, X = 8, 26, 80
    eps, L = _system(o, v, X, seed=5, scale=4.0)
    res, H = _oracle(eps, L, o)
    rng = np.random.default_rng(4)
    dim = ipeom.dim(o, v)
    k = 5
    Lv = rng.standard_normal((k, dim)) + 1j * rng.standard_normal((k, dim))
    ref = np.stack([ipeom.left_sigma(H, Lv[i], o, v) for i in range(k)])
    io, jo = np.triu_indices(o, 1)
    av, bv = np.triu_indices(v, 1)
    t2p = res["t2"][io, jo][:, av, bv].ravel()
    with P.System(eps, L, n_occ=o, tier=tier) as s:
        s.set_amplitudes(res["t1"], t2p)
        x = torch.from_numpy(np.ascontiguousarray(Lv)).cuda()
        out = torch.zeros((k, dim), dtype=torch.complex128, device="cuda")
        s.left_sigma_dev(x, out)
        got = out.cpu().numpy()
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    assert err <= 10 * REL[tier]


@pytest.mark.parametrize("tier,eom,tol_w,tol_p", [("fp64", "fp64", 1e-8, 1e-7),
                                                  ("fp16", "fp16x3", 1e-5, 1e-4)])
def test_biorthonormal_pairs_match_oracle(tier, eom, tol_w, tol_p):
    P = _gpu()
    from oracle import ipeom
    o, v, X, nr = 6, 14, 40, 4
    eps, L = _system(o, v, X, seed=7, scale=4.0)
    _, H = _oracle(eps, L, o)
    M = ipeom.dense_matrix(H, o, v)
    w_ref, R_ref, L_ref = ipeom.dense_left_right(H, o, v, nr)
    p_ref = np.array([ipeom.pole_strength(L_ref[:, k], R_ref[:, k], o) for k in range(nr)])
    with P.System(eps, L, n_occ=o, tier=tier, eom_tier=eom) as s:
        s.ccsd(tol=1e-10)
        w, R, Lv, pole = s.ipeom_lr(nr, tol=1e-9, max_iter=200)
    assert np.abs(w - w_ref).max() <= tol_w
    assert np.abs(Lv @ R.T - np.eye(nr)).max() <= 1e-8
    assert np.abs(pole - p_ref).max() <= tol_p
    for k in range(nr):
        rk, lk = R[k], Lv[k]
        assert np.linalg.norm(M @ rk - w[k] * rk) <= 1e2 * tol_w * np.linalg.norm(rk)
        assert np.linalg.norm(lk @ M - w[k] * lk) <= 1e2 * tol_w * np.linalg.norm(lk)
