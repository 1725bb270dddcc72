"""Davidson starting vectors: the first-order 2h1p start and its features
against the CPU oracle, and what the learned start gains over unit vectors
(the roots themselves must not change)."""
import numpy as np
import pytest

from paper_2506_06805_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_06805_gb300 as P
    P.lib()
    return P


def _system(o, v, X, seed, scale=4.0):
    rng = np.random.default_rng(seed)
    eps = synth.make_eps(rng, o, v)
    L = synth.make_cholesky(rng, o + v, X) * scale
    return eps, L


def _oracle_hbar(eps, L, o):
    from oracle import ccsd, integrals, ipeom
    g = integrals.blocks_from_cholesky(L, o)
    res = ccsd.solve(g, eps, tol=1e-12, max_iter=300)
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    return g, res, H


def _packed_t2(t2, o, v):
    io, jo = np.triu_indices(o, 1)
    av, bv = np.triu_indices(v, 1)
    return t2[io, jo][:, av, bv].ravel()


def test_first_order_start_and_features_match_oracle():
    """GPU first-order starting vectors (from its own H-bar of the oracle's
    amplitudes) against oracle.ipeom.first_order_guess, root by root, and the
    learned start's features against oracle.mlp.guess_features."""
    P = _gpu()
    from oracle import ipeom, mlp
    o, v, X = 6, 20, 60
    eps, L = _system(o, v, X, 21)
    g, res, H = _oracle_hbar(eps, L, o)
    nr = 4
    d = ipeom.diagonal(H, o, v)
    seeds = np.argsort(d.real, kind="stable")[:nr]
    with P.System(eps, L, n_occ=o, tier="fp64") as s:
        s.set_amplitudes(res["t1"], _packed_t2(res["t2"], o, v))
        s.ccsd(tol=1e-10)  # converged start: one iteration, marks CCSD done
        s.set_davidson_guess("first_order")
        got = s.guess_dev(nr).cpu().numpy()
        feats = {int(i): P.Mlp.guess_features(s, int(i), 300) for i in seeds if i < o}
    for r, i in enumerate(seeds):
        if i >= o:
            ref = np.zeros(ipeom.dim(o, v), complex)
            ref[i] = 1.0
        else:
            ref = ipeom.first_order_guess(H, o, v, int(i))
        assert np.abs(got[r] - ref).max() <= 1e-8 * max(1.0, np.abs(ref).max()), r
    assert feats, "no 1h-seeded root at this size"
    for i, f in feats.items():
        ref = mlp.guess_features(H, g, eps, o, i, 300)
        assert np.abs(f - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())


def test_learned_start_gain_and_invariance():
    """Trained on three converged systems, the learned start needs fewer
    Davidson iterations than unit vectors on a held-out fourth system, and
    every start gives the same IPs."""
    P = _gpu()
    o, v, X, nr = 8, 40, 120, 6
    net = P.Mlp(seed=1)
    for seed in (31, 32, 33):
        eps, L = _system(o, v, X, seed)
        with P.System(eps, L, n_occ=o, tier="fp64") as s:
            s.ccsd(tol=1e-10)
            s.ipeom(nr, tol=1e-9)
            net.add_guess_samples(s, 40000)
    perm = np.random.default_rng(0).permutation(net.num_samples())
    net.train(1500, batch=1024, lr=2e-3, perm=perm)
    eps, L = _system(o, v, X, 34)
    out = {}
    with P.System(eps, L, n_occ=o, tier="fp64") as s:
        s.ccsd(tol=1e-10)
        for mode in ("unit", "first_order", "learned"):
            s.set_davidson_guess(mode, net if mode == "learned" else None)
            w, _ = s.ipeom(nr, tol=1e-9)
            out[mode] = (np.sort_complex(w), s.davidson_iterations)
    print("Davidson iterations:", {k: it for k, (_, it) in out.items()})
    for mode in ("first_order", "learned"):
        assert np.abs(out[mode][0] - out["unit"][0]).max() <= 1e-8
    assert out["learned"][1] < out["unit"][1]
    assert out["first_order"][1] <= out["unit"][1]
