"""Learned warm start: GPU training kernels against the FP64 oracle network,
features against the oracle's, and what the trained network gains."""
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


def test_mlp_loss_and_gradient_match_oracle():
    P = _gpu()
    from oracle import mlp
    rng = np.random.default_rng(5)
    params = P.Mlp.init_params(3)
    params[-130:] = rng.standard_normal(130).astype(np.float32) * 0.2  # non-trivial last layer
    net = P.Mlp(params)
    n = 700
    X = rng.standard_normal((n, 8)).astype(np.float32)
    Y = np.column_stack([rng.standard_normal((n, 2)) * 0.1,
                         rng.uniform(0.2, 3, n)]).astype(np.float32)
    loss, g = net.loss_grad(X, Y)
    # the GPU kernels use the FP16-rounded weights
    p16 = params.astype(np.float16).astype(np.float64)
    ref_loss, ref_g = mlp.loss_grad(p16, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-5 * max(ref_loss, 1e-12)
    assert np.abs(g - ref_g).max() <= 2e-5 * np.abs(ref_g).max()


def test_mlp_features_match_oracle():
    P = _gpu()
    from oracle import mlp
    o, v, X = 4, 9, 20
    eps, L = _system(o, v, X, seed=2)
    with P.System(eps, L, n_occ=o) as s:
        got = P.Mlp.features(s, 60)
    ref = mlp.features(L, eps, o, 60)
    assert np.abs(got - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())


def test_warm_start_gain_and_invariance():
    """Trained on three converged systems, the network's start lies closer to
    the converged amplitudes of a fourth (held-out) system than MP2 does, and
    CCSD from either start converges to the same energy and IPs."""
    P = _gpu()
    o, v, X = 8, 40, 120
    net = P.Mlp(seed=0)
    for seed in (11, 12, 13):
        eps, L = _system(o, v, X, seed)
        with P.System(eps, L, n_occ=o, tier="fp64") as s:
            s.ccsd(tol=1e-10)
            net.add_samples(s, 20000)
    n = net.num_samples()
    perm = np.random.default_rng(0).permutation(n)
    net.train(1500, batch=1024, lr=2e-3, perm=perm)
    eps, L = _system(o, v, X, 14)
    out = {}
    for start in ("mp2", "mlp"):
        with P.System(eps, L, n_occ=o, tier="fp64") as s:
            t0 = None
            if start == "mlp":
                net.warm_start(s)
                t0 = s.get_amplitudes()[1]
            e = s.ccsd(tol=1e-10)
            w, _ = s.ipeom(4, tol=1e-8)
            out[start] = (e, np.sort_complex(w), s.ccsd_iterations, t0, s.get_amplitudes()[1])
    e0, w0, it0, _, tc = out["mp2"]
    e1, w1, it1, t_mlp, _ = out["mlp"]
    assert abs(e0 - e1) <= 1e-9
    assert np.abs(w0 - w1).max() <= 1e-8
    from oracle import integrals, mp2
    g = integrals.blocks_from_cholesky(L, o)
    t_mp2 = mp2.amplitudes(g, eps)
    io, jo = np.triu_indices(o, 1)
    av, bv = np.triu_indices(v, 1)
    t_mp2p = t_mp2[io, jo][:, av, bv].ravel()
    d_mp2 = np.linalg.norm(t_mp2p - tc)
    d_mlp = np.linalg.norm(t_mlp - tc)
    print(f"warm start: |t0 - t_conv| MP2 {d_mp2:.3e} MLP {d_mlp:.3e}; "
          f"iterations MP2 {it0} MLP {it1}")
    assert d_mlp < 0.7 * d_mp2
    assert it1 <= it0
