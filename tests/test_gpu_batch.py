"""Batched IP-EOM over several systems of uneven size (one grouped
persistent tensor-core launch per batched sigma, replayed from CUDA graphs)
against the CPU oracle, system by system, and the tile autotuner."""
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


SHAPES = [(6, 20, 60, 1), (8, 26, 80, 2), (5, 31, 50, 3)]


def _inputs(o, v, X, seed):
    rng = np.random.default_rng(seed)
    eps = synth.make_eps(rng, o, v)
    L = synth.make_cholesky(rng, o + v, X) * 4.0
    return eps, L


def _oracle(o, v, X, seed, n_roots):
    """Lowest n_roots IPs (by real part) and their r1 weights from the
    oracle's dense H-bar_IP (Eqs. 16-18) at the oracle's CCSD amplitudes."""
    from oracle import ccsd, integrals, ipeom
    eps, L = _inputs(o, v, X, seed)
    g = integrals.blocks_from_cholesky(L, o)
    res = ccsd.solve(g, eps, tol=1e-12, max_iter=300)
    assert res["converged"]
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    w, V = ipeom.dense_roots(H, o, v, n_roots)
    return w, np.array([ipeom.r1_weight(V[:, k], o) for k in range(n_roots)])


def _converged(P, o, v, X, seed, tier):
    eps, L = _inputs(o, v, X, seed)
    s = P.System(eps, L, n_occ=o, tier="fp64", eom_tier=tier)
    s.ccsd(tol=1e-11)
    return s


@pytest.mark.parametrize("tier", ["fp64", "tf32x3"])
def test_batch_ipeom_matches_oracle(tier):
    """Each system's batched roots and r1 weights against the oracle's dense
    eigenvalues of its own H-bar_IP."""
    P = _gpu()
    ref = [_oracle(*sh, 4) for sh in SHAPES]
    systems = [_converged(P, *sh, tier) for sh in SHAPES]
    try:
        w, r1, it, status = P.batch_ipeom(systems, 4, tol=1e-9)
    finally:
        for s in systems:
            s.close()
    assert np.all(status == 0)
    tol = 1e-9 if tier == "fp64" else 1e-8
    for q in range(len(SHAPES)):
        order = np.argsort(w[q].real, kind="stable")
        assert np.abs(w[q][order] - ref[q][0]).max() <= tol
        assert np.abs(r1[q][order] - ref[q][1]).max() <= 1e-6


def test_graph_replay_matches_oracle():
    """Roots with the batched sigma replayed from a CUDA graph and without,
    each against the oracle's dense roots."""
    P = _gpu()
    w_ref, _ = _oracle(8, 30, 90, 4, 6)
    for graphs in (False, True):
        with _converged(P, 8, 30, 90, 4, "tf32x3") as s:
            s.set_graphs(graphs)
            w, _ = s.ipeom(6, tol=1e-9)
            assert np.abs(np.sort_complex(w) - np.sort_complex(w_ref)).max() <= 1e-8


def test_autotuner_picks_and_persists(tmp_path, monkeypatch):
    P = _gpu()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("CDFNS_AUTOTUNE", "1")
    monkeypatch.setenv("CDFNS_TUNE_CACHE", str(cache))
    rng = np.random.default_rng(0)
    M, N, K = 300, 700, 900
    A = torch.from_numpy(rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).cuda()
    B = torch.from_numpy(rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))).cuda()
    ref = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    P.zgemm_dev(A, B, ref, "fp64")
    C = torch.zeros_like(ref)
    P.zgemm_dev(A, B, C, "tf32x3")
    err = ((C - ref).abs().max() / ref.abs().max()).item()
    assert err <= 2e-6
    text = cache.read_text()
    assert text.strip().startswith("{") and ":" in text
