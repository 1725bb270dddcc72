"""Batched IP-EOM over several systems of uneven size (one grouped
persistent tensor-core launch per batched sigma, replayed from CUDA graphs)
against one-at-a-time solves, and the tile autotuner."""
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


def _converged(P, o, v, X, seed, tier):
    rng = np.random.default_rng(seed)
    eps = synth.make_eps(rng, o, v)
    L = synth.make_cholesky(rng, o + v, X) * 4.0
    s = P.System(eps, L, n_occ=o, tier="fp64", eom_tier=tier)
    s.ccsd(tol=1e-11)
    return s


@pytest.mark.parametrize("tier", ["fp64", "tf32x3"])
def test_batch_ipeom_matches_individual(tier):
    P = _gpu()
    ref = []
    for o, v, X, seed in SHAPES:
        with _converged(P, o, v, X, seed, tier) as s:
            w, _ = s.ipeom(4, tol=1e-9)
            ref.append(np.sort_complex(w))
    systems = [_converged(P, *sh, tier) for sh in SHAPES]
    try:
        w, r1, it, status = P.batch_ipeom(systems, 4, tol=1e-9)
    finally:
        for s in systems:
            s.close()
    assert np.all(status == 0)
    tol = 1e-10 if tier == "fp64" else 1e-8
    for q in range(len(SHAPES)):
        assert np.abs(np.sort_complex(w[q]) - ref[q]).max() <= tol
    assert np.all((r1 > 0) & (r1 <= 1 + 1e-9))


def test_graph_replay_matches_direct():
    P = _gpu()
    out = []
    for graphs in (False, True):
        with _converged(P, 8, 30, 90, 4, "tf32x3") as s:
            s.set_graphs(graphs)
            w, _ = s.ipeom(6, tol=1e-9)
            out.append(np.sort_complex(w))
    assert np.abs(out[0] - out[1]).max() <= 1e-9


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
