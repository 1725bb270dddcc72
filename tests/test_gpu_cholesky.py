"""Single-step pivoted Cholesky decomposition (Eq. 21) through the C ABI
against the oracle.

The pivots are integer decisions taken on FP64 diagonals on both sides; the
seeded generators below keep the two largest remaining diagonals at least
2e-6 apart (relative) at every step, far above the rounding differences of
the two evaluation orders, so the pivot sequences must agree exactly. The
vectors agree to rounding. Past the rank of M, where the remaining diagonals
are rounding noise, only the count and the error bound are compared.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_06805_gb300 as P
    P.lib()
    return P


def _generator(N, r, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))) / np.sqrt(2 * r)


@pytest.mark.parametrize("N,r,tau,max_vec,seed", [(2000, 300, 1e-6, 120, 11),
                                                  (300000, 40, 0.0, 24, 12)])
def test_pivoted_cholesky_matches_oracle(N, r, tau, max_vec, seed):
    """A ragged N over 8 blocks, and N = 300000 over 1024 grid-striding
    argmax blocks."""
    P = _gpu()
    from oracle import cholesky
    B = _generator(N, r, seed)
    L_ref, piv_ref = cholesky.pivoted_cholesky(B, tau, max_vec=max_vec)
    Ld, piv = P.cholesky_dev(torch.from_numpy(B).cuda(), tau, max_vec)
    L = Ld.cpu().numpy()
    assert np.array_equal(piv, piv_ref)
    assert np.abs(L - L_ref).max() <= 1e-11 * np.abs(L_ref).max()


def test_pivoted_cholesky_stops_at_rank_within_tau():
    P = _gpu()
    N, r, tau = 2000, 60, 1e-8
    B = _generator(N, r, 13)
    Ld, piv = P.cholesky_dev(torch.from_numpy(B).cuda(), tau, 80)
    L = Ld.cpu().numpy()
    assert L.shape[0] == r
    M = B @ B.conj().T
    assert np.abs(M - L.T @ L.conj()).max() < tau
    # a threshold above every diagonal element forms no vector
    Ld, piv = P.cholesky_dev(torch.from_numpy(B).cuda(), 10.0, 8)
    assert Ld.shape[0] == 0 and len(piv) == 0
