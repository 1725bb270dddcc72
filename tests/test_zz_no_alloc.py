"""cc_zgemm_noalloc: the complex GEMM for callers that cannot allocate.

Some callers cannot let a library call cudaMalloc: a framework that has
reserved nearly all device memory for its own pool, an application whose
device-memory budget is fixed at start-up, or a latency-critical loop where
an allocation would synchronise the device. The no-allocation entry point
keeps its temporaries in a fixed device array. These tests check, through
the C ABI, that two calls in a row give what the allocating entry point
(cc_zgemm_dev) gives and what numpy gives, within the tolerances of the
parity tests; that the second call leaves free device memory unchanged;
that the tile autotuner is not run for it; and that the FP16 tiers,
problems too large for the fixed array and sizes whose byte counts overflow
are refused with CC_ERR_ARG and a message. Collected last, so a
stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# same bounds as the parity tests (relative to max |C|)
REL = {"fp64": 1e-12, "tf32": 4e-3, "tf32x3": 2e-6, "bf16x3": 1e-4}


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_06805_gb300 as P
    P.lib()
    return P


def _operands(M, N, K, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    return A, B


@pytest.mark.parametrize("tier", ["fp64", "tf32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("M,N,K", [(200, 300, 517), (64, 1000, 96)])
def test_noalloc_matches_allocating_gemm(tier, M, N, K):
    P = _lib()
    A, B = _operands(M, N, K, M + N + K)
    exact = A @ B.T
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ref = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    P.zgemm_dev(Ad, Bd, ref, tier)
    torch.cuda.synchronize()
    scale = np.abs(exact).max()
    for call in range(2):
        out = torch.full((M, N), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        P.zgemm_noalloc(Ad, Bd, out, tier)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        got = out.cpu().numpy()
        err_dev = np.abs(got - ref.cpu().numpy()).max() / scale
        err_np = np.abs(got - exact).max() / scale
        assert err_dev <= REL[tier], (call, err_dev)
        assert err_np <= REL[tier], (call, err_np)
        if call == 1:
            assert free1 == free0


def test_noalloc_never_runs_the_autotuner(tmp_path, monkeypatch):
    """With the autotuner switched on and a shape it has not seen, the call
    still allocates nothing: the tuner (which times candidates on a scratch
    output) is skipped, so no choice is recorded in its cache file."""
    P = _lib()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("CDFNS_AUTOTUNE", "1")
    monkeypatch.setenv("CDFNS_TUNE_CACHE", str(cache))
    M, N, K = 136, 712, 333  # a shape bucket no other test uses
    A, B = _operands(M, N, K, 7)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    P.zgemm_noalloc(Ad, Bd, out, "tf32x3")
    torch.cuda.synchronize()
    exact = A @ B.T
    assert np.abs(out.cpu().numpy() - exact).max() / np.abs(exact).max() <= REL["tf32x3"]
    assert not cache.exists()


@pytest.mark.parametrize("tier", ["fp16", "fp16x3"])
def test_noalloc_rejects_fp16_tiers(tier):
    P = _lib()
    A = torch.zeros((8, 8), dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(A.data_ptr())
    rc = P.lib().cc_zgemm_noalloc(P.TIERS[tier], 8, 8, 8, p, p, p)
    assert rc == -1
    assert b"FP16" in P.lib().cc_last_error(None)


def test_noalloc_rejects_oversize():
    P = _lib()
    t = P.TIERS["tf32x3"]
    A = torch.zeros((4096, 8), dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(A.data_ptr())
    rc = P.lib().cc_zgemm_noalloc(t, 4096, 4096, 4096, p, p, p)
    assert rc == -1
    assert b"scratch" in P.lib().cc_last_error(None)


@pytest.mark.parametrize("tier", ["fp64", "tf32"])
def test_noalloc_rejects_overflowing_sizes(tier):
    """Sizes whose byte counts do not fit in a long are refused on the host,
    before any device work (the pointers are never dereferenced)."""
    P = _lib()
    A = torch.zeros((8, 8), dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(A.data_ptr())
    for M, N, K in ((1 << 62, 8, 8), (8, 1 << 62, 8), (8, 8, 1 << 62), (1 << 31, 1 << 31, 8)):
        rc = P.lib().cc_zgemm_noalloc(P.TIERS[tier], M, N, K, p, p, p)
        assert rc == -1, (M, N, K)
        assert b"too large" in P.lib().cc_last_error(None) or \
            b"scratch" in P.lib().cc_last_error(None)
