"""cc_zgemm_noalloc: the complex GEMM for callers that cannot allocate.

Callers capturing a stream into a CUDA graph, or running inside a framework
that owns all device memory, cannot let a library call cudaMalloc. The
no-allocation entry point keeps its temporaries in a fixed device array;
this checks through the C ABI that two calls in a row give what the
allocating entry point (cc_zgemm_dev) gives, within the tolerances of the
parity tests, that the second call leaves free device memory unchanged, and
that a problem too large for the fixed array is refused. Collected last so a
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


@pytest.mark.parametrize("tier", ["fp64", "tf32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("M,N,K", [(200, 300, 517), (64, 1000, 96)])
def test_noalloc_matches_allocating_gemm(tier, M, N, K):
    P = _lib()
    rng = np.random.default_rng(M + N + K)
    A = torch.from_numpy(rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).cuda()
    B = torch.from_numpy(rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))).cuda()
    ref = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    P.zgemm_dev(A, B, ref, tier)
    torch.cuda.synchronize()
    scale = ref.abs().max().item()
    for call in range(2):
        out = torch.full((M, N), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        P.zgemm_noalloc(A, B, out, tier)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        err = (out - ref).abs().max().item() / scale
        assert err <= REL[tier], (call, err)
        if call == 1:
            assert free1 == free0


def test_noalloc_rejects_oversize():
    P = _lib()
    t = P.TIERS["tf32x3"]
    A = torch.zeros((4096, 8), dtype=torch.complex128, device="cuda")
    rc = P.lib().cc_zgemm_noalloc(t, 4096, 4096, 4096, ctypes.c_void_p(A.data_ptr()),
                                  ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()))
    assert rc == -1
    assert b"scratch" in P.lib().cc_last_error(None)
