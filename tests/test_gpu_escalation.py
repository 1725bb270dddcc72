"""CCSD in a one-product tier moves to its split form when the step norm
stalls above the tolerance.

The tiny workload with its Cholesky vectors scaled by 5 is strongly
correlated (E_corr = -0.044 Eh, 9-10 CCSD iterations in FP64): there the
FP16 residual's rounding keeps ||dt|| above 1e-7, so a 1e-9 target is out of
its reach. ccsd_solve then finishes in FP16x3; at the unscaled workload it
never has to.
"""
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


def _solve(P, c, eps, L, tier, tol, roots=0):
    eom = "fp64" if tier == "fp64" else "fp16x3"
    with P.System(eps, L, n_occ=c.n_occ, tier=tier, eom_tier=eom) as s:
        e = s.ccsd(tol=tol, max_iter=100)
        w = s.ipeom(roots, tol=1e-8)[0] if roots else None
        return e, w, s.stats()


def test_stalled_fp16_ccsd_finishes_in_fp16x3():
    P = _gpu()
    c, eps, L = synth.make_config("tiny")
    L = 5.0 * L
    e64, w64, _ = _solve(P, c, eps, L, "fp64", 1e-11, roots=4)
    e16, w16, st16 = _solve(P, c, eps, L, "fp16", 1e-9, roots=4)
    ex3, _, stx3 = _solve(P, c, eps, L, "fp16x3", 1e-9)
    assert st16["ccsd_escalated_at"] > 0
    assert stx3["ccsd_escalated_at"] == 0  # already the split tier
    # the same fixed point as FP16x3 throughout, and FP64 within the split
    # tier's own distance (6.7e-8 Eh at this coupling strength)
    assert abs(e16 - ex3) < 1e-8
    assert abs(e16 - e64) < 2e-7
    assert np.abs(np.sort_complex(w16) - np.sort_complex(w64)).max() < 1e-6


def test_converging_fp16_ccsd_stays_fp16():
    P = _gpu()
    c, eps, L = synth.make_config("tiny")
    _, _, st = _solve(P, c, eps, L, "fp16", 1e-9)
    assert st["ccsd_escalated_at"] == 0
