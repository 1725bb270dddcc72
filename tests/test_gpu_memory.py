"""CCSD under a cap on the context's device memory (cc_set_memory_limit).

Without a cap (and with a roomy device) ccsd_solve holds a DIIS history of
up to 8 pairs of packed vectors, caches the packed planes of the stable
operands and keeps a permuted copy of <mb||ej>. Under a cap it keeps the
residual's transient buffers allocatable first and shrinks the rest: the
converged energy must not change beyond the tolerance, the context must
never hold more than the cap, and a cap below what the iteration itself
needs must end in CC_ERR_OOM, not a fault.
"""
import pytest

from paper_2506_06805_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_06805_gb300 as P
    P.lib()
    return P


def _tiny(scale):
    c, eps, L = synth.make_config("tiny")
    o, v = c.n_occ, c.n_virt
    na = o * v + o * (o - 1) // 2 * (v * (v - 1) // 2)
    return c, eps, L * scale, 2 * 16 * na  # one DIIS pair: two complex128 vectors


def _run(P, c, eps, L, tier, cap=0):
    """CCSD with the cap set once the integrals are built (dump_integrals
    builds them), so that it bounds the iterations."""
    with P.System(eps, L, n_occ=c.n_occ, tier=tier) as s:
        s.dump_integrals(0)
        if cap:
            s.set_memory_limit(cap)
        e = s.ccsd(tol=TOL, max_iter=200)
        return e, s.stats(), s.ccsd_iterations


def test_diis_history_follows_memory_cap():
    """FP64 tier, tiny workload with its Cholesky vectors scaled by 5: strong
    enough correlation that CCSD takes 9 iterations in the oracle, so the
    DIIS history reaches 7 pairs when memory is no object."""
    P = _gpu()
    c, eps, L, pair = _tiny(5.0)
    e0, st0, it0 = _run(P, c, eps, L, "fp64")
    d0 = int(st0["diis_depth"])
    assert d0 == min(8, it0 - 2)
    assert d0 >= 4, f"only {it0} iterations: too few to cap the DIIS history"
    # 1) cap at the uncapped iterations' high-water mark: the permuted copy
    # is out of reach (its reserve is not), the history still fits
    cap1 = int(st0["ccsd_loop_peak_bytes"])
    e1, st1, _ = _run(P, c, eps, L, "fp64", cap1)
    assert st1["ccsd_loop_peak_bytes"] <= cap1
    d1 = int(st1["diis_depth"])
    assert d1 >= 3
    assert abs(e1 - e0) < 100 * TOL
    # 2) room for two pairs beyond what run 1 held without its history, with
    # half a pair to spare
    cap2 = int(st1["ccsd_loop_peak_bytes"]) - d1 * pair + 2 * pair + pair // 2
    e2, st2, _ = _run(P, c, eps, L, "fp64", cap2)
    assert st2["ccsd_loop_peak_bytes"] <= cap2
    assert int(st2["diis_depth"]) == 2
    assert abs(e2 - e0) < 100 * TOL
    # 3) no room for the iteration itself: a clean CC_ERR_OOM
    with P.System(eps, L, n_occ=c.n_occ, tier="fp64") as s:
        s.dump_integrals(0)
        s.set_memory_limit(int(s.stats()["device_bytes_held"]) + pair)
        with pytest.raises(P.CCError) as ei:
            s.ccsd(tol=TOL)
        assert ei.value.code == -3  # CC_ERR_OOM


def test_operands_packed_on_each_use_under_cap():
    """FP16 tier, tiny workload: under a cap the stable operands' packed
    planes are not cached but packed again on each use from the same data,
    with the same scales, so the iterations and the energy are unchanged."""
    P = _gpu()
    c, eps, L, pair = _tiny(1.0)
    e0, st0, it0 = _run(P, c, eps, L, "fp16")
    cap = int(st0["ccsd_loop_peak_bytes"])
    e1, st1, it1 = _run(P, c, eps, L, "fp16", cap)
    assert st1["ccsd_loop_peak_bytes"] <= cap
    assert it1 == it0
    assert abs(e1 - e0) < 1e-12
    with P.System(eps, L, n_occ=c.n_occ, tier="fp16") as s:
        s.dump_integrals(0)
        s.set_memory_limit(int(s.stats()["device_bytes_held"]) + pair)
        with pytest.raises(P.CCError) as ei:
            s.ccsd(tol=TOL)
        assert ei.value.code == -3  # CC_ERR_OOM


def test_memory_cap_below_holdings_rejected():
    P = _gpu()
    c, eps, L = synth.make_config("tiny")
    with P.System(eps, L, n_occ=c.n_occ, tier="fp16") as s:
        with pytest.raises(P.CCError) as ei:
            s.set_memory_limit(1024)
        assert ei.value.code == -1  # CC_ERR_ARG: below the bytes already held
        s.set_memory_limit(0)
        s.ccsd(tol=1e-8)
