"""Error paths of the library on a live device, exercised without any GPU
fault: the failure is made on the host (an injected NaN copied into device
memory between kernels, a context that never ran CCSD, an iteration limit)
or by a bounded device wait that a test shortens until it runs out. After
each failure the same context must still give the oracle's results."""
import ctypes

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


def _inputs(o, v, X, seed, scale=4.0):
    rng = np.random.default_rng(seed)
    eps = synth.make_eps(rng, o, v)
    L = synth.make_cholesky(rng, o + v, X) * scale
    return eps, L


def _oracle(eps, L, o, n_roots):
    from oracle import ccsd, integrals, ipeom
    g = integrals.blocks_from_cholesky(L, o)
    res = ccsd.solve(g, eps, tol=1e-12, max_iter=300)
    assert res["converged"]
    H = ipeom.hbar(g, eps, res["t1"], res["t2"])
    w, _ = ipeom.dense_roots(H, o, L.shape[1] - o, n_roots)
    return res["e_corr"], w


def test_wait_limit_expires_then_context_recovers():
    """A tensor-core wait limit of 1 ns makes the first pipeline wait that
    does not succeed at once run out: the kernel drains its copies and MMAs,
    frees TMEM and returns, and the call fails with CC_ERR_TIMEOUT. With the
    limit restored the same context computes the ladder as before."""
    P = _gpu()
    o, v, X = 6, 40, 64
    eps, L = _inputs(o, v, X, 3)
    rng = np.random.default_rng(0)
    tau = (rng.standard_normal((o, o, v, v)) + 1j * rng.standard_normal((o, o, v, v))) * 1e-2
    tau = tau - tau.transpose(1, 0, 2, 3)
    tau = tau - tau.transpose(0, 1, 3, 2)
    td = torch.from_numpy(tau).cuda()
    with P.System(eps, L, n_occ=o, tier="fp16") as s:
        ref = torch.zeros_like(td)
        s.ladder_dev(td, ref)
        torch.cuda.synchronize()
        out = torch.zeros_like(td)
        P.set_wait_limit(1)
        try:
            with pytest.raises(P.CCError) as e:
                s.ladder_dev(td, out)
                torch.cuda.synchronize()
            assert e.value.code == -7
        finally:
            P.set_wait_limit(0)
        again = torch.zeros_like(td)
        s.ladder_dev(td, again)
        torch.cuda.synchronize()
    r, a = ref.cpu().numpy(), again.cpu().numpy()
    assert np.abs(a - r).max() <= 1e-12 * np.abs(r).max()


def test_nan_in_ccsd_residual_is_reported_then_recovers():
    P = _gpu()
    o, v, X = 6, 20, 60
    eps, L = _inputs(o, v, X, 1)
    e_ref, _ = _oracle(eps, L, o, 2)
    with P.System(eps, L, n_occ=o, tier="fp64") as s:
        s.set_fault_injection(1, at_iteration=2)
        with pytest.raises(P.CCError) as e:
            s.ccsd(tol=1e-10)
        assert e.value.code == -6
        s.reset_amplitudes()
        e = s.ccsd(tol=1e-10)
    assert abs(e - e_ref) <= 1e-9


def test_iteration_limit_reports_not_converged_with_results():
    P = _gpu()
    o, v, X = 6, 20, 60
    eps, L = _inputs(o, v, X, 1)
    e_ref, w_ref = _oracle(eps, L, o, 3)
    with P.System(eps, L, n_occ=o, tier="fp64") as s:
        e = np.zeros(2)
        it = ctypes.c_int()
        rc = P.lib().ccsd_solve(s._ctx, 1e-10, 1, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.byref(it))
        assert rc == -5 and it.value == 1
        assert np.all(np.isfinite(e)) and e[0] < 0   # the first iterate was written
        assert abs(complex(e[0], e[1]) - e_ref) < 0.2 * abs(e_ref)
        ec = s.ccsd(tol=1e-10)          # continues from the written amplitudes
        assert abs(ec - e_ref) <= 1e-9
        w, _ = s.ipeom(3, tol=1e-6, max_iter=1, allow_unconverged=True)
        assert s.davidson_iterations == 1 and np.all(np.isfinite(w))
        w, _ = s.ipeom(3, tol=1e-9)
    assert np.abs(np.sort_complex(w) - np.sort_complex(w_ref)).max() <= 1e-9


SHAPES = [(6, 20, 60, 1), (8, 26, 80, 2), (5, 31, 50, 3)]


@pytest.mark.parametrize("bad", ["no_ccsd", "nan_sigma"])
def test_batch_isolates_a_failed_system(bad):
    """One system of the batch fails on its own (never ran CCSD, or its
    Davidson residual turns NaN); it reports its own status and the other
    systems' roots still equal the oracle's."""
    P = _gpu()
    refs = [_oracle(*_inputs(o, v, X, seed), o, 4)[1] for o, v, X, seed in SHAPES]
    systems = []
    try:
        for q, (o, v, X, seed) in enumerate(SHAPES):
            eps, L = _inputs(o, v, X, seed)
            s = P.System(eps, L, n_occ=o, tier="fp64", eom_tier="fp64")
            if not (q == 1 and bad == "no_ccsd"):
                s.ccsd(tol=1e-11)
            if q == 1 and bad == "nan_sigma":
                s.set_fault_injection(2, at_iteration=2)
            systems.append(s)
        w, r1, it, status = P.batch_ipeom(systems, 4, tol=1e-9, allow_unconverged=True)
    finally:
        for s in systems:
            s.close()
    assert status[1] == (-8 if bad == "no_ccsd" else -6)
    for q in (0, 2):
        assert status[q] == 0
        assert np.abs(np.sort_complex(w[q]) - np.sort_complex(refs[q])).max() <= 1e-9


def test_batch_solve_matches_oracle():
    """cc_batch_solve: CCSD and batched IP-EOM for uneven systems, each
    system's energy and IPs against the oracle."""
    P = _gpu()
    systems = []
    try:
        for o, v, X, seed in SHAPES:
            eps, L = _inputs(o, v, X, seed)
            systems.append(P.System(eps, L, n_occ=o, tier="tf32x3", eom_tier="tf32x3"))
        e, w, r1, status = P.batch_solve(systems, 4, ccsd_tol=1e-10, eom_tol=1e-9)
    finally:
        for s in systems:
            s.close()
    assert np.all(status == 0)
    # TF32x3 tolerances of the end-to-end tests (the split tier's FP32-class
    # accumulation leaves ~1e-6 relative in E_corr)
    for q, (o, v, X, seed) in enumerate(SHAPES):
        e_ref, w_ref = _oracle(*_inputs(o, v, X, seed), o, 4)
        assert abs(e[q] - e_ref) <= 1e-7
        assert np.abs(np.sort_complex(w[q]) - np.sort_complex(w_ref)).max() <= 1e-7


def test_per_context_allocator():
    """A context's own allocator serves its later allocations; buffers it
    held before are released through the functions that made them."""
    P = _gpu()
    o, v, X = 6, 20, 60
    eps, L = _inputs(o, v, X, 1)
    e_ref, w_ref = _oracle(eps, L, o, 3)
    live = {}
    count = {"alloc": 0, "free": 0}

    def alloc(n, _user):
        t = torch.empty(int(n), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        count["alloc"] += 1
        return t.data_ptr()

    def free(p, _user):
        live.pop(p)
        count["free"] += 1

    with P.System(eps, L, n_occ=o, tier="fp64") as s:
        s.set_allocator(alloc, free)
        e = s.ccsd(tol=1e-10)
        w, _ = s.ipeom(3, tol=1e-9)
        assert count["alloc"] > 0
    assert count["free"] == count["alloc"] and not live
    assert abs(e - e_ref) <= 1e-9
    assert np.abs(np.sort_complex(w) - np.sort_complex(w_ref)).max() <= 1e-9
