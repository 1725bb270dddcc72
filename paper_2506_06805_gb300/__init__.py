"""GB300 CD/FNS IP-EOM-CCSD: Python binding of libcdfns.so.

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``libcdfns.so`` (declared in ``include/cdfns.h``). PyTorch
supplies device memory (its caching allocator serves the library's
workspace) and the CUDA stream. There is no CPU fallback: importing
:func:`lib` without the built library, or calling it without a GPU, raises.

Typical use::

    from paper_2506_06805_gb300 import System, synth
    eps, L = synth.make_system(40, 300, 1200, kramers=True)
    with System(eps, L, n_occ=40, tier="tf32") as s:
        e = s.ccsd(tol=1e-8)
        w, r1w = s.ipeom(8, tol=1e-7)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["lib", "System", "Mlp", "CCError", "TIERS", "LIB_PATH"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcdfns.so")

TIERS = {"fp64": 0, "tf32": 1, "tf32x3": 2, "bf16x3": 3, "fp16": 4, "fp16x3": 5}
_ERRORS = {
    -1: "CC_ERR_ARG", -2: "CC_ERR_INPUT", -3: "CC_ERR_OOM", -4: "CC_ERR_CUDA",
    -5: "CC_ERR_NOT_CONVERGED", -6: "CC_ERR_NUMERIC", -7: "CC_ERR_TIMEOUT",
    -8: "CC_ERR_STATE", -9: "CC_ERR_UNSUPPORTED",
}

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_SIGS = {
    "cc_set_default_allocator": (ctypes.c_int, [_ALLOC, _FREE, _P]),
    "cc_set_default_stream": (ctypes.c_int, [_P]),
    "cc_init": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                               ctypes.POINTER(_P)]),
    "cc_init_chunked": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _D, ctypes.POINTER(_P)]),
    "cc_add_cholesky": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _D]),
    "cc_add_cholesky_dev": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "cc_set_precision": (ctypes.c_int, [_P, ctypes.c_int]),
    "cc_set_precision_eom": (ctypes.c_int, [_P, ctypes.c_int]),
    "cc_set_stream": (ctypes.c_int, [_P, _P]),
    "cc_set_slab_budget": (ctypes.c_int, [_P, ctypes.c_size_t]),
    "cc_get_sizes": (ctypes.c_int, [_P, _I, _I, _I]),
    "fns_truncate": (ctypes.c_int, [_P, ctypes.c_double, _I]),
    "fns_truncate_count": (ctypes.c_int, [_P, ctypes.c_int]),
    "fns_get_occupations": (ctypes.c_int, [_P, _D, ctypes.c_int]),
    "ccsd_solve": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, _D, _I]),
    "ipeom_solve": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                   _D, _D, _I]),
    "cc_get_amplitudes": (ctypes.c_int, [_P, _D, _D]),
    "cc_set_amplitudes": (ctypes.c_int, [_P, _D, _D]),
    "cc_reset_amplitudes": (ctypes.c_int, [_P]),
    "cc_ladder_dev": (ctypes.c_int, [_P, _P, _P]),
    "cc_residual_dev": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ipeom_sigma_dev": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "ipeom_left_sigma_dev": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "cc_cholesky_dev": (ctypes.c_int, [ctypes.c_long, ctypes.c_int, _P, ctypes.c_double,
                                       ctypes.c_int, _P, ctypes.POINTER(ctypes.c_long), _I]),
    "ipeom_solve_lr": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      _D, _D, _D, _D, _I]),
    "cc_dump_integrals": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "cc_selftest_conversions": (ctypes.c_int, [_P, ctypes.c_long,
                                               ctypes.POINTER(ctypes.c_longlong)]),
    "cc_zgemm_dev": (ctypes.c_int, [ctypes.c_int, ctypes.c_long, ctypes.c_long,
                                    ctypes.c_long, _P, _P, _P]),
    "cc_zgemm_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_long, ctypes.c_long,
                                        ctypes.c_long, _P, _P, _P]),
    "cc_get_stats": (ctypes.c_int, [_P, _D, ctypes.c_int]),
    "cc_last_error": (ctypes.c_char_p, [_P]),
    "cc_mlp_num_params": (ctypes.c_int, []),
    "cc_mlp_create": (ctypes.c_int, [ctypes.POINTER(_P)]),
    "cc_mlp_free": (None, [_P]),
    "cc_mlp_last_error": (ctypes.c_char_p, [_P]),
    "cc_mlp_set_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "cc_mlp_get_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "cc_mlp_add_samples": (ctypes.c_int, [_P, _P, ctypes.c_long]),
    "cc_mlp_num_samples": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_long)]),
    "cc_mlp_train": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_int), ctypes.c_long, _D]),
    "cc_mlp_loss_grad": (ctypes.c_int, [_P, ctypes.c_long, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float), _D,
                                        ctypes.POINTER(ctypes.c_float)]),
    "cc_mlp_features": (ctypes.c_int, [_P, ctypes.c_long, ctypes.POINTER(ctypes.c_float)]),
    "cc_mlp_warm_start": (ctypes.c_int, [_P, _P]),
    "cc_free": (None, [_P]),
    "cc_set_graphs": (ctypes.c_int, [_P, ctypes.c_int]),
    "cc_set_memory_limit": (ctypes.c_int, [_P, ctypes.c_size_t]),
    "cc_batch_ipeom": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, _D, _D, _I, _I]),
    "cc_batch_solve": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      _D, _D, _D, _I]),
    "cc_set_allocator": (ctypes.c_int, [_P, _ALLOC, _FREE, _P]),
    "cc_set_wait_limit": (ctypes.c_int, [ctypes.c_ulonglong]),
    "cc_set_fault_injection": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "cc_set_davidson_guess": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "cc_begin_fns_stream": (ctypes.c_int, [_P]),
    "fns_stream_truncate": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, _I]),
    "ipeom_guess_dev": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "cc_mlp_guess_features": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_long,
                                             ctypes.POINTER(ctypes.c_float)]),
    "cc_mlp_add_guess_samples": (ctypes.c_int, [_P, _P, ctypes.c_long]),
}

_lib = None


class CCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


def header_symbols():
    """Function names declared in include/cdfns.h."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(LIB_PATH)), "include",
                       "cdfns.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(c[c]?_\w+|fns_\w+|ccsd_\w+|ipeom_\w+)\s*\(",
                                 text, re.M)))


def lib():
    """Load libcdfns.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(_D)


def _check(rc, ctx=None, ok=(0,)):
    if rc not in ok:
        msg = lib().cc_last_error(ctx)
        raise CCError(rc, msg.decode() if msg else "")
    return rc


_TORCH_HOOKS = None


def use_torch_memory():
    """Route the library's device allocations through PyTorch's caching
    allocator and issue its work on torch's current stream."""
    global _TORCH_HOOKS
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required")
    dev = torch.cuda.current_device()

    def _alloc(n, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(n), dev)
        except RuntimeError:
            return None

    def _free(p, _user):
        torch.cuda.caching_allocator_delete(p)

    hooks = (_ALLOC(_alloc), _FREE(_free))
    _check(lib().cc_set_default_allocator(hooks[0], hooks[1], None))
    _check(lib().cc_set_default_stream(torch.cuda.current_stream().cuda_stream))
    _TORCH_HOOKS = hooks


def zgemm_dev(A, B, C, tier="fp64"):
    """C[m][n] = sum_k A[m][k] B[n][k] on device tensors (complex128)."""
    t = TIERS[tier] if isinstance(tier, str) else int(tier)
    M, K = A.shape
    N = B.shape[0]
    _check(lib().cc_zgemm_dev(t, M, N, K, _P(A.data_ptr()), _P(B.data_ptr()),
                              _P(C.data_ptr())))


def batch_ipeom(systems, n_roots, tol=1e-7, max_iter=100, allow_unconverged=False):
    """IP-EOM roots of several systems with batched sigma builds.

    Returns (omega [n_sys][n_roots] complex, r1_weight, n_iter, status)."""
    n = len(systems)
    arr = (_P * n)(*[s._ctx for s in systems])
    w = np.zeros((n, n_roots, 2))
    r1 = np.zeros((n, n_roots))
    it = np.zeros(n, np.int32)
    stt = np.zeros(n, np.int32)
    rc = lib().cc_batch_ipeom(arr, n, n_roots, tol, max_iter, _dptr(w), _dptr(r1),
                              it.ctypes.data_as(_I), stt.ctypes.data_as(_I))
    _check(rc, systems[0]._ctx, (0, -5) if allow_unconverged else (0,))
    return w[..., 0] + 1j * w[..., 1], r1, it, stt


def batch_solve(systems, n_roots, ccsd_tol=1e-8, eom_tol=1e-7, max_iter=100):
    """CCSD then batched IP-EOM for several systems (cc_batch_solve).

    Returns (e_corr [n_sys] complex, omega [n_sys][n_roots] complex,
    r1_weight, status [n_sys]); a failed system has a nonzero status and
    does not affect the others."""
    n = len(systems)
    arr = (_P * n)(*[s._ctx for s in systems])
    e = np.zeros((n, 2))
    w = np.zeros((n, n_roots, 2))
    r1 = np.zeros((n, n_roots))
    stt = np.zeros(n, np.int32)
    rc = lib().cc_batch_solve(arr, n, n_roots, ccsd_tol, eom_tol, max_iter, _dptr(e),
                              _dptr(w), _dptr(r1), stt.ctypes.data_as(_I))
    _check(rc, systems[0]._ctx, (0, -5))
    return e[:, 0] + 1j * e[:, 1], w[..., 0] + 1j * w[..., 1], r1, stt


def set_wait_limit(ns):
    """Limit (ns) of the tensor-core kernels' pipeline waits, process-wide
    (0: the default 2 s). A test hook for the timeout path."""
    _check(lib().cc_set_wait_limit(int(ns)))


def selftest_conversions(x):
    """Mismatch counts (narrowing, widening) of the library's integer-pipe
    FP64/FP32 conversions against the hardware ones over a device float64
    tensor x."""
    out = (ctypes.c_longlong * 2)()
    _check(lib().cc_selftest_conversions(_P(x.data_ptr()), x.numel(), out))
    return int(out[0]), int(out[1])


def cholesky_dev(B, tau, max_vec):
    """Single-step pivoted Cholesky vectors (Eq. 21) of M = B B^H for a
    device complex128 tensor B [N][r]. Returns (L [n][N] on the device,
    pivots [n])."""
    import torch
    N, r = B.shape
    L = torch.empty((max_vec, N), dtype=torch.complex128, device=B.device)
    piv = np.zeros(max_vec, dtype=np.int64)
    n = ctypes.c_int()
    _check(lib().cc_cholesky_dev(N, r, _P(B.data_ptr()), float(tau), int(max_vec),
                                 _P(L.data_ptr()),
                                 piv.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                 ctypes.byref(n)))
    return L[:n.value], piv[:n.value]


def zgemm_noalloc(A, B, C, tier="fp64"):
    """Same product as zgemm_dev with every temporary in the library's fixed
    device scratch array: no device allocation, for callers whose device
    memory is owned by a framework pool or fixed at start-up. Calls share
    the array and must not overlap on the GPU."""
    t = TIERS[tier] if isinstance(tier, str) else int(tier)
    M, K = A.shape
    N = B.shape[0]
    _check(lib().cc_zgemm_noalloc(t, M, N, K, _P(A.data_ptr()), _P(B.data_ptr()),
                                  _P(C.data_ptr())))


class System:
    """One system: orbital energies eps[n] and Cholesky vectors L[X][n][n]."""

    def __init__(self, eps, L=None, n_occ=None, n_aux=None, tier="fp64",
                 eom_tier=None, torch_memory=True, chunks=None):
        if torch_memory and _TORCH_HOOKS is None:
            use_torch_memory()
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        n = eps.shape[0]
        if n_occ is None:
            n_occ = int(np.count_nonzero(eps < 0))
        self.n_occ = n_occ
        self._ctx = _P()
        if L is not None:
            L = np.ascontiguousarray(L, dtype=np.complex128)
            X = L.shape[0]
            if L.shape != (X, n, n):
                raise ValueError("L must be [n_aux][n][n]")
            rc = lib().cc_init(n_occ, n - n_occ, X, _dptr(eps),
                               L.view(np.float64).ctypes.data_as(_D),
                               ctypes.byref(self._ctx))
        else:
            X = n_aux
            rc = lib().cc_init_chunked(n_occ, n - n_occ, X, _dptr(eps),
                                       ctypes.byref(self._ctx))
            if rc == 0 and chunks is not None:
                for p0, p1, Lc in chunks:
                    Lc = np.ascontiguousarray(Lc, dtype=np.complex128)
                    _check(lib().cc_add_cholesky(self._ctx, p0, p1,
                                                 Lc.view(np.float64).ctypes.data_as(_D)),
                           self._ctx)
        _check(rc, None)
        self.set_precision(tier, eom_tier)

    # ---- lifecycle ----
    def close(self):
        if self._ctx:
            lib().cc_free(self._ctx)
            self._ctx = _P()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- configuration ----
    def set_precision(self, tier, eom_tier=None):
        t = TIERS[tier] if isinstance(tier, str) else int(tier)
        _check(lib().cc_set_precision(self._ctx, t), self._ctx)
        if eom_tier is not None:
            e = TIERS[eom_tier] if isinstance(eom_tier, str) else int(eom_tier)
            _check(lib().cc_set_precision_eom(self._ctx, e), self._ctx)

    def set_stream(self, stream_handle):
        _check(lib().cc_set_stream(self._ctx, _P(stream_handle)), self._ctx)

    def set_slab_budget(self, nbytes):
        _check(lib().cc_set_slab_budget(self._ctx, int(nbytes)), self._ctx)

    def sizes(self):
        o, v, x = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().cc_get_sizes(self._ctx, ctypes.byref(o), ctypes.byref(v),
                                  ctypes.byref(x)), self._ctx)
        return o.value, v.value, x.value

    def add_cholesky(self, p0, p1, Lc):
        """Cholesky vectors P in [p0, p1): a numpy array (host) or a
        contiguous torch complex128 CUDA tensor (device), [p1-p0][n][n]."""
        if hasattr(Lc, "is_cuda") and Lc.is_cuda:
            _check(lib().cc_add_cholesky_dev(self._ctx, p0, p1, _P(Lc.data_ptr())), self._ctx)
            return
        Lc = np.ascontiguousarray(Lc, dtype=np.complex128)
        _check(lib().cc_add_cholesky(self._ctx, p0, p1,
                                     Lc.view(np.float64).ctypes.data_as(_D)), self._ctx)

    # ---- solvers ----
    def fns_truncate(self, threshold=None, n_keep=None):
        if n_keep is not None:
            _check(lib().fns_truncate_count(self._ctx, int(n_keep)), self._ctx)
            return self.sizes()[1]
        kept = ctypes.c_int()
        _check(lib().fns_truncate(self._ctx, float(threshold), ctypes.byref(kept)),
               self._ctx)
        return kept.value

    def fns_stream(self, chunks, threshold=None, n_keep=None):
        """Streamed natural spinors (cc_begin_fns_stream) on a system made
        with L=None: chunks() must return a fresh iterable of (p0, p1, L_chunk)
        covering every P; it is consumed twice. Returns the kept count."""
        _check(lib().cc_begin_fns_stream(self._ctx), self._ctx)
        for p0, p1, Lc in chunks():
            self.add_cholesky(p0, p1, Lc)
        kept = ctypes.c_int()
        _check(lib().fns_stream_truncate(self._ctx, float(threshold if threshold is not None else 0.0),
                                         int(n_keep or 0), ctypes.byref(kept)), self._ctx)
        for p0, p1, Lc in chunks():
            self.add_cholesky(p0, p1, Lc)
        return kept.value

    def fns_occupations(self, n):
        out = np.empty(n)
        _check(lib().fns_get_occupations(self._ctx, _dptr(out), n), self._ctx)
        return out

    def ccsd(self, tol=1e-8, max_iter=100, allow_unconverged=False):
        e = np.zeros(2)
        it = ctypes.c_int()
        ok = (0, -5) if allow_unconverged else (0,)
        _check(lib().ccsd_solve(self._ctx, tol, max_iter, _dptr(e), ctypes.byref(it)),
               self._ctx, ok)
        self.ccsd_iterations = it.value
        return complex(e[0], e[1])

    def ipeom(self, n_roots, tol=1e-7, max_iter=100, allow_unconverged=False):
        w = np.zeros(2 * n_roots)
        r1 = np.zeros(n_roots)
        it = ctypes.c_int()
        ok = (0, -5) if allow_unconverged else (0,)
        _check(lib().ipeom_solve(self._ctx, n_roots, tol, max_iter, _dptr(w), _dptr(r1),
                                 ctypes.byref(it)), self._ctx, ok)
        self.davidson_iterations = it.value
        return w[0::2] + 1j * w[1::2], r1

    def ipeom_lr(self, n_roots, tol=1e-7, max_iter=100, allow_unconverged=False):
        """IPs with right and left vectors (Eqs. 18-20), biorthonormal:
        L @ R.T = 1 over the roots. Returns (omega, R, L, pole) with R, L
        [n_roots][dim] in the packed layout and pole[k] = sum_i L[k,i] R[k,i]."""
        o, v, _ = self.sizes()
        dim = o + o * (o - 1) // 2 * v
        w = np.zeros(2 * n_roots)
        pole = np.zeros(2 * n_roots)
        R = np.empty((n_roots, dim), np.complex128)
        Lv = np.empty((n_roots, dim), np.complex128)
        it = (ctypes.c_int * 2)()
        ok = (0, -5) if allow_unconverged else (0,)
        _check(lib().ipeom_solve_lr(self._ctx, n_roots, tol, max_iter, _dptr(w),
                                    R.view(np.float64).ctypes.data_as(_D),
                                    Lv.view(np.float64).ctypes.data_as(_D), _dptr(pole),
                                    ctypes.cast(it, _I)), self._ctx, ok)
        self.davidson_iterations = (it[0], it[1])
        return w[0::2] + 1j * w[1::2], R, Lv, pole[0::2] + 1j * pole[1::2]

    def set_graphs(self, on=True):
        _check(lib().cc_set_graphs(self._ctx, 1 if on else 0), self._ctx)

    def set_allocator(self, alloc, free, user=None):
        """Route this system's later device allocations through ctypes
        callbacks alloc(nbytes, user) -> ptr and free(ptr, user) (None, None:
        cudaMalloc/cudaFree). The callbacks must outlive the system."""
        if alloc is None:
            _check(lib().cc_set_allocator(self._ctx, _ALLOC(), _FREE(), None), self._ctx)
            self._alloc_hooks = None
            return
        hooks = (_ALLOC(alloc), _FREE(free))
        _check(lib().cc_set_allocator(self._ctx, hooks[0], hooks[1], user), self._ctx)
        self._alloc_hooks = hooks

    def set_fault_injection(self, kind, at_iteration=1):
        """Test hook: kind 1 = NaN into the CCSD residual of an iteration,
        2 = NaN into the Davidson sigma vectors of an iteration, 0 = off."""
        _check(lib().cc_set_fault_injection(self._ctx, int(kind), int(at_iteration)), self._ctx)

    def set_davidson_guess(self, mode, mlp=None):
        """Davidson start: "unit" (0), "first_order" (1) or "learned" (2,
        needs a trained Mlp that outlives this system)."""
        m = {"unit": 0, "first_order": 1, "learned": 2}.get(mode, mode)
        _check(lib().cc_set_davidson_guess(self._ctx, int(m), mlp._h if mlp else None),
               self._ctx)
        self._guess_mlp = mlp

    def guess_dev(self, n_roots):
        """The n_roots Davidson starting vectors of the current mode (device
        complex128 tensor [n_roots][dim])."""
        import torch
        o, v, _ = self.sizes()
        dim = o + o * (o - 1) // 2 * v
        out = torch.zeros((n_roots, dim), dtype=torch.complex128, device="cuda")
        _check(lib().ipeom_guess_dev(self._ctx, int(n_roots), _P(out.data_ptr())), self._ctx)
        return out

    def set_memory_limit(self, nbytes):
        """Cap the device bytes this system holds (0: no cap)."""
        _check(lib().cc_set_memory_limit(self._ctx, int(nbytes)), self._ctx)

    def get_amplitudes(self):
        o, v, _ = self.sizes()
        t1 = np.empty(o * v, np.complex128)
        t2 = np.empty(o * (o - 1) // 2 * (v * (v - 1) // 2), np.complex128)
        _check(lib().cc_get_amplitudes(self._ctx, t1.view(np.float64).ctypes.data_as(_D),
                                       t2.view(np.float64).ctypes.data_as(_D)), self._ctx)
        return t1.reshape(o, v), t2

    def reset_amplitudes(self):
        _check(lib().cc_reset_amplitudes(self._ctx), self._ctx)

    def set_amplitudes(self, t1, t2_packed):
        t1 = np.ascontiguousarray(t1, np.complex128)
        t2 = np.ascontiguousarray(t2_packed, np.complex128)
        _check(lib().cc_set_amplitudes(self._ctx, t1.view(np.float64).ctypes.data_as(_D),
                                       t2.view(np.float64).ctypes.data_as(_D)), self._ctx)

    # ---- components on device tensors (torch complex128, contiguous) ----
    def ladder_dev(self, tau, out):
        _check(lib().cc_ladder_dev(self._ctx, _P(tau.data_ptr()), _P(out.data_ptr())),
               self._ctx)

    def residual_dev(self, t1, t2, r1, r2):
        _check(lib().cc_residual_dev(self._ctx, _P(t1.data_ptr()), _P(t2.data_ptr()),
                                     _P(r1.data_ptr()), _P(r2.data_ptr())), self._ctx)

    def sigma_dev(self, r, s):
        _check(lib().ipeom_sigma_dev(self._ctx, int(r.shape[0]), _P(r.data_ptr()),
                                     _P(s.data_ptr())), self._ctx)

    def left_sigma_dev(self, l, s):
        _check(lib().ipeom_left_sigma_dev(self._ctx, int(l.shape[0]), _P(l.data_ptr()),
                                          _P(s.data_ptr())), self._ctx)

    def dump_integrals(self, block):
        o, v, _ = self.sizes()
        shapes = {0: (o, o, o, o), 1: (o, o, o, v), 2: (o, o, v, v), 3: (o, v, v, o)}
        out = np.empty(shapes[block], np.complex128)
        _check(lib().cc_dump_integrals(self._ctx, block,
                                       out.view(np.float64).ctypes.data_as(_D)), self._ctx)
        return out

    def stats(self):
        s = np.zeros(20)
        _check(lib().cc_get_stats(self._ctx, _dptr(s), 20), self._ctx)
        keys = ["ladder_ms", "ladder_calls", "ladder_flops", "fns_ms", "ccsd_ms",
                "ipeom_ms", "launches", "ccsd_iter", "davidson_iter", "ladder_tc_ms",
                "ladder_tc_launches", "device_peak_bytes", "diis_depth",
                "ccsd_loop_peak_bytes", "device_bytes_held", "ccsd_escalated_at",
                "sigma_ms", "sigma_calls", "sigma_flops", "sigma_vectors"]
        return {k: float(s[i]) for i, k in enumerate(keys)}


_FP = ctypes.POINTER(ctypes.c_float)


def _fptr(a):
    return a.ctypes.data_as(_FP)


class Mlp:
    """The learned warm start (8 -> 64 -> 64 -> 2 MLP, FP16 weights).

    Parameters are a flat float32 array (W1, b1, W2, b2, W3, b3); see
    cc_mlp_* in cdfns.h for the features and the loss.
    """

    def __init__(self, params=None, seed=0):
        self._h = _P()
        _check(lib().cc_mlp_create(ctypes.byref(self._h)))
        self.n_params = lib().cc_mlp_num_params()
        if params is None:
            params = self.init_params(seed)
        self.set_params(params)

    @staticmethod
    def init_params(seed=0):
        """He-uniform weights, zero biases (the last layer starts small)."""
        rng = np.random.default_rng(seed)
        parts = []
        for fan_in, fan_out, scale in ((8, 64, 1.0), (64, 64, 1.0), (64, 2, 0.01)):
            lim = scale * np.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, (fan_out, fan_in)).ravel())
            parts.append(np.zeros(fan_out))
        return np.concatenate(parts).astype(np.float32)

    def _err(self, rc, ok=(0,)):
        if rc not in ok:
            raise CCError(rc, lib().cc_mlp_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib().cc_mlp_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._err(lib().cc_mlp_set_params(self._h, _fptr(p), p.size))

    def params(self):
        out = np.empty(self.n_params, np.float32)
        self._err(lib().cc_mlp_get_params(self._h, _fptr(out), out.size))
        return out

    def add_samples(self, system, max_samples):
        self._err(lib().cc_mlp_add_samples(self._h, system._ctx, int(max_samples)))

    def num_samples(self):
        n = ctypes.c_long()
        self._err(lib().cc_mlp_num_samples(self._h, ctypes.byref(n)))
        return n.value

    def train(self, steps, batch=4096, lr=1e-3, perm=None):
        loss = ctypes.c_double()
        if perm is not None:
            perm = np.ascontiguousarray(perm, dtype=np.int32)
            pp, pl = perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), perm.size
        else:
            pp, pl = None, 0
        self._err(lib().cc_mlp_train(self._h, int(steps), int(batch), float(lr), pp, pl,
                                     ctypes.byref(loss)))
        return loss.value

    def loss_grad(self, X, Y):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_double()
        self._err(lib().cc_mlp_loss_grad(self._h, X.shape[0], _fptr(X), _fptr(Y),
                                         ctypes.byref(loss), _fptr(g)))
        return loss.value, g

    def add_guess_samples(self, system, max_samples):
        """Davidson-start training samples from system's last converged
        ipeom_solve."""
        self._err(lib().cc_mlp_add_guess_samples(self._h, system._ctx, int(max_samples)))

    @staticmethod
    def guess_features(system, seed, n):
        out = np.empty((n, 8), np.float32)
        _check(lib().cc_mlp_guess_features(system._ctx, int(seed), int(n), _fptr(out)),
               system._ctx)
        return out

    def warm_start(self, system):
        self._err(lib().cc_mlp_warm_start(self._h, system._ctx))

    @staticmethod
    def features(system, n):
        out = np.empty((n, 8), np.float32)
        _check(lib().cc_mlp_features(system._ctx, int(n), _fptr(out)), system._ctx)
        return out
