"""Seeded synthetic systems: orbital energies and complex Cholesky vectors.

This module only draws random inputs. It holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it.

A system is (n_occ, n_virt, n_aux, eps, L):

* ``eps``  float64 [n], occupied spinors first, in Hartree.
  Occupied energies are uniform in [-2.0, -0.3], virtual ones uniform in
  [0.2, 5.0]; each group is sorted ascending.
* ``L``    complex128 [n_aux][n][n], every L^P Hermitian in (p, q), the
  Cholesky vectors of the two-electron integrals in the spinor basis
  (Cholesky factorisation, Eq. 21; molecular-orbital form, Eq. 22).

Random-number recipe (numpy ``default_rng(seed)``, PCG64), in draw order:

1. occupied energies, 2. virtual energies,
3. for each P in ascending order: x (n x n) then y (n x n), both N(0, 1);
   Z^P = s (x + i y) / sqrt(2) with s = 0.05 / sqrt(n_aux), and
   L^P = (Z^P + Z^P^H) / 2.

Because every P draws the same amount in the same order, a P-chunked
generation is bit-identical to the whole-array one.

Kramers-paired (time-reversal-symmetric) systems: n_occ and n_virt are even,
h = n/2 spatial-like pairs are drawn (o/2 occupied then v/2 virtual energies,
each duplicated into spinors 2k and 2k+1), and for each P: x, y (h x h) give
A = Herm(Z) and x2, y2 (h x h) give Z2 with B = (Z2 - Z2^T)/2. In the
(unbarred block, barred block) basis L^P = [[A, B], [-B*, A*]], which is
Hermitian and even under time reversal; the blocks are then interleaved so
that Kramers partners sit at (2k, 2k+1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "SystemSpec", "CONFIGS", "make_eps", "make_cholesky", "make_system",
    "cholesky_chunks", "cholesky_chunks_device", "batch_specs",
]

EPS_OCC_RANGE = (-2.0, -0.3)
EPS_VIRT_RANGE = (0.2, 5.0)
L_SCALE = 0.05


class SystemSpec(dict):
    """Plain dict with attribute access: n_occ, n_virt, n_aux, seed, kramers."""

    __getattr__ = dict.__getitem__


def _spec(n_occ, n_virt, n_aux, seed=0, kramers=False, **extra):
    return SystemSpec(n_occ=n_occ, n_virt=n_virt, n_aux=n_aux, seed=seed,
                      kramers=kramers, **extra)


# Workload shapes. "tiny" is the oracle-in-seconds case; "medium" the
# Kramers-paired time-to-roots workload; the others are FNS, batched and
# large shapes.
CONFIGS = {
    "tiny": _spec(10, 30, 120, n_roots=4, ccsd_tol=1e-8, eom_tol=1e-7),
    "mid": _spec(12, 72, 288, n_roots=4, ccsd_tol=1e-8, eom_tol=1e-7),
    "small": _spec(20, 160, 640, kramers=True, n_roots=8, ccsd_tol=1e-8,
                   eom_tol=1e-7),
    "medium": _spec(40, 300, 1200, kramers=True, n_roots=8, ccsd_tol=1e-8,
                    eom_tol=1e-7),
    "fns": _spec(40, 800, 2400, n_roots=8, fns_threshold=1e-5,
                 ccsd_tol=1e-8, eom_tol=1e-7),
    "batched_big": _spec(60, 600, 2400, n_roots=16, ccsd_tol=1e-8,
                         eom_tol=1e-7),
    "large": _spec(80, 1698, 4000, n_roots=8, ccsd_tol=1e-8, eom_tol=1e-7),
}


def _energies(rng, n, lo_hi):
    lo, hi = lo_hi
    return np.sort(rng.uniform(lo, hi, size=n))


def make_eps(rng, n_occ, n_virt, kramers=False):
    """Orbital energies, occupied first (draws 1 and 2 of the recipe)."""
    if kramers:
        if n_occ % 2 or n_virt % 2:
            raise ValueError("Kramers-paired systems need even n_occ, n_virt")
        eo = np.repeat(_energies(rng, n_occ // 2, EPS_OCC_RANGE), 2)
        ev = np.repeat(_energies(rng, n_virt // 2, EPS_VIRT_RANGE), 2)
    else:
        eo = _energies(rng, n_occ, EPS_OCC_RANGE)
        ev = _energies(rng, n_virt, EPS_VIRT_RANGE)
    return np.concatenate([eo, ev])


def _herm_gauss(rng, m, s):
    x = rng.standard_normal((m, m))
    y = rng.standard_normal((m, m))
    z = s * (x + 1j * y) / np.sqrt(2.0)
    return z


def _kramers_perm(n):
    """Index map from the (unbarred block, barred block) basis to interleaved."""
    h = n // 2
    perm = np.empty(n, dtype=np.int64)
    perm[0::2] = np.arange(h)
    perm[1::2] = h + np.arange(h)
    return perm


def cholesky_chunks(rng, n, n_aux, p0, p1, kramers=False, out=None):
    """Cholesky vectors P in [p0, p1), drawn from ``rng`` positioned at P=p0.

    The caller draws P in ascending order across calls; the result equals the
    same slice of the whole-array generation.
    """
    s = L_SCALE / np.sqrt(n_aux)
    if out is None:
        out = np.empty((p1 - p0, n, n), dtype=np.complex128)
    if kramers:
        h = n // 2
        perm = _kramers_perm(n)
        blk = np.empty((n, n), dtype=np.complex128)
        for k in range(p1 - p0):
            z = _herm_gauss(rng, h, s)
            a = 0.5 * (z + z.conj().T)
            z2 = _herm_gauss(rng, h, s)
            b = 0.5 * (z2 - z2.T)
            blk[:h, :h] = a
            blk[:h, h:] = b
            blk[h:, :h] = -b.conj()
            blk[h:, h:] = a.conj()
            out[k] = blk[np.ix_(perm, perm)]
    else:
        for k in range(p1 - p0):
            z = _herm_gauss(rng, n, s)
            out[k] = 0.5 * (z + z.conj().T)
    return out


def cholesky_chunks_device(seed, n, n_aux, p0, p1, device="cuda"):
    """Cholesky vectors P in [p0, p1) with the distribution of
    ``cholesky_chunks`` (non-Kramers), drawn on the GPU by torch from a
    generator seeded with (seed, p0): L^P = (Z + Z^H) / 2 with
    Z = s (x + i y) / sqrt(2), s = L_SCALE / sqrt(n_aux). For the inputs too
    large to draw on the host in reasonable time (the large configuration:
    4000 vectors of 1778 x 1778); reproducible for the same chunking on the
    same software, not equal to the numpy stream of ``cholesky_chunks``.
    Returns a contiguous complex128 CUDA tensor [p1-p0][n][n]."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + int(p0))
    s = L_SCALE / np.sqrt(n_aux)
    x = torch.randn((p1 - p0, n, n), generator=g, device=device, dtype=torch.float64)
    y = torch.randn((p1 - p0, n, n), generator=g, device=device, dtype=torch.float64)
    z = torch.complex(x, y) * (s / np.sqrt(2.0))
    del x, y
    return (0.5 * (z + z.conj().transpose(1, 2))).contiguous()


def make_cholesky(rng, n, n_aux, kramers=False):
    return cholesky_chunks(rng, n, n_aux, 0, n_aux, kramers=kramers)


def make_system(n_occ, n_virt, n_aux, seed=0, kramers=False):
    """Return (eps, L) for one system following the module recipe."""
    rng = np.random.default_rng(seed)
    eps = make_eps(rng, n_occ, n_virt, kramers)
    L = make_cholesky(rng, n_occ + n_virt, n_aux, kramers)
    return eps, L


def make_config(name):
    c = CONFIGS[name]
    eps, L = make_system(c.n_occ, c.n_virt, c.n_aux, c.seed, c.kramers)
    return c, eps, L


def batch_specs(n_sys=8, seed=0, occ_range=(20, 50), virt_range=(150, 400)):
    """Shapes of the uneven batch: n_occ in [20, 50], n_virt in [150, 400]
    (inclusive ranges, replaceable for batches of smaller systems).

    Shapes come from ``default_rng(seed)``; system s draws its own inputs from
    ``default_rng([seed, s + 1])`` with n_aux = 4 n_virt.
    """
    rng = np.random.default_rng(seed)
    occ = rng.integers(occ_range[0], occ_range[1] + 1, size=n_sys)
    virt = rng.integers(virt_range[0], virt_range[1] + 1, size=n_sys)
    return [
        _spec(int(o), int(v), int(4 * v), seed=[seed, s + 1])
        for s, (o, v) in enumerate(zip(occ, virt))
    ]


def gauge_transform(L, theta):
    """Multiply spinor p by exp(i theta_p): L^P_pq -> e^{-i th_p} L^P_pq e^{i th_q}.

    Physical observables (energies, IPs) are invariant under this change of
    phase conventions; it is an input transformation, used by tests.
    """
    ph = np.exp(1j * np.asarray(theta))
    return ph.conj()[None, :, None] * L * ph[None, None, :]
