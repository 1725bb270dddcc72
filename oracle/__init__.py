"""Plain FP64 CPU oracle for CD/FNS IP-EOM-CCSD (test infrastructure only).

This package is the slow, obviously correct reference that the CUDA path is
checked against. It is test infrastructure: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it. The library in ``paper_2506_06805_gb300`` never imports it, and
it never imports the library; the two share no code. Inputs come from
``paper_2506_06805_gb300.synth``, which draws random numbers only.

Modules (each function cites the passage of the paper it follows):

* ``integrals`` -- antisymmetrised integrals from Cholesky vectors (Eq. 23).
* ``mp2``       -- first-order doubles and the MP2 energy.
* ``fns``       -- frozen natural spinors (Eqs. 24-28).
* ``ccsd``      -- spin-orbital CCSD with DIIS (Eqs. 12-15).
* ``ipeom``     -- IP-EOM-CCSD sigma, dense H-bar, its eigenvalues and
                   left vectors (Eqs. 16-20).
* ``davidson``  -- a plain non-Hermitian Davidson for larger sizes.
* ``cholesky``  -- single-step pivoted Cholesky decomposition (Eq. 21).
* ``fci``       -- brute-force second quantisation on determinant
                   bitstrings, used to pin the working equations.

Everything is numpy complex128/float64; library calls (einsum, eigh, eig,
solve) serve as steps, with no blocking or reordering beyond the
definitions.
"""
