"""Micro-benchmarks of the library's hot kernels on synthetic inputs.

    python -m paper_2506_06805_gb300.kernel_bench ladder --o 20 --v 160 --X 640
    python -m paper_2506_06805_gb300.kernel_bench gemm --M 4096 --N 4096 --K 4096

``ladder`` times cc_ladder_dev (1/2 sum_cd <ab||cd> tau_ij^cd with <ab||cd>
formed from Cholesky vectors) and reports algorithmic TFLOP/s with the
symmetry-reduced count 8 [X v^3 (v-1)/2 + (v(v-1)/2)^2 o(o-1)/2].
``gemm`` times the complex GEMM entry point (8 M N K flops).
One JSON line per run.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    import torch

    from . import System, synth, use_torch_memory, zgemm_dev
    p = argparse.ArgumentParser()
    p.add_argument("what", choices=["ladder", "gemm"])
    p.add_argument("--o", type=int, default=20)
    p.add_argument("--v", type=int, default=160)
    p.add_argument("--X", type=int, default=640)
    p.add_argument("--M", type=int, default=4096)
    p.add_argument("--N", type=int, default=4096)
    p.add_argument("--K", type=int, default=4096)
    p.add_argument("--tier", default="tf32")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=1)
    a = p.parse_args()
    use_torch_memory()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if a.what == "ladder":
        eps, L = synth.make_system(a.o, a.v, a.X, seed=0, kramers=False)
        rng = np.random.default_rng(1)
        tau = (rng.standard_normal((a.o, a.o, a.v, a.v))
               + 1j * rng.standard_normal((a.o, a.o, a.v, a.v))) * 1e-3
        tau = tau - tau.transpose(1, 0, 2, 3)
        tau = tau - tau.transpose(0, 1, 3, 2)
        td = torch.from_numpy(tau).cuda()
        out = torch.empty_like(td)
        with System(eps, L, n_occ=a.o, tier=a.tier) as s:
            for _ in range(a.warmup):
                s.ladder_dev(td, out)
            torch.cuda.synchronize()
            ev0.record()
            for _ in range(a.reps):
                s.ladder_dev(td, out)
            ev1.record()
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / a.reps
        o, v, X = a.o, a.v, a.X
        fl = 8.0 * (X * v ** 3 * (v - 1) / 2 + (v * (v - 1) / 2) ** 2 * (o * (o - 1) / 2))
        print(json.dumps({"kernel": "ladder", "o": o, "v": v, "X": X, "tier": a.tier,
                          "ms": ms, "tflops": fl / ms / 1e9}))
    else:
        rng = np.random.default_rng(0)
        A = torch.from_numpy(rng.standard_normal((a.M, a.K)) + 1j * rng.standard_normal((a.M, a.K))).cuda()
        B = torch.from_numpy(rng.standard_normal((a.N, a.K)) + 1j * rng.standard_normal((a.N, a.K))).cuda()
        C = torch.empty((a.M, a.N), dtype=torch.complex128, device="cuda")
        for _ in range(a.warmup):
            zgemm_dev(A, B, C, a.tier)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(a.reps):
            zgemm_dev(A, B, C, a.tier)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / a.reps
        print(json.dumps({"kernel": "zgemm", "M": a.M, "N": a.N, "K": a.K, "tier": a.tier,
                          "ms": ms, "tflops": 8.0 * a.M * a.N * a.K / ms / 1e9}))


if __name__ == "__main__":
    main()
