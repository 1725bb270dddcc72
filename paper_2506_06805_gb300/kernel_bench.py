"""Micro-benchmarks of the library's hot kernels on synthetic inputs.

    python -m paper_2506_06805_gb300.kernel_bench ladder --o 20 --v 160 --X 640
    python -m paper_2506_06805_gb300.kernel_bench gemm --M 4096 --N 4096 --K 4096
    python -m paper_2506_06805_gb300.kernel_bench fns --config fns --keep-frac 0.4
    python -m paper_2506_06805_gb300.kernel_bench batch --n-sys 8 --roots 8
    python -m paper_2506_06805_gb300.kernel_bench solve --config batched_big --roots 16

``ladder`` times cc_ladder_dev (1/2 sum_cd <ab||cd> tau_ij^cd with <ab||cd>
formed from Cholesky vectors) and reports algorithmic TFLOP/s with the
symmetry-reduced count 8 [X v^3 (v-1)/2 + (v(v-1)/2)^2 o(o-1)/2].
``gemm`` times the complex GEMM entry point (8 M N K flops).
``fns`` feeds a configured system's Cholesky vectors in chunks of 200
(cc_add_cholesky), reports the natural-spinor occupations and the count
kept at the literal threshold, then runs FNS with the kept fraction,
CCSD and IP-EOM with CCSD in --tier and in --eom-tier (the EOM sigma in
--eom-tier both times) and compares their IPs.
``batch`` builds the uneven batch of systems (n_occ 20-50, n_virt 150-400,
n_aux = 4 n_virt, shapes and inputs from ``synth.batch_specs``), solves
CCSD for each, then times IP-EOM for all of them one after another and as
one batch (batched sigma in grouped launches, with and without CUDA graphs)
and compares the roots; ``--small`` draws systems with n_occ 6-12 and
n_virt 30-80 instead, none of which fills the GPU alone.
``solve`` runs one configured system end to end (Cholesky vectors fed in
chunks of 200, CCSD, IP-EOM with all roots in one block) on the library's
own cudaMalloc allocations, and reports the phase times, iteration counts,
the ladder rate, the DIIS depth the device memory allowed and the high-water
mark of the library's device memory; with --left it then solves for the
right and left vectors together (ipeom_solve_lr) and reports their
biorthonormality and 1h overlaps.
``warmstart`` trains the amplitude and Davidson-start networks on generated
smaller systems and solves a configured system with and without them.
``cholesky`` times the single-step pivoted Cholesky decomposition (Eq. 21)
of M = B B^H for a seeded generator B [N][r] and reports the HBM rate on its
algorithmic bytes.
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
    p.add_argument("what", choices=["ladder", "gemm", "fns", "batch", "solve", "cholesky",
                                    "warmstart"])
    p.add_argument("--train", default="12,96,384,3",
                   help="warmstart: o,v,X,count of the generated training systems")
    p.add_argument("--pairs", type=int, default=435600, help="cholesky: N (orbital pairs)")
    p.add_argument("--rank", type=int, default=600, help="cholesky: columns of the generator")
    p.add_argument("--tau", type=float, default=0.0, help="cholesky: threshold")
    p.add_argument("--max-vec", type=int, default=600, help="cholesky: vector limit")
    p.add_argument("--n-sys", type=int, default=8)
    p.add_argument("--small", action="store_true",
                   help="batch: systems with n_occ 6-12 and n_virt 30-80 instead of 20-50 / 150-400")
    p.add_argument("--roots", type=int, default=8)
    p.add_argument("--config", default="fns")
    p.add_argument("--keep-frac", type=float, default=0.4)
    p.add_argument("--o", type=int, default=20)
    p.add_argument("--v", type=int, default=160)
    p.add_argument("--X", type=int, default=640)
    p.add_argument("--M", type=int, default=4096)
    p.add_argument("--N", type=int, default=4096)
    p.add_argument("--K", type=int, default=4096)
    p.add_argument("--tier", default="fp16")
    p.add_argument("--eom-tier", default="fp16x3")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=1)
    p.add_argument("--left", action="store_true",
                   help="solve: left vectors too (ipeom_solve_lr)")
    p.add_argument("--fns-keep", type=int, default=0,
                   help="solve: streamed natural spinors keeping this many virtuals")
    p.add_argument("--device-inputs", action="store_true",
                   help="solve: draw the Cholesky vectors on the GPU (synth.cholesky_chunks_device)")
    a = p.parse_args()
    if a.what == "solve":
        return solve_run(a)
    if a.what == "warmstart":
        return warmstart_run(a)
    use_torch_memory()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if a.what == "fns":
        return fns_run(a)
    if a.what == "batch":
        return batch_run(a)
    if a.what == "cholesky":
        return cholesky_run(a)
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


def fns_run(a):
    import time

    import torch

    from . import System, synth
    c = synth.CONFIGS[a.config]
    o, v, X = c.n_occ, c.n_virt, c.n_aux
    out = {"config": a.config, "o": o, "v": v, "X": X}

    def make(tier, eom):
        rng = np.random.default_rng(c.seed)
        eps = synth.make_eps(rng, o, v, c.kramers)
        s = System(eps, None, n_occ=o, n_aux=X, tier=tier, eom_tier=eom)
        for p0 in range(0, X, 200):
            p1 = min(X, p0 + 200)
            s.add_cholesky(p0, p1, synth.cholesky_chunks(rng, o + v, X, p0, p1, c.kramers))
        return s

    thr = c.get("fns_threshold", 1e-5)
    with make(a.tier, a.eom_tier) as s:
        t0 = time.perf_counter()
        out["kept_at_threshold"] = s.fns_truncate(threshold=thr)
        torch.cuda.synchronize()
        out["fns_s"] = time.perf_counter() - t0
        occ = s.fns_occupations(v)
        out["threshold"] = thr
        out["occ_max"] = float(occ[0])
        out["n_ge"] = {f"{t:.3g}": int((occ >= t).sum()) for t in (1e-4, 10 ** -4.5, 1e-5, 1e-6)}
    n_keep = max(1, int(round(a.keep_frac * v)))
    res = {}
    # the CCSD tier against the accurate EOM tier used throughout
    pairs = ((a.tier, a.eom_tier), (a.eom_tier, a.eom_tier))
    for tier, eom in pairs:
        with make(tier, eom) as s:
            t0 = time.perf_counter()
            s.fns_truncate(n_keep=n_keep)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            e = s.ccsd(tol=c.ccsd_tol, max_iter=60)
            t2 = time.perf_counter()
            w, _ = s.ipeom(c.n_roots, tol=c.eom_tol, max_iter=100)
            t3 = time.perf_counter()
            res[tier] = {"fns_s": t1 - t0, "ccsd_s": t2 - t1, "ipeom_s": t3 - t2,
                         "e_corr": [e.real, e.imag], "ccsd_iter": s.ccsd_iterations,
                         "ips": [float(x) for x in np.sort(w.real)]}
    out["n_keep"] = n_keep
    out["runs"] = res
    t0, t1 = pairs[0][0], pairs[1][0]
    out[f"max_dIP_{t0}_vs_{t1}"] = float(np.abs(np.array(res[t0]["ips"])
                                               - np.array(res[t1]["ips"])).max())
    print(json.dumps(out))


def cholesky_run(a):
    """Times cc_cholesky_dev on a seeded generator B [N][r] (the oracle's
    test recipe) and reports HBM throughput on the algorithmic bytes: each
    step k reads B and the k vectors so far, 16 N (r + k) bytes."""
    import torch

    from . import cholesky_dev
    N, r = a.pairs, a.rank
    rng = np.random.default_rng(0)
    B = torch.empty((N, r), dtype=torch.complex128, device="cuda")
    for q0 in range(0, N, 65536):  # generate in slices to bound host memory
        q1 = min(N, q0 + 65536)
        x = (rng.standard_normal((q1 - q0, r)) + 1j * rng.standard_normal((q1 - q0, r)))
        B[q0:q1] = torch.from_numpy(x / np.sqrt(2 * r))
    cholesky_dev(B[:4096].contiguous(), a.tau, 4)  # warm-up (module load)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    L, piv = cholesky_dev(B, a.tau, a.max_vec)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    n = L.shape[0]
    byts = 16.0 * N * (n * r + n * (n - 1) / 2)
    print(json.dumps({"kernel": "pivoted_cholesky", "N": N, "r": r, "tau": a.tau, "n_vec": n,
                      "ms": ms, "ms_per_vector": ms / max(1, n),
                      "algorithmic_GB": byts / 1e9, "GBps": byts / ms / 1e6}))


def solve_run(a):
    import time

    from . import System, synth
    c = synth.CONFIGS[a.config]
    o, v, X = c.n_occ, c.n_virt, c.n_aux
    nr = a.roots if a.roots > 0 else c.n_roots
    rng = np.random.default_rng(c.seed)
    eps = synth.make_eps(rng, o, v, c.kramers)
    out = {"config": a.config, "o": o, "v": v, "X": X, "roots": nr, "tier": a.tier,
           "eom_tier": a.eom_tier}
    step = max(1, min(200, int(2e9 // (16 * (o + v) ** 2))))

    def chunks():
        # the same draws each time: eps first, then the vectors P in order
        if a.device_inputs:
            for p0 in range(0, X, step):
                p1 = min(X, p0 + step)
                yield p0, p1, synth.cholesky_chunks_device(c.seed, o + v, X, p0, p1)
            return
        r = np.random.default_rng(c.seed)
        synth.make_eps(r, o, v, c.kramers)
        for p0 in range(0, X, step):
            p1 = min(X, p0 + step)
            yield p0, p1, synth.cholesky_chunks(r, o + v, X, p0, p1, c.kramers)

    t0 = time.perf_counter()
    with System(eps, None, n_occ=o, n_aux=X, tier=a.tier, eom_tier=a.eom_tier,
                torch_memory=False) as s:
        if a.fns_keep > 0:
            out["fns_kept"] = s.fns_stream(chunks, n_keep=a.fns_keep)
            out["fns_s"] = s.stats()["fns_ms"] / 1e3
            occ = s.fns_occupations(v)
            out["fns_occ_range"] = [float(occ[0]), float(occ[a.fns_keep - 1]), float(occ[-1])]
            out["fns_kept_at_1e-5"] = int(np.count_nonzero(occ >= 1e-5))
        else:
            for p0, p1, Lc in chunks():
                s.add_cholesky(p0, p1, Lc)
        t1 = time.perf_counter()
        e = s.ccsd(tol=c.ccsd_tol, max_iter=60)
        t2 = time.perf_counter()
        w, r1 = s.ipeom(nr, tol=c.eom_tol, max_iter=100)
        t3 = time.perf_counter()
        st = s.stats()
        if a.left:
            # right and left vectors again from the same H-bar (built above)
            t4 = time.perf_counter()
            wl, R, Lv, pole = s.ipeom_lr(nr, tol=c.eom_tol, max_iter=100)
            out["ipeom_lr_s"] = time.perf_counter() - t4
            out["davidson_iter_right_left"] = list(s.davidson_iterations)
            out["biorth_err"] = float(np.abs(Lv @ R.T - np.eye(nr)).max())
            out["max_dIP_lr_vs_right"] = float(np.abs(np.sort_complex(wl) - np.sort_complex(w)).max())
            out["pole"] = [[p.real, p.imag] for p in pole]
    order = np.argsort(w.real)
    out.update({
        "input_s": t1 - t0, "ccsd_s": t2 - t1, "ipeom_s": t3 - t2,
        "ccsd_iter": s.ccsd_iterations, "davidson_iter": s.davidson_iterations,
        "e_corr": [e.real, e.imag],
        "ips": [float(x) for x in w.real[order]],
        "r1_weight": [float(x) for x in r1[order]],
        "ladder_tflops": st["ladder_flops"] * st["ladder_calls"] / st["ladder_ms"] / 1e9
        if st["ladder_ms"] > 0 else None,
        "ladder_ms_per_call": st["ladder_ms"] / max(1.0, st["ladder_calls"]),
        "diis_depth": int(st["diis_depth"]), "device_peak_gb": st["device_peak_bytes"] / 1e9,
    })
    print(json.dumps(out))


def warmstart_run(a):
    """Learned starts on a configured system: the amplitude network (t2 =
    rho t_MP2) and the Davidson-start network (rho on first-order 2h1p
    components), both trained on generated smaller systems of the same
    recipe, against the MP2 / unit-vector start: CCSD and Davidson
    iterations, their times, and the IP differences."""
    import time

    import torch

    from . import Mlp, System, synth
    o_t, v_t, x_t, n_t = (int(x) for x in a.train.split(","))
    c = synth.CONFIGS[a.config]
    nr = a.roots if a.roots > 0 else c.n_roots
    t0 = time.perf_counter()
    amp, guess = Mlp(seed=0), Mlp(seed=1)
    for k in range(n_t):
        rng = np.random.default_rng([c.seed, 100 + k])
        eps = synth.make_eps(rng, o_t, v_t, c.kramers)
        L = synth.make_cholesky(rng, o_t + v_t, x_t, c.kramers)
        with System(eps, L, n_occ=o_t, tier=a.tier, eom_tier=a.eom_tier) as s:
            s.ccsd(tol=c.ccsd_tol, max_iter=100)
            s.ipeom(nr, tol=c.eom_tol, max_iter=200)
            amp.add_samples(s, 200000)
            guess.add_guess_samples(s, 200000)
    for net in (amp, guess):
        perm = np.random.default_rng(0).permutation(net.num_samples())
        net.train(2000, batch=2048, lr=2e-3, perm=perm)
    torch.cuda.synchronize()
    out = {"config": a.config, "tier": a.tier, "eom_tier": a.eom_tier, "roots": nr,
           "train_systems": [o_t, v_t, x_t, n_t], "train_s": time.perf_counter() - t0}
    res = {}
    o, v, X = c.n_occ, c.n_virt, c.n_aux
    if a.fns_keep > 0:
        # streamed natural spinors from GPU-drawn vectors (the large configuration)
        rng = np.random.default_rng(c.seed)
        eps = synth.make_eps(rng, o, v, c.kramers)
        step = max(1, min(200, int(2e9 // (16 * (o + v) ** 2))))

        def chunks():
            for p0 in range(0, X, step):
                yield p0, min(X, p0 + step), synth.cholesky_chunks_device(c.seed, o + v, X, p0,
                                                                           min(X, p0 + step))
        sys_ = System(eps, None, n_occ=o, n_aux=X, tier=a.tier, eom_tier=a.eom_tier)
        out["fns_kept"] = sys_.fns_stream(chunks, n_keep=a.fns_keep)
    else:
        _, eps, L = synth.make_config(a.config)
        sys_ = System(eps, L, n_occ=o, tier=a.tier, eom_tier=a.eom_tier)
        del L
    # with two rounds (small systems), the second is the one reported
    rounds = ("plain", "learned") if a.fns_keep > 0 else ("plain", "learned", "plain", "learned")
    with sys_ as s:
        for mode in rounds:
            s.reset_amplitudes()
            s.set_davidson_guess("unit" if mode == "plain" else "learned",
                                 None if mode == "plain" else guess)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if mode == "learned":
                amp.warm_start(s)
            e = s.ccsd(tol=c.ccsd_tol, max_iter=100)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            w, _ = s.ipeom(nr, tol=c.eom_tol, max_iter=200)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            st = s.stats()
            res[mode] = {"ccsd_iter": s.ccsd_iterations, "davidson_iter": s.davidson_iterations,
                         "diis_depth": int(st["diis_depth"]),
                         "ccsd_s": t2 - t1, "ipeom_s": t3 - t2, "time_to_roots_s": t3 - t1,
                         "e_corr": [e.real, e.imag], "ips": np.sort_complex(w)}
    d = float(np.abs(res["plain"]["ips"] - res["learned"]["ips"]).max())
    for m in res:
        res[m]["ips"] = [float(x) for x in res[m]["ips"].real]
    out.update({"plain": res["plain"], "learned": res["learned"], "max_dIP_learned_vs_plain": d})
    print(json.dumps(out))


def batch_run(a):
    import time

    import torch

    from . import System, batch_ipeom, synth
    specs = (synth.batch_specs(a.n_sys, occ_range=(6, 12), virt_range=(30, 80)) if a.small
             else synth.batch_specs(a.n_sys))
    systems = []
    t0 = time.perf_counter()
    for sp in specs:
        rng = np.random.default_rng(sp.seed)
        eps = synth.make_eps(rng, sp.n_occ, sp.n_virt)
        L = synth.make_cholesky(rng, sp.n_occ + sp.n_virt, sp.n_aux)
        s = System(eps, L, n_occ=sp.n_occ, tier=a.tier, eom_tier=a.eom_tier)
        del L
        s.ccsd(tol=1e-8, max_iter=60)
        systems.append(s)
    torch.cuda.synchronize()
    out = {"systems": [[sp.n_occ, sp.n_virt, sp.n_aux] for sp in specs],
           "tier": a.tier, "eom_tier": a.eom_tier,
           "ccsd_all_s": time.perf_counter() - t0, "roots": a.roots}
    # one at a time (a first untimed pass builds every system's H-bar)
    for s in systems:
        s.ipeom(a.roots, tol=1e-7, max_iter=100)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = [np.sort_complex(s.ipeom(a.roots, tol=1e-7, max_iter=100)[0]) for s in systems]
    torch.cuda.synchronize()
    out["eom_sequential_s"] = time.perf_counter() - t0
    for graphs in (False, True):
        for s in systems:
            s.set_graphs(graphs)
        t0 = time.perf_counter()
        w, _, it, status = batch_ipeom(systems, a.roots, tol=1e-7, max_iter=100)
        torch.cuda.synchronize()
        key = "eom_batched_graphs_s" if graphs else "eom_batched_s"
        out[key] = time.perf_counter() - t0
        out["max_dIP_batched_vs_sequential"] = float(max(
            np.abs(np.sort_complex(w[q]) - seq[q]).max() for q in range(len(systems))))
        out["davidson_iterations"] = [int(x) for x in it]
    for s in systems:
        s.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
