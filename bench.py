"""IP-EOM-CCSD time-to-roots on one GB300 (and N replicas), JSON line out.

Workload (N=1): the medium Kramers-paired system, n_occ=40, n_virt=300,
n_aux=1200, seed 0, 8 IP roots; CCSD tol 1e-8, Davidson tol 1e-7.

One step = the whole hot path on resident inputs: reset amplitudes, CCSD
from the MP2 start (every iteration: T1-dressed ladder + all other terms +
Jacobi/DIIS), H-bar build, block Davidson for 8 roots. The timed region
holds K steps between barriers and device synchronisation (CUDA events on
the library's stream). Inputs (L 2.2 GB, t2 2.3 GB) exceed the 129 MB L2,
so no flush is needed between steps.

``e2e`` repeats the step through the public C ABI from pinned host memory:
cc_init (H2D copy of eps and L) + ccsd_solve + ipeom_solve + result D2H.

After the timed region (and outside it) the same workload is solved again
for the metric's accuracy gate and comparator: once with every contraction
in the split FP16x3 tier, then from those amplitudes in the plain FP64 tier
until FP64 CCSD converges (one iteration, timed) and through a full FP64
H-bar build and Davidson (timed). The IPs of the timed run must lie within
1e-5 Eh of that FP64 solution (else the run fails); the FP64 time-to-roots
is the timed FP64 CCSD iteration times the CCSD iteration count of the
timed run, plus the timed FP64 IP-EOM step (labelled "extrapolated").

``--impl reference`` times the CPU oracle (numpy FP64) on bounded samples
of the same workload and extrapolates to the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("IP-EOM-CCSD time-to-roots & ladder TFLOP/s vs plain FP64, "
          "at |ΔIP|≤1e-5 Eh")

# DRAM bytes (read + write) per ladder call at the medium workload in the
# FP16 tier, from the one-pass ncu capture summarised in
# profiles/launches_medium_fp16.md; to be retaken whenever the ladder's
# kernels change
LADDER_TRAFFIC = 131.6e9
WORKLOAD = "medium"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default=WORKLOAD)
    p.add_argument("--tier", default="fp16")
    p.add_argument("--eom-tier", default="fp16x3")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true",
                   help="skip the FP64 comparator and the accuracy gate")
    return p.parse_args()


# |IP - IP(FP64)| the metric allows (Eh)
IP_GATE_EH = 1e-5


def fp64_comparator(P, eps, L, o, c, w_fast, ccsd_iters):
    """Accuracy gate and FP64 comparator for one workload (outside the timed
    region). Returns the dict reported under "fp64_comparator"."""
    import torch
    nr = c.n_roots
    with P.System(eps, L, n_occ=o, tier="fp16x3", eom_tier="fp16x3") as s3:
        s3.ccsd(tol=c.ccsd_tol, max_iter=100)
        w3, _ = s3.ipeom(nr, tol=c.eom_tol, max_iter=200)
        t1, t2 = s3.get_amplitudes()
    with P.System(eps, L, n_occ=o, tier="fp64", eom_tier="fp64") as s64:
        s64.set_amplitudes(t1, t2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64.ccsd(tol=c.ccsd_tol, max_iter=5)
        torch.cuda.synchronize()
        n64 = s64.ccsd_iterations
        t_iter = (time.perf_counter() - t0) / max(n64, 1)
        t0 = time.perf_counter()
        w64, _ = s64.ipeom(nr, tol=c.eom_tol, max_iter=200)
        torch.cuda.synchronize()
        t_eom = time.perf_counter() - t0
        dav64 = s64.davidson_iterations
    w64 = np.sort_complex(w64)
    d_fast = float(np.abs(np.sort_complex(w_fast) - w64).max())
    d_split = float(np.abs(np.sort_complex(w3) - w64).max())
    t_fp64 = t_iter * ccsd_iters + t_eom
    return {
        "max_dIP_vs_fp64_eh": d_fast, "gate_eh": IP_GATE_EH, "pass": d_fast <= IP_GATE_EH,
        "max_dIP_fp16x3_vs_fp64_eh": d_split,
        "fp64_time_to_roots_s": t_fp64,
        "fp64_kind": (f"extrapolated: one timed FP64 CCSD iteration ({t_iter:.1f} s) x "
                      f"{ccsd_iters} (the timed run's CCSD iteration count) + the timed FP64 "
                      f"H-bar build and Davidson ({t_eom:.1f} s, {dav64} iterations)"),
        "fp64_reference": (f"FP64 CCSD converged ({n64} FP64 iteration(s) from the FP16x3 "
                           "solution) and FP64 H-bar + Davidson to the workload's tolerances"),
    }


def max_over_ranks(value, device):
    """Largest value over the ranks of the initialised process group (the
    value itself with one rank): the step time all replicas waited for."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# CCSD iterations the oracle's algorithm (DIIS from its third iteration)
# needs on the medium workload, as measured with the library's FP64 path,
# which runs the same algorithm in FP64.
ORACLE_CCSD_ITERATIONS = 5


def workload_config(name, c, world):
    """The JSON `config` of both arms for one workload."""
    return {"workload": f"{name}: o={c.n_occ} v={c.n_virt} X={c.n_aux} kramers={c.kramers} "
                        f"roots={c.n_roots} ccsd_tol={c.ccsd_tol} eom_tol={c.eom_tol}",
            "l2": "inputs > L2 (L 2.2 GB, t2 2.3 GB); no flush",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={q}",
                     "--format=csv,noheader,nounits"],
                    capture_output=True, text=True, timeout=5).stdout.strip()
                f = [x.strip() for x in out.split(",")]
                self.samples.append(f)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(s[0]) for s in self.samples if s and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) > 1 and s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, n in enumerate(names):
                if len(s) > 3 + k and s[3 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
            "bf16_tflops_sustained": 1700.0}, "fallback"


# --------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of the same workload)
# --------------------------------------------------------------------------

def oracle_ladder_rows(L, eps, o, n_rows, budget_s):
    """Time the oracle's particle-particle ladder (Eq. 23 integrals, full
    sums) for a few rows a of the output; returns seconds per row."""
    from oracle import integrals, mp2
    v = L.shape[1] - o
    O, V = slice(0, o), slice(o, o + v)
    # tau = MP2 amplitudes (the first iteration's input)
    Lov = L[:, O, V]
    t_rows = []
    rng = np.random.default_rng(0)
    rows = rng.choice(v, size=min(n_rows, v), replace=False)
    # t2 for all ij, cd (MP2), built once (not timed): <ab||ij>/D
    g_oovv = integrals.antisym_block(L, O, O, V, V)
    t2 = g_oovv.conj() / mp2.denom2(eps, o)
    del g_oovv
    t_start = time.perf_counter()
    for a in rows:
        t0 = time.perf_counter()
        gab = integrals.antisym_block(L, slice(o + a, o + a + 1), V, V, V)[0]
        out = 0.5 * np.einsum("ijcd,bcd->ijb", t2, gab, optimize=True)
        t_rows.append(time.perf_counter() - t0)
        del gab, out
        if time.perf_counter() - t_start > budget_s:
            break
    return float(np.mean(t_rows)), len(t_rows), v, Lov.shape


def cpu_baseline(L, eps, o, ccsd_iters, budget_s=20.0):
    sec_per_row, n, v, _ = oracle_ladder_rows(L, eps, o, 4, budget_s)
    ladder_iter = sec_per_row * v
    value = ladder_iter * max(ccsd_iters, 1)
    return {
        "value": value, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
        "sample": (f"{n} of {v} rows a of the oracle's particle-particle ladder "
                   f"(numpy FP64, full <ab||cd> per row from L, Eq. 23) on this "
                   f"workload, scaled to all rows x {ccsd_iters} CCSD iterations; "
                   "ladder only (the dominant CCSD term), EOM not included: a "
                   "lower bound of the oracle's time-to-roots"),
    }


# --------------------------------------------------------------------------

def run_reference(args):
    r, w, _ = dist_env()
    if r != 0:
        return 0
    from paper_2506_06805_gb300 import synth
    c, eps, L = synth.make_config(args.config)
    o = c.n_occ
    vals = []
    steps = args.warmup + args.steps
    for s in range(steps):
        t0 = time.perf_counter()
        sec_row, n, v, _ = oracle_ladder_rows(L, eps, o, 1, 60.0)
        if s >= args.warmup:
            vals.append(sec_row * v * ORACLE_CCSD_ITERATIONS)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.config, c, 1),
        "cpu_baseline": {"value": value, "unit": "s", "cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": "per step one row a of the oracle ladder, scaled to "
                                   f"all rows x {ORACLE_CCSD_ITERATIONS} CCSD iterations "
                                   "(ladder only)"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    r, world, lr = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(lr)
    import paper_2506_06805_gb300 as P
    from paper_2506_06805_gb300 import synth
    c, eps, L = synth.make_config(args.config)
    o, v, X, nr = c.n_occ, c.n_virt, c.n_aux, c.n_roots
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t_init = time.perf_counter()
    s = P.System(eps, L, n_occ=o, tier=args.tier, eom_tier=args.eom_tier)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t_init
    if "fns_threshold" in c:
        pass  # the medium workload has no FNS step

    def step():
        s.reset_amplitudes()
        e = s.ccsd(tol=c.ccsd_tol, max_iter=100)
        w, r1 = s.ipeom(nr, tol=c.eom_tol, max_iter=200)
        return e, w, r1

    for _ in range(args.warmup):
        e, w, r1 = step()
    torch.cuda.synchronize()
    st0 = s.stats()
    clocks = Clocks(lr)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with clocks:
        ev0.record(stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e, w, r1 = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    st1 = s.stats()
    ms = max_over_ranks(ms, "cuda")
    ladder_calls = st1["ladder_calls"] - st0["ladder_calls"]
    ladder_ms = (st1["ladder_ms"] - st0["ladder_ms"]) / max(ladder_calls, 1)
    ladder_tf = st1["ladder_flops"] / (ladder_ms * 1e-3) / 1e12 if ladder_ms > 0 else None
    launches = int(st1["launches"] - st0["launches"])
    phases = {k: (st1[k] - st0[k]) / args.steps for k in ("ccsd_ms", "ipeom_ms", "fns_ms")}
    phases["ladder_ms_per_step"] = (st1["ladder_ms"] - st0["ladder_ms"]) / args.steps
    ccsd_iters = int(st1["ccsd_iter"])
    w = np.sort_complex(w)
    kramers_split = float(np.abs(w.real[0::2] - w.real[1::2]).max()) if c.kramers else None
    s.close()

    # end to end through the C ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        Lp = torch.from_numpy(L.view(np.float64)).pin_memory().numpy().view(np.complex128)
        epsp = torch.from_numpy(eps).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            with P.System(epsp, Lp, n_occ=o, tier=args.tier, eom_tier=args.eom_tier) as s2:
                s2.ccsd(tol=c.ccsd_tol, max_iter=100)
                s2.ipeom(nr, tol=c.eom_tol, max_iter=200)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(Lp.nbytes + epsp.nbytes),
               "d2h_bytes_per_step": int(16 + nr * 24)}

    fp64 = None
    if not args.no_fp64 and r == 0:
        fp64 = fp64_comparator(P, eps, L, o, c, w, ccsd_iters)
        fp64["speedup_vs_fp64"] = fp64["fp64_time_to_roots_s"] / (ms / 1e3)
        if not fp64["pass"]:
            print(json.dumps({"error": "accuracy gate failed", "fp64_comparator": fp64}))
            raise SystemExit(f"max |dIP| vs FP64 {fp64['max_dIP_vs_fp64_eh']:.3e} Eh "
                             f"exceeds {IP_GATE_EH:.0e} Eh")

    peaks, src = measured_peaks()
    # the ladder runs inside a seconds-long step: the sustained dense rate of
    # the operand type (fp16 = bf16 rate; tf32 = half of it, nominal ratio)
    base = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    ratio = 1.0 if args.tier in ("fp16", "bf16x3") else 0.5
    peak = base * ratio
    kind = {"fp16": "f16", "bf16x3": "f16 (bf16)", "tf32": "tf32", "tf32x3": "tf32"}.get(args.tier, args.tier)
    roofline = {
        "bound": "tensor",
        "kernel": f"particle-particle ladder (tcgen05 kind::{kind} GEMMs + antisymmetrise)",
        "achieved": ladder_tf, "peak": peak, "unit": "TFLOP/s",
        "frac": (ladder_tf / peak) if ladder_tf else None,
        "traffic": LADDER_TRAFFIC if (args.config, args.tier) == (WORKLOAD, "fp16") else None,
        "peak_source": f"{src} bf16 sustained x {ratio} (of measured)",
        "algorithmic_flops_per_call": st1["ladder_flops"], "ms_per_call": ladder_ms,
    }
    # the IP sigma builds of the timed steps (all roots of a Davidson round
    # in one batched build): algorithmic flops / device time, and the
    # executed tensor rate (split tiers run three products per term)
    sig_calls = st1["sigma_calls"] - st0["sigma_calls"]
    sig_ms = st1["sigma_ms"] - st0["sigma_ms"]
    sig_fl = st1["sigma_flops"] - st0["sigma_flops"]
    sig_vec = st1["sigma_vectors"] - st0["sigma_vectors"]
    eratio = 1.0 if args.eom_tier in ("fp16", "fp16x3", "bf16x3") else 0.5
    nprod = 3 if args.eom_tier in ("fp16x3", "bf16x3", "tf32x3") else 1
    sig_alg = sig_fl / (sig_ms * 1e-3) / 1e12 if sig_ms > 0 else None
    roofline_sigma = {
        "bound": "tensor", "kernel": f"IP-EOM sigma build ({args.eom_tier}, grouped tcgen05 launch)",
        "achieved": sig_alg * nprod if sig_alg else None, "peak": base * eratio,
        "unit": "TFLOP/s", "frac": (sig_alg * nprod / (base * eratio)) if sig_alg else None,
        "traffic": None, "algorithmic_tflops": sig_alg,
        "executed_products_per_term": nprod,
        "ms_per_build": sig_ms / max(sig_calls, 1), "builds_per_step": sig_calls / args.steps,
        "vectors_per_build": sig_vec / max(sig_calls, 1),
        "algorithmic_flops_per_build": sig_fl / max(sig_calls, 1),
        "peak_source": f"{src} bf16 sustained x {eratio} (of measured)",
    }
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{args.tier}/{args.eom_tier} tensor (c128 FP64 control)",
        "data": "synthetic",
        "config": workload_config(args.config, c, world),
        "roofline": roofline, "roofline_sigma": roofline_sigma,
        "fp64_comparator": fp64, "clocks": clocks.summary(), "gpu_launches": launches,
        "ladder_tflops": ladder_tf, "ccsd_iterations": ccsd_iters,
        "e_corr": [e.real, e.imag], "ips_eh": [float(x) for x in w.real],
        "kramers_max_split_eh": kramers_split, "wall_s_per_step": wall / args.steps,
        "e2e": e2e, "phase_ms_per_step": phases, "init_s": init_s,
    }
    if r == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(L, eps, o, ccsd_iters)
    if r == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
