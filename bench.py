#!/usr/bin/env python
"""Throughput of the VMC-PEPS hot path: samples/s of (Psi, E_loc, dlnPsi) on GB300.

One step = one pass of the whole hot path over every chain: a sequential Metropolis
sweep (boundary-MPS fits, three-line environments, ratios, decisions), fresh
environments of the final configurations, E_loc (three- and four-line ratios),
G = Delta/Psi, the float64 gradient sums and the sign-SGD update.  One sample = one
chain through one step.  The default workload is 24x24 J1-J2 (J2/J1 = 0.5), D=8,
Dc=32, 512 chains (seeded iid N(0,1) tensors standing in for optimised PEPS).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own chains (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "samples/s (Ψ, E_loc, ∂lnΨ) on 1 GB300 at 24×24 D=8; plain FP32 vs chosen form"
UNIT = "samples/s"
# FP32 CUDA-core peak of one GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz.
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="peps_24x24")
    p.add_argument("--n-fit", type=int, default=3)
    p.add_argument("--precision", default="bf16x3", choices=["fp32", "bf16", "tf32", "bf16x3"],
                   help="bf16x3 (split-BF16 tensor cores, the chosen form) or fp32 (plain)")
    p.add_argument("--chi", type=int, default=None, help="sampling cutoff Dc1 (default: the workload's Dc)")
    p.add_argument("--chi-measure", type=int, default=0,
                   help="measurement cutoff Dc2 (default 0: the same as the sampling cutoff)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_seeds(w, rank):
    """One rank's share of the workload: the tensors are replicated, every rank runs its
    own n_chains chains with its own start configurations and Metropolis key (weak
    scaling over independent Markov chains; no data-path collective)."""
    return {"spins": w["seed"] + 7919 * rank, "key": w["seed"] + rank}


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (timings: the job is as slow as its slowest rank)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, chains_per_rank, steps, seconds):
    """Samples/s of the whole job: every rank's chains over the slowest rank's time."""
    return world * chains_per_rank * steps / seconds


class Clocks:
    """nvidia-smi samples (every 200 ms) of one GPU during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.lines, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def binding_roofline(flops, nbytes, seconds, compute_peak, hbm_peak):
    """(binding roof, other roof, flop per byte, ridge) of a kernel that did `flops`
    algorithmic flops over `nbytes` algorithmic bytes in `seconds`.  compute_peak =
    (bound name, TFLOP/s, source), hbm_peak = (GB/s, source).  The binding roof is HBM
    when the intensity lies below the ridge point of the compute peak, else the compute
    unit; each roof carries achieved, peak, unit and frac = achieved / peak."""
    cbound, cpeak, csrc = compute_peak
    hbm, hsrc = hbm_peak
    intensity = flops / nbytes if nbytes > 0 else None
    ridge = cpeak * 1e12 / (hbm * 1e9)
    compute = {"bound": cbound, "achieved": flops / seconds / 1e12 if seconds > 0 else None, "peak": cpeak,
               "unit": "TFLOP/s", "peak_source": csrc}
    compute["frac"] = compute["achieved"] / cpeak if compute["achieved"] else None
    memory = {"bound": "hbm", "achieved": nbytes / seconds / 1e9 if seconds > 0 else None, "peak": hbm,
              "unit": "GB/s", "peak_source": hsrc}
    memory["frac"] = memory["achieved"] / hbm if memory["achieved"] else None
    if intensity is not None and intensity < ridge:
        return memory, compute, intensity, ridge
    return compute, memory, intensity, ridge


def oracle_sample_seconds(name, reps=1):
    """Seconds per sample of the FP64 oracle on this host, from a bounded sample of the
    workload: one bulk-row truncation fit, one sampling row, one measurement row (three-
    line) and one row pair (four-line), each timed once on one chain and weighted by how
    often a step performs it.  Returns (seconds, description, threads)."""
    import numpy as np

    from oracle import vmc
    from paper_1908_09359_gb300 import inputs
    w = inputs.workload(name, n_chains=1)
    Ly, Lx, chi = w["Ly"], w["Lx"], w["chi"]
    g = vmc.unpack(w["tensors"], Ly, Lx, w["D"])
    sp = np.array(w["spins"][0])
    k = min(3, Ly - 2)
    Ts, _ = vmc.top_envs(g, sp, chi, w["sketch"], 3, upto=k + 1)
    Bs = Ts  # any bond-saturated MPS of the right shape stands in for the bottom environment
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        vmc.compress(vmc.mpo_times_mps(Ts[k], vmc.row_tensors(g, sp, k)), chi, w["sketch"], 3)
        t1 = time.perf_counter()
        vmc._sample_row(g, sp.copy(), k, Ts[k], Bs[k + 1], 1, 0, 0, 0, None)
        t2 = time.perf_counter()
        G = [[None] * Lx for _ in range(Ly)]
        vmc._row_terms(g, sp, k, Ts[k], Bs[k + 1], w["J1"], G, [0.0])
        t3 = time.perf_counter()
        vmc._pair_terms(g, sp, k, Ts[k], Bs[k + 1], w["J1"], w["J2"], [0.0])
        t4 = time.perf_counter()
        cur = (t1 - t0, t2 - t1, t3 - t2, t4 - t3)
        best = cur if best is None or sum(cur) < sum(best) else best
    n_fit = 2 * (Lx - 1) + 2 * (Ly - 1) + (Ly - 1)   # two sweep phases x two directions + fresh bottom
    per_sample = n_fit * best[0] + (Lx + Ly) * best[1] + Ly * best[2] + (Ly - 1) * best[3]
    desc = (f"{name}, 1 chain: one bulk-row fit ({best[0]:.2f}s) x{n_fit}, one sampling row "
            f"({best[1]:.2f}s) x{Lx + Ly}, one three-line measurement row ({best[2]:.2f}s) x{Ly}, one "
            f"four-line row pair ({best[3]:.2f}s) x{Ly - 1}; summed = s/sample")
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count()
    return per_sample, desc, threads, sum(best)


def run_reference(args):
    rank, world, _ = dist_info()
    if world > 1 and rank != 0:
        return
    from paper_1908_09359_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_sample_seconds(args.workload)
    per = []
    cpu = None
    for _ in range(args.steps):
        s, desc, threads, work = oracle_sample_seconds(args.workload)
        per.append(s)
        cpu = (desc, threads, work)
    sec = statistics.median(per)
    value = 1.0 / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded iid N(0,1) PEPS tensors)",
        "config": {"workload": args.workload, "Ly": w["Ly"], "Lx": w["Lx"], "D": w["D"], "Dc": w["chi"],
                   "J2": w["J2"], "chains": 1, "n_fit": 3},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu[1], "kind": "oracle", "sample": cpu[0]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1908_09359_gb300 import api, inputs
    rank, world, local = dist_info()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    w = inputs.workload(args.workload)
    C = w["n_chains"]
    seeds = rank_seeds(w, rank)
    spins = inputs.start_spins(C, w["Ly"], w["Lx"], seeds["spins"], "random")
    prec = api.PRECISIONS[args.precision]
    chi_s = args.chi or w["chi"]
    chi_x = max(chi_s, args.chi_measure)
    sk = w["sketch"] if chi_x == w["chi"] else inputs.sketch(max(w["Ly"], w["Lx"]), chi_x, w["D"], w["seed"])
    ctx = api.PepsVMC(w["Ly"], w["Lx"], w["D"], chi_s, C, w["tensors"], sk, J1=w["J1"],
                      J2=w["J2"], seed=seeds["key"], n_fit=args.n_fit, precision=prec, chi_measure=args.chi_measure)
    ctx.set_spins(spins)
    delta = 1e-3

    def step(i, host=None):
        if host is None:
            ctx.energy_and_grad(1, want_samples=False, want_grad=False)
        else:
            ctx.set_tensors(host["tensors"])
            ctx._check(ctx.lib.pepsvmc_energy_and_grad(ctx.ctx, 1, None, None, host["p_eloc"],
                                                       host["p_logpsi"], host["p_sign"], host["p_grad"]))
        ctx.update(delta, i)
        if host is not None:
            ctx._check(ctx.lib.pepsvmc_get_tensors(ctx.ctx, host["p_tensors"]))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        step(i)
    stream = torch.cuda.current_stream()
    l0 = ctx.launches
    barrier()
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        e1.record(stream)
        barrier()
    launches = ctx.launches - l0
    ms = e0.elapsed_time(e1)
    # Roofline of the contraction kernel: one more step with every contraction launch
    # bracketed by CUDA events on the library's stream (eager, so the events can sit
    # between launches; the timed steps above replay a CUDA graph without them).
    ctx.set_profiling(True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    step(args.warmup + args.steps)
    pe1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.get_profile()
    prof_step_ms = pe0.elapsed_time(pe1)
    ctx.set_profiling(False)
    ms = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(world, C, args.steps, ms / 1e3)

    e2e = None
    if not args.no_e2e:
        import ctypes as ct
        P = ctx.n_params
        pin = lambda n, dt: torch.empty(n, dtype=dt).pin_memory().numpy()  # noqa: E731
        host = dict(tensors=pin(P, torch.float64), eloc=pin(C, torch.float64), logpsi=pin(C, torch.float64),
                    sign=pin(C, torch.int8), grad=pin(P, torch.float64), out=pin(P, torch.float64))
        host["tensors"][:] = ctx.get_tensors()
        dp = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))  # noqa: E731
        host.update(p_eloc=dp(host["eloc"]), p_logpsi=dp(host["logpsi"]),
                    p_sign=host["sign"].ctypes.data_as(ct.POINTER(ct.c_int8)), p_grad=dp(host["grad"]),
                    p_tensors=dp(host["out"]))
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            step(args.warmup + args.steps + 1 + i, host)
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": whole_job_rate(world, C, args.steps, max_over_ranks(e2e_s, dist, "cuda")), "unit": UNIT,
               "h2d_bytes_per_step": P * 8,
               "d2h_bytes_per_step": C * (8 + 8 + 1) + 2 * P * 8}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    step_ms = ms / args.steps
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm, hbm_src = peaks.get("hbm_gbs"), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    if hbm is None:
        hbm, hbm_src = 6800.0, "fallback 6.8 TB/s (of fallback)"
    if args.precision == "fp32":
        kname = "gemm_f32_kernel (batched contraction, FP32 CUDA cores)"
        cbound, cpeak = "alu", FP32_ALU_PEAK_TFLOPS
        csrc = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived)"
    else:
        bf16 = peaks.get("bf16_tflops_sustained")
        src = "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
        if bf16 is None:
            bf16, src = 1700.0, "fallback sustained bf16 1.7 PFLOP/s (of fallback)"
        # TF32 dense rate is half the BF16 rate; split BF16 issues three BF16 MMAs per
        # product, so its algorithmic flops are reported against a third of the BF16 peak
        cpeak = {"bf16": bf16, "tf32": bf16 / 2.0, "bf16x3": bf16 / 3.0}[args.precision]
        kname = ("gemm_tc_kernel (batched contraction, tcgen05 "
                 + {"bf16": "kind::f16", "tf32": "kind::tf32", "bf16x3": "kind::f16, split hi+lo, 3 MMAs"}[
                     args.precision] + ", tile autotuned per shape)")
        cbound = "tensor"
        csrc = src + {"bf16": "", "tf32": " x 1/2 for TF32", "bf16x3": " x 1/3 for three BF16 MMAs"}[args.precision]
    bind, other, intensity, ridge = binding_roofline(prof["gemm_flops"], prof["gemm_bytes"], prof["gemm_ms"] / 1e3,
                                                     (cbound, cpeak, csrc), (hbm, hbm_src))
    flops, nbytes = prof["gemm_flops"], prof["gemm_bytes"]
    roofline = {
        "kernel": kname, "bound": bind["bound"], "achieved": bind["achieved"], "peak": bind["peak"],
        "unit": bind["unit"], "frac": bind["frac"], "peak_source": bind["peak_source"],
        "traffic": None,
        "intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge,
        "other_roof": other,
        "algorithmic_flops_per_step": flops, "algorithmic_bytes_per_step": nbytes,
        "share_of_step": prof["gemm_ms"] / prof_step_ms,
        "launches": prof["gemm_launches"],
        "qr_ms_per_step": prof["qr_ms"],
        "measured_on": "one extra eager step with per-launch CUDA events on the library's stream (ms %.0f)"
                       % prof_step_ms,
    }
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        s, desc, threads, _ = oracle_sample_seconds(args.workload)
        cpu = {"value": 1.0 / s, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16 operands, f32 accumulate",
                                      "tf32": "tf32 operands, f32 accumulate",
                                      "bf16x3": "bf16 hi+lo operands, f32 accumulate"}[args.precision],
        "data": "synthetic (seeded iid N(0,1) PEPS tensors, random S^z=0 starts)",
        "config": {"workload": args.workload, "Ly": w["Ly"], "Lx": w["Lx"], "D": w["D"], "Dc": chi_s,
                   "Dc_measure": args.chi_measure or chi_s,
                   "J1": w["J1"], "J2": w["J2"], "chains_per_gpu": C, "n_fit": args.n_fit,
                   "form": {"fp32": "plain FP32", "bf16": "mixed BF16 (tcgen05)", "tf32": "mixed TF32 (tcgen05)",
                            "bf16x3": "mixed split-BF16 (tcgen05)"}[args.precision], "step": "sweep + measure + gradient sums + sign-SGD",
                   "l2": "working set (boundary-MPS caches, GBs) larger than L2; no flush"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
