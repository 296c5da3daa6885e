#!/usr/bin/env python
"""Throughput of the VMC-PEPS hot path: samples/s of (Psi, E_loc, dlnPsi) on GB300.

One step = one pass of the whole hot path over every chain: a sequential Metropolis
sweep (boundary-MPS fits, three-line environments, ratios, decisions), fresh
environments of the final configurations, E_loc (three- and four-line ratios),
G = Delta/Psi, the float64 gradient sums and the sign-SGD update.  One sample = one
chain through one step.  The default workload is 24x24 J1-J2 (J2/J1 = 0.5), D=8,
Dc=32, 512 chains (seeded iid N(0,1) tensors standing in for optimised PEPS).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The JSON line carries the chosen form (split-BF16 tensor cores with the fused column
steps, batched chains, graph-replayed steps) and, in ``arms``, plain FP32 batched and
plain FP32 with one chain per launch, each with raw and effective samples/s (samples/s
over 2 tau_int) and the energy difference against the chosen form on the same
configurations.  Under torchrun every rank runs its own chains (weak scaling); the one
collective is the all-reduce of the float64 gradient sums before the identical sign-SGD
step of every rank.  Rank 0 prints one JSON line.

Measurement helpers (not part of the timed line):
    python bench.py --case env3|env4|step   one launch shape or one profiled step
    python bench.py --study mixing|cutoff|nnasp    plain vs learned sampler; convergence in Dc;
                                                  random-NNASP vs sequential sweep
"""
from __future__ import annotations

import argparse
import hashlib
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

# DRAM traffic of one bulk launch of each fused step (Dc 32, D 8), dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the kernel whose source hashed to
# `source_sha`, per chain of that capture; the bench reports it only while the source is
# unchanged.
NCU_TRAFFIC = {
    "fused4": {"bytes_per_chain": (167.906304e6 + 91.586304e6) / 512,
               "source": "paper_1908_09359_gb300/csrc/fused_env4.cu", "source_sha": "2cb0277a6c9307e6",
               "summary": "profiles/fused4_env4_bulk_peps24x24.md"},
    "fused3": {"bytes_per_chain": (201.532416e6 + 45.497088e6) / 2048,
               "source": "paper_1908_09359_gb300/csrc/fused_env3.cu", "source_sha": "49d7a78cd75df968",
               "summary": "profiles/fused3_env3_bulk_peps24x24.md"},
}


def parse(argv=None):
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
    p.add_argument("--no-arms", action="store_true", help="skip the plain-FP32 comparison arms")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle work per core for cpu_baseline")
    # measurement helpers
    p.add_argument("--case", choices=["env3", "env4", "step"], default=None)
    p.add_argument("--chains", type=int, default=None)
    p.add_argument("--reps", type=int, default=10)
    p.add_argument("--separate", action="store_true", help="--case env3/env4: three/four separate products")
    p.add_argument("--top", type=int, default=25)
    p.add_argument("--study", choices=["mixing", "cutoff", "nnasp"], default=None)
    p.add_argument("--structured", action="store_true", help="bond spectra exp(-i) instead of iid tensors")
    p.add_argument("--therm", type=int, default=50)
    p.add_argument("--sweeps", type=int, default=200)
    p.add_argument("--collect", type=int, default=100)
    p.add_argument("--epochs", type=int, default=20)
    p.add_argument("--lr", type=float, default=2e-3)
    p.add_argument("--arms", default="plain,learned")
    p.add_argument("--L", type=int, default=16)
    p.add_argument("--D", type=int, default=4)
    p.add_argument("--cutoffs", default="4,8,12,16,24,32")
    p.add_argument("--ref", type=int, default=64)
    p.add_argument("--cutoff-sweeps", type=int, default=10)
    return p.parse_args(argv)


# ------------------------------------------------------------------ multi-rank helpers

def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_share(w, rank, world):
    """One rank's share of a job of world x n_chains chains: its start configurations
    (a slice of the job's seeded starts) and the global index of its first chain (the
    chain word of the Philox counters), with the job's one key on every rank so that
    the sign-SGD draws -- and therefore the updated tensors -- are identical."""
    import numpy as np

    from paper_1908_09359_gb300 import inputs
    C = w["n_chains"]
    starts = inputs.start_spins(world * C, w["Ly"], w["Lx"], w["seed"], "random")
    return {"spins": np.ascontiguousarray(starts[rank * C:(rank + 1) * C]), "chain_offset": rank * C,
            "key": w["seed"]}


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


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(path)) if os.path.exists(path) else {}
    bf16 = (peaks.get("bf16_tflops_sustained"), "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)")
    if bf16[0] is None:
        bf16 = (1700.0, "fallback sustained bf16 1.7 PFLOP/s (of fallback)")
    hbm = (peaks.get("hbm_gbs"), "MEASURED_PEAKS.json hbm_gbs (of measured)")
    if hbm[0] is None:
        hbm = (6800.0, "fallback 6.8 TB/s (of fallback)")
    return bf16, hbm


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


def kernel_groups(shapes):
    """Per-launch-shape profile records -> totals per kernel: the fused four-line and
    three-line steps, the fit's fused optimal site, the separate tensor-core and FP32
    products, the QR and the per-chain reductions (normalisations, ratios, decisions)."""
    groups = {}
    for r in shapes:
        s = r["shape"]
        g = ("fused4" if s.startswith("fused4") else "fused3" if s.startswith("fused3") else
             "fusedP" if s.startswith("fusedP") else
             "gemm_tc" if s.startswith("gemm tc") else "gemm_f32" if s.startswith("gemm f32") else
             "qr" if s.startswith("qr") else "reductions" if r["flops"] == 0 else "other")
        acc = groups.setdefault(g, {"launches": 0, "flops": 0.0, "ms": 0.0})
        acc["launches"] += r["launches"]
        acc["flops"] += r["flops"]
        acc["ms"] += r["ms"]
    return groups


def source_sha(rel):
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


# ------------------------------------------------------------------ the oracle on the host

def oracle_bounded_sample(name, chain):
    """Seconds of FP64 oracle work for a bounded sample of one chain's sample step, and
    the fraction of a full sample that work stands for: one bulk-row truncation fit, one
    sampling row, one measurement row (three-line) and one row pair (four-line), each
    weighted by how often a step performs it."""
    import numpy as np

    from oracle import vmc
    from paper_1908_09359_gb300 import inputs
    w = inputs.workload(name, n_chains=1)
    Ly, Lx, chi = w["Ly"], w["Lx"], w["chi"]
    g = vmc.unpack(w["tensors"], Ly, Lx, w["D"])
    sp = np.array(inputs.start_spins(chain + 1, Ly, Lx, w["seed"], "random")[chain])
    k = min(3, Ly - 2)
    Ts, _ = vmc.top_envs(g, sp, chi, w["sketch"], 3, upto=k + 1)
    Bs = Ts  # any bond-saturated MPS of the right shape stands in for the bottom environment
    t0 = time.perf_counter()
    vmc.compress(vmc.mpo_times_mps(Ts[k], vmc.row_tensors(g, sp, k)), chi, w["sketch"], 3)
    t1 = time.perf_counter()
    vmc._sample_row(g, sp.copy(), k, Ts[k], Bs[k + 1], 1, chain, 0, 0, None)
    t2 = time.perf_counter()
    G = [[None] * Lx for _ in range(Ly)]
    vmc._row_terms(g, sp, k, Ts[k], Bs[k + 1], w["J1"], G, [0.0])
    t3 = time.perf_counter()
    vmc._pair_terms(g, sp, k, Ts[k], Bs[k + 1], w["J1"], w["J2"], [0.0])
    t4 = time.perf_counter()
    parts = (t1 - t0, t2 - t1, t3 - t2, t4 - t3)
    counts = (2 * (Lx - 1) + 2 * (Ly - 1) + (Ly - 1), Lx + Ly, Ly, Ly - 1)
    per_sample = sum(c * p for c, p in zip(counts, parts))
    return sum(parts), sum(parts) / per_sample, parts, counts


def _oracle_worker(job):
    name, chain, seconds = job
    work = frac = 0.0
    parts = counts = None
    while work < seconds:
        s, f, parts, counts = oracle_bounded_sample(name, chain)
        work += s
        frac += f
    return work, frac, parts, counts


def _one_thread():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[v] = "1"


def oracle_rate(name, procs, seconds):
    """Samples/s of the FP64 oracle with `procs` single-threaded processes (spawned),
    each running bounded samples of its own chain for about `seconds` of work; the
    chains are independent, so all cores work in parallel.  Returns a dict with
    value, cores, wall seconds and a description of the sample."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs, initializer=_one_thread) as pool:
        res = pool.map(_oracle_worker, [(name, c, seconds) for c in range(procs)])
    wall = time.perf_counter() - t0
    samples = sum(r[1] for r in res)
    parts, counts = res[0][2], res[0][3]
    desc = (f"{name}: {procs} single-threaded processes, one chain each, ~{seconds:.0f} s of work each, "
            "repeating one bounded sample = one bulk-row fit ({:.2f}s) x{}, one sampling row ({:.2f}s) x{}, "
            "one three-line measurement row ({:.2f}s) x{}, one four-line row pair ({:.2f}s) x{} of a full "
            "sample; samples counted as the fraction of a full sample done; rate = samples / wall "
            "(extrapolated from the bounded sample)").format(parts[0], counts[0], parts[1], counts[1], parts[2],
                                                              counts[2], parts[3], counts[3])
    return {"value": samples / wall, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": desc,
            "wall_s": wall, "samples_equivalent": samples}


def cpu_baselines(name, seconds):
    one = oracle_rate(name, 1, seconds)
    cores = os.cpu_count() or 1
    allc = oracle_rate(name, cores, seconds) if cores > 1 else one
    out = dict(allc)
    out["one_core"] = {"value": one["value"], "cores": 1, "wall_s": one["wall_s"]}
    return out


def run_reference(args):
    rank, world, _ = dist_info()
    if world > 1 and rank != 0:
        return
    from paper_1908_09359_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    cores = os.cpu_count() or 1
    per_step = max(2.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(args.workload, cores, per_step / 4)
    walls, samples, last = [], 0.0, None
    for _ in range(args.steps):
        last = oracle_rate(args.workload, cores, per_step)
        walls.append(last["wall_s"])
        samples += last["samples_equivalent"]
    wall = sum(walls)
    value = samples / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded iid N(0,1) PEPS tensors)",
        "config": {"workload": args.workload, "Ly": w["Ly"], "Lx": w["Lx"], "D": w["D"], "Dc": w["chi"],
                   "J2": w["J2"], "n_fit": 3,
                   "step": "a bounded sample of every core's chain (timed wall seconds per step in ms_per_step; "
                           "samples counted as the fraction of a full sample done)"},
        "timed_seconds": wall, "samples_equivalent": samples,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": last["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def make_ctx(w, n_chains, precision, share=None, chi=None, chi_measure=0, n_fit=3, tensors=None):
    from paper_1908_09359_gb300 import api, inputs
    chi_s = chi or w["chi"]
    chi_x = max(chi_s, chi_measure)
    sk = w["sketch"] if chi_x == w["chi"] else inputs.sketch(max(w["Ly"], w["Lx"]), chi_x, w["D"], w["seed"])
    share = share or {"key": w["seed"], "chain_offset": 0}
    ctx = api.PepsVMC(w["Ly"], w["Lx"], w["D"], chi_s, n_chains, w["tensors"] if tensors is None else tensors, sk,
                      J1=w["J1"], J2=w["J2"], seed=share["key"], n_fit=n_fit, precision=api.PRECISIONS[precision],
                      chi_measure=chi_measure, chain_offset=share["chain_offset"])
    return ctx


def timed_steps(ctx, steps, warmup, delta=1e-3, dist=None, collect=True, step0=0):
    """warmup + steps hot-path steps (energy_and_grad(1), the gradient-sum all-reduce
    when several ranks run, sign-SGD); CUDA events bracket the timed steps.  Returns
    (ms, eloc (steps, C), mz2 (steps, C), launches)."""
    import numpy as np
    import torch

    from paper_1908_09359_gb300 import autocorr, dist as xdist

    def step(i):
        r = ctx.energy_and_grad(1, want_samples=collect, want_grad=False)
        if dist:
            xdist.allreduce_device(ctx)
        ctx.update(delta, step0 + i)
        return r

    for i in range(warmup):
        step(i)
    stream = torch.cuda.current_stream()
    el, mz = [], []
    l0 = ctx.launches
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        r = step(warmup + i)
        if collect:
            el.append(r["eloc"])
            mz.append(autocorr.staggered_mz2(ctx.get_spins()))
    e1.record(stream)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), np.array(el), np.array(mz), ctx.launches - l0


def tau_of(el, mz):
    from paper_1908_09359_gb300 import autocorr
    if len(el) < 2:
        return None, None
    return autocorr.tau_int(el)[0], autocorr.tau_int(mz)[0]


def precision_gap(ctx_a, ctx_b, spins, N):
    """E_loc of the same configurations in two contexts: |dE_loc| / N, mean and max."""
    import numpy as np
    ctx_a.set_spins(spins)
    ctx_b.set_spins(spins)
    ea, _, _ = ctx_a.measure()
    eb, _, _ = ctx_b.measure()
    d = np.abs(ea - eb) / N
    return {"mean_abs_dE_per_site": float(d.mean()), "max_abs_dE_per_site": float(d.max()),
            "configs": int(len(d))}


def run_arms(args, w, chosen, spins_final, tau, C):
    """Plain FP32 batched, plain FP32 one chain per launch, and the precision gap of the
    chosen form on identical configurations (iid and bond-decay tensors)."""
    import numpy as np

    from paper_1908_09359_gb300 import inputs
    N = w["Ly"] * w["Lx"]
    arms = {}
    fp = make_ctx(w, C, "fp32", chi=args.chi, chi_measure=args.chi_measure, n_fit=args.n_fit)
    fp.set_spins(rank_share(w, 0, 1)["spins"])
    ms, _, _, _ = timed_steps(fp, 1, 2, collect=False)
    sps = C / (ms / 1e3)
    arms["plain_fp32_batched"] = {"samples_per_s": sps, "eff_samples_per_s": sps / (2 * tau) if tau else None,
                                  "chains_per_launch": C, "steps": 1, "warmup": 2, "ms_per_step": ms,
                                  "tau_int": tau, "tau_note": "the chosen form's tau_int (same transition rule)"}
    arms["precision_gap_iid"] = precision_gap(chosen, fp, spins_final, N)
    fp.close()
    one = make_ctx(w, 1, "fp32", chi=args.chi, chi_measure=args.chi_measure, n_fit=args.n_fit)
    one.set_spins(rank_share(w, 0, 1)["spins"][:1])
    ms, _, _, launches = timed_steps(one, 2, 2, collect=False)
    sps = 2 / (ms / 1e3)
    arms["plain_fp32_single_chain"] = {"samples_per_s": sps,
                                       "eff_samples_per_s": sps / (2 * tau) if tau else None,
                                       "chains_per_launch": 1, "steps": 2, "warmup": 2, "ms_per_step": ms / 2,
                                       "launches_per_step": launches / 2, "tau_int": tau}
    one.close()
    # bond spectra exp(-i) (App. A's simple-update form): the contraction is well
    # conditioned there, so the gap measures the precision, not chaos of the truncation
    sd = inputs.peps_tensors(w["Ly"], w["Lx"], w["D"], w["seed"], w["normalise"], bond_decay=1.0)
    nb = min(C, 64)
    a = make_ctx(w, nb, args.precision, chi=args.chi, chi_measure=args.chi_measure, n_fit=args.n_fit, tensors=sd)
    b = make_ctx(w, nb, "fp32", chi=args.chi, chi_measure=args.chi_measure, n_fit=args.n_fit, tensors=sd)
    a.set_spins(rank_share(w, 0, 1)["spins"][:nb])
    a.sample_sweep(2)
    arms["precision_gap_bond_decay"] = precision_gap(a, b, a.get_spins(), N)
    a.close()
    b.close()
    return arms


def run_ours(args):
    import ctypes as ct

    import numpy as np
    import torch

    from paper_1908_09359_gb300 import inputs
    rank, world, local = dist_info()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    w = inputs.workload(args.workload)
    C = w["n_chains"]
    N = w["Ly"] * w["Lx"]
    share = rank_share(w, rank, world)
    ctx = make_ctx(w, C, args.precision, share, args.chi, args.chi_measure, args.n_fit)
    ctx.set_spins(share["spins"])

    with Clocks(local) as clk:
        ms, el, mz, launches = timed_steps(ctx, args.steps, args.warmup, dist=dist)
    ms = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(world, C, args.steps, ms / 1e3)
    tau_e, tau_m = tau_of(el, mz)
    tau = max(tau_e, tau_m) if tau_e is not None else None
    spins_final = ctx.get_spins()

    # one further step with per-launch CUDA events on the library's stream (eager, so
    # the events sit between launches; the timed steps replay a CUDA graph)
    stream = torch.cuda.current_stream()
    ctx.set_profiling(True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    ctx.energy_and_grad(1, want_samples=False, want_grad=False)
    ctx.update(1e-3, 10 ** 6)
    pe1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.get_profile()
    shapes = ctx.get_profile_shapes()
    prof_step_ms = pe0.elapsed_time(pe1)
    ctx.set_profiling(False)

    e2e = None
    if not args.no_e2e:
        # through the C ABI with host buffers: the tensors uploaded from pinned memory,
        # E_loc / ln|Psi| / sign and the gradient read back, the updated tensors read back
        P = ctx.n_params
        pin = lambda n, dt: torch.empty(n, dtype=dt).pin_memory().numpy()  # noqa: E731
        host = dict(tensors=pin(P, torch.float64), eloc=pin(C, torch.float64), logpsi=pin(C, torch.float64),
                    sign=pin(C, torch.int8), grad=pin(P, torch.float64), out=pin(P, torch.float64))
        host["tensors"][:] = ctx.get_tensors()
        dp = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_double))  # noqa: E731
        from paper_1908_09359_gb300 import dist as xdist
        n_e2e = max(1, min(args.steps, 3))
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(n_e2e):
            ctx.set_tensors(host["tensors"])
            ctx._check(ctx.lib.pepsvmc_energy_and_grad(ctx.ctx, 1, None, None, dp(host["eloc"]), dp(host["logpsi"]),
                                                       host["sign"].ctypes.data_as(ct.POINTER(ct.c_int8)),
                                                       dp(host["grad"])))
            if dist:
                xdist.allreduce_device(ctx)
            ctx.update(1e-3, 2 * 10 ** 6 + i)
            ctx._check(ctx.lib.pepsvmc_get_tensors(ctx.ctx, dp(host["out"])))
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": whole_job_rate(world, C, n_e2e, max_over_ranks(e2e_s, dist, "cuda")), "unit": UNIT,
               "h2d_bytes_per_step": P * 8, "d2h_bytes_per_step": C * (8 + 8 + 1) + 2 * P * 8, "steps": n_e2e}

    if rank != 0:
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return

    (bf16, bf16_src), (hbm, hbm_src) = measured_peaks()
    groups = kernel_groups(shapes)
    contraction = {k: v for k, v in groups.items() if k not in ("qr", "reductions", "other")}
    dominant = max(contraction, key=lambda k: contraction[k]["ms"]) if contraction else None
    roofline = None
    if dominant:
        bulk = None
        if dominant in ("fused4", "fused3", "fusedP"):
            key = {"fused4": "fused4 32 32 32 32", "fused3": "fused3 32 32 32 32 x 8 8 8 8",
                   "fusedP": "fusedP 32 32 32 32 x 8 8 8 8"}[dominant]
            bulk = next((r for r in shapes if r["shape"] == key), None)
        rec = bulk or {"shape": dominant, **contraction[dominant]}
        per_launch_flops = rec["flops"] / rec["launches"]
        per_launch_ms = rec["ms"] / rec["launches"]
        if args.precision == "fp32":
            cpeak, csrc, cbound = FP32_ALU_PEAK_TFLOPS, "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived)", "alu"
        else:
            cpeak, csrc, cbound = bf16, bf16_src + "; algorithmic flops counted once (split BF16 issues three " \
                                                    "BF16 MMAs per product)", "tensor"
        # algorithmic bytes of one bulk fused launch: E, T, B and the result per chain in FP32
        chi, D = w["chi"], w["D"]
        nbytes = None
        if rec["shape"].startswith("fused4"):
            nbytes = 4.0 * C * (chi * D * D * chi * 2 + 2 * chi * D * chi)
        elif rec["shape"].startswith("fused3") or rec["shape"].startswith("fusedP"):
            nbytes = 4.0 * C * 4 * chi * D * chi
        # the binding roof of this kernel: HBM when its algorithmic intensity lies below the
        # ridge point of the compute peak, else the compute unit
        primary, other, _, _ = binding_roofline(per_launch_flops, nbytes or 0.0, per_launch_ms / 1e3,
                                                (cbound, cpeak, csrc), (hbm, hbm_src))
        traffic = None
        t = NCU_TRAFFIC.get(dominant)
        if t and rec is bulk and t["source_sha"] == source_sha(t["source"]):
            traffic = t["bytes_per_chain"] * C
        step_flops = prof["gemm_flops"]
        roofline = {
            "kernel": {"fused4": "env4_fused_kernel (four-line column step, tcgen05, split BF16)",
                       "fused3": "env3_fused_kernel (three-line column step, tcgen05, split BF16)",
                       "fusedP": "proj3_fused_kernel (optimal site of the truncation fit, tcgen05, split BF16)",
                       "gemm_tc": "gemm_tc_kernel (separate products, tcgen05)",
                       "gemm_f32": "gemm_f32_kernel (separate products, FP32 CUDA cores)"}[dominant],
            "shape": rec["shape"], "bound": primary["bound"], "achieved": primary["achieved"],
            "peak": primary["peak"], "unit": primary["unit"], "frac": primary["frac"],
            "peak_source": primary["peak_source"], "other_roof": other, "traffic": traffic,
            "traffic_source": (t["summary"] if traffic else "null: no ncu capture of this kernel source"),
            "flops_per_launch": per_launch_flops, "ms_per_launch": per_launch_ms,
            "algorithmic_bytes_per_launch": nbytes,
            "intensity_flop_per_byte": per_launch_flops / nbytes if nbytes else None,
            "ridge_flop_per_byte": cpeak * 1e12 / (hbm * 1e9), "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src,
            "launches_of_shape_per_step": rec["launches"],
            "step_contraction": {
                "algorithmic_flops": step_flops, "ms": prof["gemm_ms"],
                "tflops": step_flops / (prof["gemm_ms"] / 1e3) / 1e12 if prof["gemm_ms"] > 0 else None,
                "frac_of_peak": (step_flops / (prof["gemm_ms"] / 1e3) / 1e12) / cpeak if prof["gemm_ms"] > 0 else None,
                "method_frac": (step_flops / (prof_step_ms / 1e3) / 1e12) / cpeak,
                "method_frac_note": "all contraction flops of the step over the whole step's time",
                "share_of_step": prof["gemm_ms"] / prof_step_ms, "qr_ms": prof["qr_ms"],
                "profiled_step_ms": prof_step_ms,
                "shares": {k: v["ms"] / prof_step_ms for k, v in groups.items()},
            },
        }
    arms = None
    if not args.no_arms and world == 1:
        arms = run_arms(args, w, ctx, spins_final, tau, C)
        eff = value / (2 * tau) if tau else None
        if eff and arms["plain_fp32_single_chain"]["eff_samples_per_s"]:
            arms["chosen_over_single_chain_fp32_eff"] = eff / arms["plain_fp32_single_chain"]["eff_samples_per_s"]
            arms["chosen_over_batched_fp32_eff"] = eff / arms["plain_fp32_batched"]["eff_samples_per_s"]
    ctx.close()
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baselines(args.workload, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16 operands, f32 accumulate",
                                      "tf32": "tf32 operands, f32 accumulate",
                                      "bf16x3": "bf16 hi+lo operands, f32 accumulate"}[args.precision],
        "data": "synthetic (seeded iid N(0,1) PEPS tensors, random S^z=0 starts)",
        "config": {"workload": args.workload, "Ly": w["Ly"], "Lx": w["Lx"], "D": w["D"], "Dc": args.chi or w["chi"],
                   "Dc_measure": args.chi_measure or args.chi or w["chi"],
                   "J1": w["J1"], "J2": w["J2"], "chains_per_gpu": C, "n_fit": args.n_fit,
                   "form": {"fp32": "plain FP32", "bf16": "mixed BF16 (tcgen05)", "tf32": "mixed TF32 (tcgen05)",
                            "bf16x3": "mixed split-BF16 (tcgen05, fused column steps)"}[args.precision],
                   "step": "sweep + measure + gradient sums (+ all-reduce when N > 1) + sign-SGD",
                   "l2": "working set (boundary-MPS caches, GBs) larger than L2; no flush"},
        "tau_int": {"eloc": tau_e, "mz2": tau_m, "samples": int(el.size) if len(el) else 0,
                    "estimator": "Sokal automatic window (c = 5) on the chain-averaged autocovariance of the "
                                 "timed steps"},
        "eff_samples_per_s": value / (2 * tau) if tau else None,
        "roofline": roofline, "arms": arms, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ measurement helpers

def run_case(args):
    """--case env3 / env4: one bulk launch shape of the three- or four-line step through
    the C ABI (the small, bounded cases that ncu captures use); --case step: one profiled
    hot-path step with the per-shape device-time table."""
    import torch

    from paper_1908_09359_gb300 import api, inputs
    w = inputs.workload(args.workload, n_chains=1)
    n = args.chains or inputs.WORKLOADS[args.workload]["n_chains"]
    D, chi = w["D"], w["chi"]
    prec = api.PRECISIONS[args.precision]
    if args.case == "step":
        wl = inputs.workload(args.workload, n_chains=n)
        ctx = api.PepsVMC(wl["Ly"], wl["Lx"], D, chi, n, wl["tensors"], wl["sketch"], J1=wl["J1"], J2=wl["J2"],
                          seed=1, precision=prec)
        ctx.set_spins(wl["spins"])
        ctx.set_fused(not args.separate)
        ctx.energy_and_grad(1, want_samples=False, want_grad=False)
        ctx.set_profiling(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.energy_and_grad(1, want_samples=False, want_grad=False)
        ctx.update(1e-3, 1)
        e1.record()
        torch.cuda.synchronize()
        rows = sorted(ctx.get_profile_shapes(), key=lambda r: -r["ms"])
        total = sum(r["ms"] for r in rows)
        print(json.dumps({"case": "step", "workload": args.workload, "precision": args.precision, "chains": n,
                          "step_ms": e0.elapsed_time(e1), "profiled_ms": total}))
        for r in rows[:args.top]:
            tf = r["flops"] / (r["ms"] / 1e3) / 1e12 if r["ms"] > 0 else 0.0
            print(f'{r["shape"]:32s} launches {r["launches"]:7d}  ms {r["ms"]:10.1f}  '
                  f'share {r["ms"] / total:6.3f}  TFLOP/s {tf:7.2f}')
        ctx.close()
        return
    ctx = api.PepsVMC(w["Ly"], w["Lx"], D, chi, n, w["tensors"], w["sketch"], seed=1, precision=prec)
    ctx.set_fused(not args.separate)
    g = torch.Generator(device="cuda").manual_seed(0)
    r = lambda *s: torch.randn(*s, generator=g, device="cuda")  # noqa: E731
    spins = torch.where(torch.rand(n, generator=g, device="cuda") < 0.5, 1, -1).to(torch.int8)
    if args.case == "env3":
        E, T, B, A = r(n, chi, D, chi), r(n, chi, D, chi), r(n, chi, D, chi), r(2, D, D, D, D)
        out = torch.empty(n, chi, D, chi, device="cuda")
        dims = (n, chi, chi, chi, chi, D, D, D, D)
        run = lambda: ctx.env3_left(E, T, A, spins, B, out, dims)  # noqa: E731
        flops = 2.0 * (2 * chi ** 3 * D ** 2 + chi ** 2 * D ** 4) * n
    else:
        E, T, B = r(n, chi, D, D, chi), r(n, chi, D, chi), r(n, chi, D, chi)
        A1, A2 = r(2, D, D, D, D), r(2, D, D, D, D)
        out = torch.empty(n, chi, D, D, chi, device="cuda")
        dims = (n, chi, chi, chi, chi, D, D, D, D, D, D, D)
        # the engine's own layout of four-line environments when its steps are fused
        run = lambda: ctx.env4_left(E, T, A1, spins, A2, spins, B, out, dims, bmajor=not args.separate)  # noqa: E731
        flops = 2.0 * (2 * chi ** 3 * D ** 3 + 2 * chi ** 2 * D ** 5) * n
    for _ in range(3):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    print(json.dumps({"case": args.case, "workload": args.workload, "precision": args.precision, "chains": n,
                      "fused": not args.separate, "ms_per_launch": ms, "tflops": flops / (ms / 1e3) / 1e12}))
    ctx.close()


def _mixing_arm(ctx, start, sweep0, sweeps, N):
    import numpy as np

    from paper_1908_09359_gb300 import autocorr
    ctx.set_spins(start)
    ctx.set_sweep_counter(sweep0)
    el = np.empty((sweeps, ctx.n_chains))
    mz = np.empty((sweeps, ctx.n_chains))
    secs = 0.0
    for t in range(sweeps):
        t0 = time.perf_counter()
        r = ctx.energy_and_grad(1, want_samples=True, want_grad=True)
        secs += time.perf_counter() - t0
        el[t] = r["eloc"]
        mz[t] = autocorr.staggered_mz2(ctx.get_spins())
    e_mean, e_err = autocorr.mean_and_error(el / N)
    tau_e, _ = autocorr.tau_int(el)
    tau_m, _ = autocorr.tau_int(mz)
    sps = sweeps * ctx.n_chains / secs
    tau = max(tau_e, tau_m)
    return dict(E_per_site=e_mean, E_err=e_err, tau_eloc=tau_e, tau_mz2=tau_m, Mz2=float(mz.mean()),
                s_per_step=secs / sweeps, samples_per_s=sps, eff_samples_per_s=sps / (2 * tau))


def study_mixing(args):
    """Plain sequential sampler against plain + learned band moves from the same
    thermalised configurations, one sample per chain per step through
    pepsvmc_energy_and_grad: E per site with its tau-corrected error, tau_int of E_loc
    and of M_z^2, raw and effective samples/s.  The network is trained first on the
    plain sampler's configurations (one-off cost reported separately)."""
    import numpy as np

    from paper_1908_09359_gb300 import api, inputs
    arms = args.arms.split(",")
    w = inputs.workload(args.workload, n_chains=args.chains)
    Ly, Lx, D, chi, C = w["Ly"], w["Lx"], w["D"], w["chi"], w["n_chains"]
    if args.structured:
        w["tensors"] = inputs.peps_tensors(Ly, Lx, D, w["seed"], inputs.WORKLOADS[args.workload].get("normalise", False),
                                           bond_decay=1.0)
    N = Ly * Lx
    ctx = api.PepsVMC(Ly, Lx, D, chi, C, w["tensors"], w["sketch"], J1=w["J1"], J2=w["J2"], seed=w["seed"],
                      precision=api.PRECISIONS[args.precision])
    ctx.set_spins(w["spins"])
    ctx.sample_sweep(args.therm)
    start, sweep0 = ctx.get_spins(), ctx.sweep_counter
    base = dict(study="mixing", workload=args.workload, precision=args.precision, chains=C, sweeps=args.sweeps,
                therm=args.therm, tensors="structured" if args.structured else "iid")
    plain = _mixing_arm(ctx, start, sweep0, args.sweeps, N) if "plain" in arms else None
    if plain:
        print(json.dumps(dict(arm="plain", **base, **plain)), flush=True)
    if "learned" not in arms:
        ctx.close()
        return
    ctx.set_spins(start)
    ctx.set_sweep_counter(sweep0 + 10 ** 6)
    ctx.set_proposal_params(inputs.proposal_params(w["seed"]))
    t0 = time.perf_counter()
    n_train = ctx.proposal_collect(args.collect)
    t1 = time.perf_counter()
    loss0 = ctx.proposal_train(1, 256, args.lr)
    loss = ctx.proposal_train(args.epochs - 1, 256, args.lr) if args.epochs > 1 else loss0
    t2 = time.perf_counter()
    ctx.set_spins(start)
    ctx.amplitude(0)
    acc = ctx.learned_sweep(4)
    ctx.set_proposal(1)
    learned = _mixing_arm(ctx, start, sweep0, args.sweeps, N)
    print(json.dumps(dict(arm="learned", **base, **learned, train_configs=n_train, collect_s=t1 - t0,
                          train_s=t2 - t1, loss_first_epoch=loss0, loss_last_epoch=loss,
                          learned_accept=acc)), flush=True)
    if plain:
        dE = learned["E_per_site"] - plain["E_per_site"]
        sig = float(np.hypot(learned["E_err"], plain["E_err"]))
        print(json.dumps(dict(summary=True, **base, dE_per_site=dE, dE_sigma=dE / sig if sig > 0 else 0.0,
                              eff_speedup=learned["eff_samples_per_s"] / plain["eff_samples_per_s"],
                              raw_speedup=learned["samples_per_s"] / plain["samples_per_s"])), flush=True)
    ctx.close()


def study_nnasp(args):
    """The paper's check of the sequential sweep (Sec. II A, Fig. SweepScheme): the random
    NNASP scheme (N uniformly chosen antiparallel-pair attempts per sweep, Eq. (prob_r))
    and the sequential sweep run from the same thermalised configurations; per scheme E
    per site with its tau-corrected error, tau_int of E_loc and M_z^2, sweeps/s and
    effective samples/s, and the difference of the two energies in units of its error."""
    import numpy as np

    from paper_1908_09359_gb300 import api, autocorr, inputs
    w = inputs.workload(args.workload, n_chains=args.chains)
    Ly, Lx, D, chi, C = w["Ly"], w["Lx"], w["D"], w["chi"], w["n_chains"]
    if args.structured:
        w["tensors"] = inputs.peps_tensors(Ly, Lx, D, w["seed"], inputs.WORKLOADS[args.workload].get("normalise", False),
                                           bond_decay=1.0)
    N = Ly * Lx
    ctx = api.PepsVMC(Ly, Lx, D, chi, C, w["tensors"], w["sketch"], J1=w["J1"], J2=w["J2"], seed=w["seed"],
                      precision=api.PRECISIONS[args.precision])
    ctx.set_spins(w["spins"])
    ctx.sample_sweep(args.therm)
    start, sweep0 = ctx.get_spins(), ctx.sweep_counter
    base = dict(study="nnasp", workload=args.workload, precision=args.precision, chains=C, sweeps=args.sweeps,
                therm=args.therm, tensors="structured" if args.structured else "iid")
    out = {}
    for scheme in ("sequential", "random"):
        ctx.set_spins(start)
        ctx.set_sweep_counter(sweep0)
        el, mz, secs = np.empty((args.sweeps, C)), np.empty((args.sweeps, C)), 0.0
        for t in range(args.sweeps):
            t0 = time.perf_counter()
            (ctx.sample_sweep if scheme == "sequential" else ctx.random_sweep)(1)
            e, _, _ = ctx.measure()
            secs += time.perf_counter() - t0
            el[t] = e
            mz[t] = autocorr.staggered_mz2(ctx.get_spins())
        mean, err = autocorr.mean_and_error(el / N)
        tau = max(autocorr.tau_int(el)[0], autocorr.tau_int(mz)[0])
        sps = args.sweeps * C / secs
        out[scheme] = dict(E_per_site=mean, E_err=err, tau_eloc=autocorr.tau_int(el)[0],
                           tau_mz2=autocorr.tau_int(mz)[0], Mz2=float(mz.mean()), samples_per_s=sps,
                           eff_samples_per_s=sps / (2 * tau))
        print(json.dumps(dict(scheme=scheme, **base, **out[scheme])), flush=True)
    d = out["random"]["E_per_site"] - out["sequential"]["E_per_site"]
    sig = float(np.hypot(out["random"]["E_err"], out["sequential"]["E_err"]))
    print(json.dumps(dict(summary=True, **base, dE_per_site=d, dE_sigma=d / sig if sig > 0 else 0.0,
                          eff_ratio_sequential_over_random=out["sequential"]["eff_samples_per_s"]
                          / out["random"]["eff_samples_per_s"])), flush=True)
    ctx.close()


def study_cutoff(args):
    """Convergence in the boundary cutoff Dc (App. D): eps = |Psi_Dc / Psi_ref - 1| and
    |E_loc,Dc - E_loc,ref| / max(|E_loc,ref|, 1) per configuration against a much larger
    reference cutoff, on configurations the plain sampler draws at the reference cutoff."""
    import numpy as np

    from paper_1908_09359_gb300 import api, inputs
    L, D, C, ref = args.L, args.D, args.chains or 128, args.ref
    seed = inputs.SEED_BASE + 100 + L
    t = inputs.peps_tensors(L, L, D, seed, True, bond_decay=1.0 if args.structured else 0.0)
    sk = inputs.sketch(L, ref, D, seed)
    prec = api.PRECISIONS[args.precision]

    def measure(chi, spins):
        ctx = api.PepsVMC(L, L, D, chi, C, t, np.ascontiguousarray(sk[:, :chi, :, :chi]), seed=seed, precision=prec)
        ctx.set_spins(spins)
        e, lp, sg = ctx.measure()
        ctx.close()
        return e, lp, sg

    ctx = api.PepsVMC(L, L, D, ref, C, t, sk, seed=seed, precision=prec)
    ctx.set_spins(inputs.start_spins(C, L, L, seed, "random"))
    ctx.sample_sweep(args.cutoff_sweeps)
    spins = ctx.get_spins()
    e_ref, lp_ref, sg_ref = ctx.measure()
    ctx.close()
    for chi in [int(x) for x in args.cutoffs.split(",")]:
        e, lp, sg = measure(chi, spins)
        eps = np.abs(sg * sg_ref * np.exp(lp - lp_ref) - 1.0)
        de = np.abs(e - e_ref) / np.maximum(np.abs(e_ref), 1.0)
        print(json.dumps({"study": "cutoff", "L": L, "D": D, "Dc": chi, "Dc_ref": ref,
                          "tensors": "structured" if args.structured else "iid", "configs": C,
                          "eps_median": float(np.median(eps)), "eps_max": float(np.max(eps)),
                          "dEloc_median": float(np.median(de)), "dEloc_max": float(np.max(de)),
                          "sign_flips": int(np.sum(sg != sg_ref))}), flush=True)


def main(argv=None):
    args = parse(argv)
    if args.case:
        run_case(args)
    elif args.study == "mixing":
        study_mixing(args)
    elif args.study == "cutoff":
        study_cutoff(args)
    elif args.study == "nnasp":
        study_nnasp(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
