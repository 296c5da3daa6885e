"""Microbenchmarks of single hot-path launches at a workload's bulk shapes.

    python -m paper_1908_09359_gb300.kernel_cases env3 --workload peps_24x24 [--chains N] [--reps R]

``step`` runs one full hot-path step (sweep, measurement, gradient, sign-SGD) of every
chain with per-launch timing and prints the contraction shapes by total device time.

``env3`` runs the three-line environment step (App. C) through the C ABI
(pepsvmc_env3_left) with bulk bond dimensions (all boundary bonds = Dc), the shape
that dominates the sweep; it prints the device time per step and the achieved
algorithmic FLOP/s (2 * (2 Dc^3 D^2 + Dc^2 D^4) per chain).  These are the small,
bounded cases that ncu captures use.
"""
from __future__ import annotations

import argparse
import json


def main():
    import torch

    from . import api, inputs
    p = argparse.ArgumentParser()
    p.add_argument("case", choices=["env3", "step"])
    p.add_argument("--top", type=int, default=25)
    p.add_argument("--workload", default="peps_24x24")
    p.add_argument("--chains", type=int, default=None)
    p.add_argument("--reps", type=int, default=10)
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "tf32", "bf16x3"])
    p.add_argument("--kernel", default="auto",
                   help="auto, or f32:CFG / tc:BN to fix every contraction's kernel")
    a = p.parse_args()

    def fix_kernel(ctx):
        if a.kernel != "auto":
            kind, tile = a.kernel.split(":")
            ctx.set_contraction_kernel(kind, int(tile))
    w = inputs.workload(a.workload, n_chains=1)
    n = a.chains or inputs.WORKLOADS[a.workload]["n_chains"]
    D, chi = w["D"], w["chi"]
    prec = api.PRECISIONS[a.precision]
    if a.case == "step":
        wl = inputs.workload(a.workload, n_chains=n)
        ctx = api.PepsVMC(wl["Ly"], wl["Lx"], D, chi, n, wl["tensors"], wl["sketch"], J1=wl["J1"], J2=wl["J2"],
                          seed=1, precision=prec)
        ctx.set_spins(wl["spins"])
        fix_kernel(ctx)
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
        print(json.dumps({"case": "step", "workload": a.workload, "precision": a.precision, "chains": n,
                          "step_ms": e0.elapsed_time(e1), "profiled_ms": total}))
        for r in rows[:a.top]:
            tf = r["flops"] / (r["ms"] / 1e3) / 1e12 if r["ms"] > 0 else 0.0
            print(f'{r["shape"]:32s} launches {r["launches"]:7d}  ms {r["ms"]:10.1f}  '
                  f'share {r["ms"] / total:6.3f}  TFLOP/s {tf:7.2f}')
        picks = {}
        for t in ctx.get_tuning():
            picks[t["choice"]] = picks.get(t["choice"], 0) + 1
        print("autotuner choices (kernel: shapes):", json.dumps(picks, sort_keys=True))
        ctx.close()
        return
    ctx = api.PepsVMC(w["Ly"], w["Lx"], D, chi, n, w["tensors"], w["sketch"], seed=1, precision=prec)
    fix_kernel(ctx)
    g = torch.Generator(device="cuda").manual_seed(0)
    r = lambda *s: torch.randn(*s, generator=g, device="cuda")  # noqa: E731
    E, T, B = r(n, chi, D, chi), r(n, chi, D, chi), r(n, chi, D, chi)
    A = r(2, D, D, D, D)
    spins = torch.where(torch.rand(n, generator=g, device="cuda") < 0.5, 1, -1).to(torch.int8)
    out = torch.empty(n, chi, D, chi, device="cuda")
    dims = (n, chi, chi, chi, chi, D, D, D, D)
    for _ in range(3):
        ctx.env3_left(E, T, A, spins, B, out, dims)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.reps):
        ctx.env3_left(E, T, A, spins, B, out, dims)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    flops = 2.0 * (2 * chi ** 3 * D ** 2 + chi ** 2 * D ** 4) * n
    print(json.dumps({"case": a.case, "workload": a.workload, "precision": a.precision, "chains": n,
                      "kernel": a.kernel, "ms_per_step": ms,
                      "tflops": flops / (ms / 1e3) / 1e12}))
    ctx.close()


if __name__ == "__main__":
    main()
