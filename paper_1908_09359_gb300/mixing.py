"""Mixing study: plain sequential sampler against plain + learned band moves.

    python -m paper_1908_09359_gb300.mixing --workload peps_8x8 --sweeps 200

Both arms start from the same thermalised configurations and run the full sample step
(sweep, fresh environments, E_loc, G) through pepsvmc_energy_and_grad, one sample per
chain per step.  For each arm it reports the energy per site with its tau-corrected
error, tau_int of E_loc and of the squared staggered magnetisation (Sec. III's M_z^2),
the raw samples/s and the effective independent samples/s = samples/s / (2 max tau).
The learned arm's network is first trained on configurations of the plain sampler
(pepsvmc_proposal_collect + pepsvmc_proposal_train); that one-off cost is reported
separately.  Output: one JSON line per arm and a summary line.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np


def run_arm(ctx, start, sweep0, sweeps, N):
    ctx.set_spins(start)
    ctx.set_sweep_counter(sweep0)
    el = np.empty((sweeps, ctx.n_chains))
    mz = np.empty((sweeps, ctx.n_chains))
    secs = 0.0
    from . import autocorr
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


def main():
    from . import api, inputs
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="peps_8x8")
    p.add_argument("--chains", type=int, default=None)
    p.add_argument("--precision", default="fp32", choices=sorted(api.PRECISIONS))
    p.add_argument("--structured", action="store_true",
                   help="simple-update-like bond spectra (lambda_i = exp(-i)) instead of iid tensors")
    p.add_argument("--therm", type=int, default=50)
    p.add_argument("--sweeps", type=int, default=200)
    p.add_argument("--collect", type=int, default=100, help="plain sweeps whose configurations train the net")
    p.add_argument("--epochs", type=int, default=20)
    p.add_argument("--batch", type=int, default=256)
    p.add_argument("--lr", type=float, default=2e-3)
    p.add_argument("--arms", default="plain,learned", help="plain, learned or both (comma separated)")
    a = p.parse_args()
    arms = a.arms.split(",")
    w = inputs.workload(a.workload, n_chains=a.chains)
    Ly, Lx, D, chi, C = w["Ly"], w["Lx"], w["D"], w["chi"], w["n_chains"]
    if a.structured:
        w["tensors"] = inputs.peps_tensors(Ly, Lx, D, w["seed"], inputs.WORKLOADS[a.workload].get("normalise", False),
                                           bond_decay=1.0)
    N = Ly * Lx
    ctx = api.PepsVMC(Ly, Lx, D, chi, C, w["tensors"], w["sketch"], J1=w["J1"], J2=w["J2"], seed=w["seed"],
                      precision=api.PRECISIONS[a.precision],
                      stream=0 if os.environ.get("PEPSVMC_DRY_RUN") == "1" else None)
    ctx.set_spins(w["spins"])
    ctx.sample_sweep(a.therm)
    start, sweep0 = ctx.get_spins(), ctx.sweep_counter
    base = dict(workload=a.workload, precision=a.precision, chains=C, sweeps=a.sweeps, therm=a.therm,
                tensors="structured" if a.structured else "iid")

    plain = run_arm(ctx, start, sweep0, a.sweeps, N) if "plain" in arms else None
    if plain:
        print(json.dumps(dict(arm="plain", **base, **plain)), flush=True)
    if "learned" not in arms:
        ctx.close()
        return

    ctx.set_spins(start)
    ctx.set_sweep_counter(sweep0 + 10 ** 6)
    ctx.set_proposal_params(inputs.proposal_params(w["seed"]))
    t0 = time.perf_counter()
    n_train = ctx.proposal_collect(a.collect)
    t1 = time.perf_counter()
    loss0 = ctx.proposal_train(1, a.batch, a.lr)
    loss = ctx.proposal_train(a.epochs - 1, a.batch, a.lr) if a.epochs > 1 else loss0
    t2 = time.perf_counter()
    ctx.set_spins(start)
    ctx.amplitude(0)
    acc = ctx.learned_sweep(4)
    ctx.set_proposal(1)
    learned = run_arm(ctx, start, sweep0, a.sweeps, N)
    print(json.dumps(dict(arm="learned", **base, **learned, train_configs=n_train, collect_s=t1 - t0,
                          train_s=t2 - t1, loss_first_epoch=loss0, loss_last_epoch=loss,
                          learned_accept=acc)), flush=True)
    if not plain:
        ctx.close()
        return
    dE = learned["E_per_site"] - plain["E_per_site"]
    sig = float(np.hypot(learned["E_err"], plain["E_err"]))
    print(json.dumps(dict(summary=True, **base, dE_per_site=dE, dE_sigma=dE / sig if sig > 0 else 0.0,
                          eff_speedup=learned["eff_samples_per_s"] / plain["eff_samples_per_s"],
                          raw_speedup=learned["samples_per_s"] / plain["samples_per_s"])), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
