"""Convergence in the boundary cutoff Dc (App. D): how far Psi(S) and E_loc(S) at a
cutoff Dc are from their values at a much larger reference cutoff, on the GPU.

    python -m paper_1908_09359_gb300.cutoff_study --L 16 --D 4 --cutoffs 4,8,12,16,24,32 --ref 64

For each cutoff the same configurations are measured (pepsvmc_measure) and compared
with the reference cutoff: eps = |Psi_Dc / Psi_ref - 1| per configuration (App. D's
relative amplitude error, Psi_ref standing in for the exact value) and
|E_loc,Dc - E_loc,ref| / max(|E_loc,ref|, 1).  Configurations come from the plain sampler at the
reference cutoff (so they are typical of |Psi|^2); tensors are the seeded iid workload
recipe or the bond-decay one (--structured).  Output: one JSON line per cutoff.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    from . import api, inputs
    p = argparse.ArgumentParser()
    p.add_argument("--L", type=int, default=16)
    p.add_argument("--D", type=int, default=4)
    p.add_argument("--cutoffs", default="4,8,12,16,24,32")
    p.add_argument("--ref", type=int, default=64)
    p.add_argument("--chains", type=int, default=128)
    p.add_argument("--sweeps", type=int, default=10, help="plain sweeps at the reference cutoff before measuring")
    p.add_argument("--structured", action="store_true")
    p.add_argument("--precision", default="fp32", choices=sorted(api.PRECISIONS))
    a = p.parse_args()
    L, D, C, ref = a.L, a.D, a.chains, a.ref
    seed = inputs.SEED_BASE + 100 + L
    t = inputs.peps_tensors(L, L, D, seed, True, bond_decay=1.0 if a.structured else 0.0)
    sk = inputs.sketch(L, ref, D, seed)
    prec = api.PRECISIONS[a.precision]

    def measure(chi, spins):
        # the fit at cutoff c starts from the leading [c][D][c] corner of the sketch
        ctx = api.PepsVMC(L, L, D, chi, C, t, np.ascontiguousarray(sk[:, :chi, :, :chi]), seed=seed,
                          precision=prec)
        ctx.set_spins(spins)
        e, lp, sg = ctx.measure()
        ctx.close()
        return e, lp, sg

    ctx = api.PepsVMC(L, L, D, ref, C, t, sk, seed=seed, precision=prec)
    ctx.set_spins(inputs.start_spins(C, L, L, seed, "random"))
    ctx.sample_sweep(a.sweeps)
    spins = ctx.get_spins()
    e_ref, lp_ref, sg_ref = ctx.measure()
    ctx.close()
    for chi in [int(x) for x in a.cutoffs.split(",")]:
        e, lp, sg = measure(chi, spins)
        ratio = sg * sg_ref * np.exp(lp - lp_ref)
        eps = np.abs(ratio - 1.0)
        de = np.abs(e - e_ref) / np.maximum(np.abs(e_ref), 1.0)
        print(json.dumps({"L": L, "D": D, "Dc": chi, "Dc_ref": ref, "tensors": "structured" if a.structured else "iid",
                          "configs": C, "eps_median": float(np.median(eps)), "eps_max": float(np.max(eps)),
                          "dEloc_median": float(np.median(de)), "dEloc_max": float(np.max(de)),
                          "sign_flips": int(np.sum(sg != sg_ref))}), flush=True)


if __name__ == "__main__":
    main()
