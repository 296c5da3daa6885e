"""Write oracle-sampled spin configurations used as parity inputs.

Calls only ``oracle/`` and the seeded input generator.  Configurations sampled from
|Psi|^2 by the oracle's own sequential sweep (Sec. II A, Eq. (9)) are the inputs on
which the CUDA path is compared with the oracle: on uniformly random configurations
Psi(S) is often near a node and E_loc is ill-conditioned (float32 rounding of the
inputs alone moves it by ~1e-5 relative), which says nothing about the kernels.

    python tests/golden/make_sampled_configs.py [name ...]
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import vmc  # noqa: E402
from paper_1908_09359_gb300 import inputs  # noqa: E402

SWEEP_SEED = 77

# name -> (workload recipe, chains, sweeps)
CASES = {
    "peps_8x8": (dict(workload="peps_8x8"), 8, 12),
    "j1j2_6x6": (dict(Ly=6, Lx=6, D=3, chi=9, J2=0.5, seed=4), 4, 12),
    "peps_24x24": (dict(workload="peps_24x24"), 1, 4),
}


def case_inputs(name):
    """(grid, chi, sketch, start spins, J1, J2) of a case, from the seeded generator."""
    rec, n, _ = CASES[name]
    if "workload" in rec:
        w = inputs.workload(rec["workload"], n_chains=n)
        return (vmc.unpack(w["tensors"], w["Ly"], w["Lx"], w["D"]), w["chi"], w["sketch"],
                w["spins"], w["J1"], w["J2"])
    Ly, Lx, D, chi = rec["Ly"], rec["Lx"], rec["D"], rec["chi"]
    t = inputs.peps_tensors(Ly, Lx, D, rec["seed"])
    return (vmc.unpack(t, Ly, Lx, D), chi, inputs.sketch(max(Ly, Lx), chi, D, rec["seed"]),
            inputs.start_spins(n, Ly, Lx, rec["seed"], "random"), 1.0, rec["J2"])


def write(name):
    g, chi, W, spins, _, _ = case_inputs(name)
    _, n, sweeps = CASES[name]
    out = []
    for c in range(n):
        s = spins[c].copy()
        for t in range(sweeps):
            s, _, _ = vmc.sweep(g, s, chi, W, 3, SWEEP_SEED, c, t)
        out.append(s)
    path = os.path.join(HERE, f"{name}_sampled.txt")
    with open(path, "w") as f:
        f.write(f"# {name}: {n} chain(s), {sweeps} oracle sweeps each (n_fit=3, Philox key "
                f"{SWEEP_SEED}, chain c, sweeps 0..{sweeps - 1}) from the seeded random S^z=0 start.\n")
        f.write("# written by tests/golden/make_sampled_configs.py (oracle only); one block per chain,"
                " '+' = spin up\n")
        for s in out:
            for row in s:
                f.write("".join("+" if v > 0 else "-" for v in row) + "\n")
            f.write("\n")
    return path


def load(name):
    """Spins (n, Ly, Lx) int8 stored for ``name``."""
    blocks, cur = [], []
    for line in open(os.path.join(HERE, f"{name}_sampled.txt")):
        line = line.strip()
        if line.startswith("#"):
            continue
        if not line:
            if cur:
                blocks.append(cur)
            cur = []
            continue
        cur.append([1 if ch == "+" else -1 for ch in line])
    if cur:
        blocks.append(cur)
    return np.array(blocks, dtype=np.int8)


if __name__ == "__main__":
    for nm in sys.argv[1:] or list(CASES):
        print(write(nm))
