"""Host logic of the CUDA engine, run without a GPU.

With PEPSVMC_DRY_RUN=1 the library skips every device call but still walks the whole
orchestration -- boundary-MPS fits in four lattice orientations, both sweep phases,
the three- and four-line measurement, gradient accumulation and sign-SGD -- and
checks the memory span of every launch against its allocation.  This runs each
workload's full launch sequence in a subprocess (the mode is process-wide), in FP32
(separate products) and in split BF16 (fused three- and four-line steps where the bonds
fit, separate tensor-core products elsewhere).
"""
import json
import os
import subprocess
import sys

import pytest

from paper_1908_09359_gb300 import build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
from paper_1908_09359_gb300 import inputs, api
w = inputs.WORKLOADS[sys.argv[1]]
L = max(w["Ly"], w["Lx"])
t = inputs.peps_tensors(w["Ly"], w["Lx"], w["D"], 1)
# the sampler at 2/3 of the cutoff, the measurement at the full cutoff (Dc1 < Dc2)
chi_s = max(1, (2 * w["chi"]) // 3) if sys.argv[2] == "split" else w["chi"]
chi_m = w["chi"] if sys.argv[2] == "split" else 0
sk = np.zeros((L, w["chi"], w["D"], w["chi"]))
c = api.PepsVMC(w["Ly"], w["Lx"], w["D"], chi_s, w["n_chains"], t, sk, J1=w["J1"], J2=w["J2"],
                seed=1, n_fit=3, stream=0, chi_measure=chi_m, precision=int(sys.argv[3]))
n0 = c.launches
c.sample_sweep(1)
n1 = c.launches
c.measure()
n2 = c.launches
c.amplitude(w["Ly"] // 2)
c.energy_and_grad(1)
c.update(0.01, 1)
c.enable_trace(True)
c.sample_sweep(1)
c.set_proposal_params(inputs.proposal_params(1))
c.learned_sweep(1)
c.proposal_collect(1)
c.proposal_train(1, min(w["n_chains"], 64), 1e-3)
c.set_proposal(1)
c.energy_and_grad(2)
if w["Ly"] * w["Lx"] <= 64:
    c.random_sweep(1)
    c.get_random_trace()
    c.measure()
print(json.dumps(dict(sweep=n1 - n0, measure=n2 - n1)))
"""


@pytest.mark.parametrize("precision", [0, 3])
@pytest.mark.parametrize("cutoffs", ["one", "split"])
@pytest.mark.parametrize("name", list(inputs.WORKLOADS))
def test_every_launch_in_bounds(name, cutoffs, precision):
    build.build()
    env = dict(os.environ, PEPSVMC_DRY_RUN="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT, name, cutoffs, str(precision)], capture_output=True,
                       text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    counts = json.loads(r.stdout.strip().splitlines()[-1])
    assert counts["sweep"] > 0 and counts["measure"] > 0


SCRIPT_SYM = r"""
import sys
import numpy as np
from paper_1908_09359_gb300 import inputs, api
w = inputs.WORKLOADS[sys.argv[1]]
L = max(w["Ly"], w["Lx"])
t = inputs.peps_tensors(w["Ly"], w["Lx"], w["D"], 1)
sk = np.zeros((L, w["chi"], w["D"], w["chi"]))
n = w["n_chains"] + w["n_chains"] % 2
c = api.PepsVMC(w["Ly"], w["Lx"], w["D"], w["chi"], n, t, sk, J1=w["J1"], J2=w["J2"], seed=1, n_fit=3,
                stream=0, precision=int(sys.argv[2]), symmetrize=True)
sp = inputs.start_spins(n // 2, w["Ly"], w["Lx"], 3, "random")
c.set_spins(np.concatenate([sp, -sp]))
try:
    c.set_spins(np.concatenate([sp, sp]))
    raise SystemExit("a second half that is not the inversion was accepted")
except api.PepsvmcError as e:
    assert e.code == api.EINVAL
c.enable_trace(True)
c.sample_sweep(1)
c.measure()
c.phi()
c.energy_and_grad(1)
c.update(0.01, 1)
for call in (lambda: c.random_sweep(1), lambda: c.set_proposal(1)):
    try:
        call()
        raise SystemExit("symmetrised context ran a non-sequential sampler")
    except api.PepsvmcError as e:
        assert e.code == api.EINVAL
print("ok")
"""


@pytest.mark.parametrize("precision", [0, 3])
@pytest.mark.parametrize("name", ["peps_4x4", "peps_8x8", "peps_24x24"])
def test_symmetrised_launches_in_bounds(name, precision):
    """The spin-inversion symmetrised sampler and measurement (S and S-bar chains in
    pairs) walk their launch sequence with every span checked; inconsistent pairs and
    the non-sequential samplers are refused with EINVAL."""
    build.build()
    env = dict(os.environ, PEPSVMC_DRY_RUN="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT_SYM, name, str(precision)], capture_output=True,
                       text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:] + r.stdout[-500:]
    assert r.stdout.strip().endswith("ok")
