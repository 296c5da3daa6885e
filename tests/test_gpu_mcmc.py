"""Statistical pins of the GPU sampler: at exact Dc on 4x4 lattices the Markov chains of
the sequential sweep (Sec. II A) -- alone, and with the learned band moves accepted by
the Metropolis-Hastings rule -- must sample |Psi|^2, so the mean of E_loc over the run
equals <Psi|H|Psi>/<Psi|Psi> from the S^z = 0 enumeration (oracle/exact.py) within five
tau_int-corrected standard errors, for the Heisenberg and the J1-J2 (J2/J1 = 0.5) model.
A sampler that drops a bond family, mis-weights a move or breaks detailed balance
biases the mean by many standard errors at these sample counts."""
import numpy as np
import pytest

from oracle import exact, vmc
from paper_1908_09359_gb300 import autocorr, inputs

pytestmark = pytest.mark.gpu

CHAINS, THERM, SWEEPS = 2048, 20, 60


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1908_09359_gb300 import api as a
    from paper_1908_09359_gb300 import build
    build.build()
    return a


@pytest.mark.parametrize("J2", [0.0, 0.5])
@pytest.mark.parametrize("learned", [False, True])
def test_mean_eloc_matches_exact_energy(api, J2, learned):
    t = inputs.peps_tensors(4, 4, 2, 11, True)
    sk = inputs.sketch(4, 4, 2, 11)
    E, _, _ = exact.energy_exact(vmc.unpack(t, 4, 4, 2), 1.0, J2)
    ctx = api.PepsVMC(4, 4, 2, 4, CHAINS, t, sk, J1=1.0, J2=J2, seed=3, n_fit=1)
    ctx.set_spins(inputs.start_spins(CHAINS, 4, 4, 7, "random"))
    if learned:
        ctx.set_proposal_params(inputs.proposal_params(5))
        ctx.proposal_collect(4)
        ctx.proposal_train(5, 256, 2e-3)
        ctx.set_proposal(1)
    ctx.sample_sweep(THERM)
    el = ctx.energy_and_grad(SWEEPS, want_grad=False)["eloc"].reshape(SWEEPS, CHAINS)
    mean, err = autocorr.mean_and_error(el)
    assert err > 0
    assert abs(mean - E) <= 5 * err, (mean, E, err)
    if learned:
        ctx.amplitude(0)                    # top environments of the current configurations
        assert ctx.learned_sweep(1) > 0.0   # the learned moves are accepted at all
    ctx.close()
