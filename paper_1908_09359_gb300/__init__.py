"""GB300-native (sm_103a) per-sample single-layer PEPS contraction for variational
Monte Carlo (Liu, Huang, Gong, Gu, arXiv:1908.09359).

The hot path -- boundary-MPS row sweeps with truncation, cached environments,
log-scaled amplitudes, Metropolis ratios, E_loc of the Heisenberg / J1-J2 model and
the log-derivatives accumulated into the energy gradient -- runs in the CUDA library
built from ``csrc/`` behind the C ABI of ``include/pepsvmc.h``.  ``api.PepsVMC`` is
its Python binding; ``inputs`` draws the seeded synthetic workloads.
"""
from .api import PepsVMC, PepsvmcError  # noqa: F401
