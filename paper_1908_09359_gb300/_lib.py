"""ctypes declarations of the pepsvmc C ABI (include/pepsvmc.h).

Loading fails loudly when the CUDA library has not been built: there is no CPU
fallback anywhere in the product path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpepsvmc.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EZEROPSI, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
FP32, MIXED_BF16, MIXED_TF32, MIXED_BF16X3 = 0, 1, 2, 3

NOALLOC_SCRATCH_FLOATS = 4194304  # PEPSVMC_NOALLOC_SCRATCH_FLOATS
NET_PARAMS = 10146                # parameters of the proposal network

ERRORS = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT",
          ENONFINITE: "ENONFINITE", EZEROPSI: "EZEROPSI", ESTATE: "ESTATE"}

# Every symbol include/pepsvmc.h declares (checked by the CPU tests).
SYMBOLS = [
    "pepsvmc_init", "pepsvmc_destroy", "pepsvmc_last_error", "pepsvmc_n_params",
    "pepsvmc_set_spins", "pepsvmc_get_spins", "pepsvmc_set_tensors", "pepsvmc_get_tensors",
    "pepsvmc_set_sweep_counter", "pepsvmc_get_sweep_counter", "pepsvmc_sample_sweep",
    "pepsvmc_enable_trace", "pepsvmc_get_trace", "pepsvmc_measure", "pepsvmc_n_grad_entries",
    "pepsvmc_get_chain_grad", "pepsvmc_amplitude", "pepsvmc_energy_and_grad", "pepsvmc_update",
    "pepsvmc_launch_count", "pepsvmc_set_profiling", "pepsvmc_get_profile", "pepsvmc_env3_left",
    "pepsvmc_env3_left_noalloc", "pepsvmc_get_profile_shapes", "pepsvmc_set_autotune", "pepsvmc_get_tuning",
    "pepsvmc_set_contraction_kernel",
    "pepsvmc_set_graphs", "pepsvmc_set_proposal_params", "pepsvmc_get_proposal_params",
    "pepsvmc_proposal_logits", "pepsvmc_proposal_collect", "pepsvmc_proposal_dataset_size", "pepsvmc_proposal_load",
    "pepsvmc_proposal_train", "pepsvmc_train_proposal", "pepsvmc_set_proposal", "pepsvmc_learned_sweep", "pepsvmc_get_learned_trace",
    "pepsvmc_env4_left", "pepsvmc_set_fused", "pepsvmc_random_sweep", "pepsvmc_get_random_trace", "pepsvmc_set_wait_budget", "pepsvmc_get_sums", "pepsvmc_set_sums", "pepsvmc_sums_device", "pepsvmc_finalize_sums",
    "pepsvmc_get_phi", "pepsvmc_simple_update", "pepsvmc_qr_pos",
]


class Config(C.Structure):
    _fields_ = [("Ly", C.c_int32), ("Lx", C.c_int32), ("D", C.c_int32), ("chi", C.c_int32),
                ("n_chains", C.c_int32), ("n_fit", C.c_int32), ("J1", C.c_double),
                ("J2", C.c_double), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("chi_measure", C.c_int32), ("wait_budget_cycles", C.c_uint64), ("chain_offset", C.c_int32),
                ("symmetrize", C.c_int32), ("reserved", C.c_int32 * 2)]


class PepsvmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load libpepsvmc.so (built by paper_1908_09359_gb300.build); raise if missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"pepsvmc CUDA library not found at {path}; run "
                           "`python -m paper_1908_09359_gb300.build` (needs nvcc)")
    lib = C.CDLL(path)
    P, D, I32, I64, U64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64, C.c_uint64
    I8 = C.POINTER(C.c_int8)
    sig = {
        "pepsvmc_init": (C.c_int, [C.POINTER(Config), D, D, P, C.POINTER(P)]),
        "pepsvmc_destroy": (None, [P]),
        "pepsvmc_last_error": (C.c_char_p, [P]),
        "pepsvmc_n_params": (I64, [P]),
        "pepsvmc_set_spins": (C.c_int, [P, I8]),
        "pepsvmc_get_spins": (C.c_int, [P, I8]),
        "pepsvmc_set_tensors": (C.c_int, [P, D]),
        "pepsvmc_get_tensors": (C.c_int, [P, D]),
        "pepsvmc_set_sweep_counter": (C.c_int, [P, U64]),
        "pepsvmc_get_sweep_counter": (U64, [P]),
        "pepsvmc_sample_sweep": (C.c_int, [P, I32, D]),
        "pepsvmc_enable_trace": (C.c_int, [P, I32]),
        "pepsvmc_get_trace": (C.c_int, [P, D, I8]),
        "pepsvmc_measure": (C.c_int, [P, D, D, I8]),
        "pepsvmc_n_grad_entries": (I64, [P]),
        "pepsvmc_get_chain_grad": (C.c_int, [P, I32, D]),
        "pepsvmc_amplitude": (C.c_int, [P, I32, D, I8]),
        "pepsvmc_energy_and_grad": (C.c_int, [P, I32, D, D, D, D, I8, D]),
        "pepsvmc_update": (C.c_int, [P, C.c_double, U64]),
        "pepsvmc_launch_count": (I64, [P]),
        "pepsvmc_set_profiling": (C.c_int, [P, I32]),
        "pepsvmc_get_profile": (C.c_int, [P, D]),
        "pepsvmc_env3_left": (C.c_int, [P, P, P, P, P, P, P] + [I32] * 9),
        "pepsvmc_env3_left_noalloc": (C.c_int, [P, P, P, P, P, P] + [I32] * 9 + [P]),
        "pepsvmc_qr_pos": (C.c_int, [P, P, I32, I32, I32, I32, P]),
        "pepsvmc_get_profile_shapes": (C.c_int, [P, C.c_char_p, I64]),
        "pepsvmc_set_autotune": (C.c_int, [P, I32]),
        "pepsvmc_set_contraction_kernel": (C.c_int, [P, I32, I32]),
        "pepsvmc_set_graphs": (C.c_int, [P, I32]),
        "pepsvmc_set_proposal_params": (C.c_int, [P, D]),
        "pepsvmc_get_proposal_params": (C.c_int, [P, D]),
        "pepsvmc_proposal_logits": (C.c_int, [P, D]),
        "pepsvmc_proposal_collect": (C.c_int, [P, I32]),
        "pepsvmc_proposal_dataset_size": (I64, [P]),
        "pepsvmc_proposal_load": (C.c_int, [P, I8, D, I64]),
        "pepsvmc_proposal_train": (C.c_int, [P, I32, I32, C.c_double, D]),
        "pepsvmc_train_proposal": (C.c_int, [P, C.POINTER(C.c_int8), C.c_int64, I32, C.c_double, C.POINTER(C.c_double)]),
        "pepsvmc_set_proposal": (C.c_int, [P, I32]),
        "pepsvmc_learned_sweep": (C.c_int, [P, I32, D]),
        "pepsvmc_get_learned_trace": (C.c_int, [P, D, D, I8]),
        "pepsvmc_get_tuning": (C.c_int, [P, C.c_char_p, I64]),
        "pepsvmc_set_wait_budget": (C.c_int, [P, U64]),
        "pepsvmc_set_fused": (C.c_int, [P, I32]),
        "pepsvmc_random_sweep": (C.c_int, [P, I32, D]),
        "pepsvmc_get_random_trace": (C.c_int, [P, C.POINTER(C.c_int32), D, I8]),
        "pepsvmc_env4_left": (C.c_int, [P] + [P] * 8 + [I32] * 13),
        "pepsvmc_get_sums": (C.c_int, [P, D, D, D]),
        "pepsvmc_set_sums": (C.c_int, [P, D, D, D]),
        "pepsvmc_sums_device": (C.c_int, [P, C.POINTER(P), C.POINTER(P), C.POINTER(P)]),
        "pepsvmc_finalize_sums": (C.c_int, [P]),
        "pepsvmc_get_phi": (C.c_int, [P, D, D]),
        "pepsvmc_simple_update": (C.c_int, [I32, I32, I32, C.c_double, C.c_double, C.c_double, I32, C.c_double,
                                            D, D, D, D, C.POINTER(C.c_int32), D, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
