"""The C-ABI library builds, loads and exports every symbol include/pepsvmc.h declares.

No compute call is made (this machine may have no GPU); only argument validation,
which returns before any CUDA call, is exercised.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1908_09359_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "pepsvmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pepsvmc_[a-z_0-9]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(_lib.SYMBOLS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def _cfg(**kw):
    c = _lib.Config()
    c.Ly, c.Lx, c.D, c.chi, c.n_chains, c.n_fit = 4, 4, 2, 4, 1, 1
    c.J1, c.J2, c.seed, c.precision = 1.0, 0.0, 1, 0
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("bad", [dict(Ly=3, Lx=3), dict(D=0), dict(chi=0), dict(n_fit=2),
                                 dict(n_chains=0), dict(precision=7), dict(chi=64, D=16),
                                 dict(chi_measure=-1), dict(chi_measure=65), dict(chi_measure=64, D=16),
                                 dict(chain_offset=-1), dict(wait_budget_cycles=(1 << 62) + 1),
                                 dict(symmetrize=2), dict(symmetrize=1, n_chains=3)])
def test_invalid_config_is_rejected_before_any_cuda_call(lib, bad):
    cfg = _cfg(**bad)
    t = np.zeros(10)
    ctx = C.c_void_p()
    rc = lib.pepsvmc_init(C.byref(cfg), t.ctypes.data_as(C.POINTER(C.c_double)),
                          t.ctypes.data_as(C.POINTER(C.c_double)), None, C.byref(ctx))
    assert rc == _lib.EINVAL
    assert lib.pepsvmc_last_error(ctx).decode()
    lib.pepsvmc_destroy(ctx)


def test_reserved_fields_must_be_zero(lib):
    cfg = _cfg()
    cfg.reserved[1] = 1
    t = np.zeros(10)
    ctx = C.c_void_p()
    rc = lib.pepsvmc_init(C.byref(cfg), t.ctypes.data_as(C.POINTER(C.c_double)),
                          t.ctypes.data_as(C.POINTER(C.c_double)), None, C.byref(ctx))
    assert rc == _lib.EINVAL and "reserved" in lib.pepsvmc_last_error(ctx).decode()
    lib.pepsvmc_destroy(ctx)


def test_null_arguments(lib):
    assert lib.pepsvmc_init(None, None, None, None, None) == _lib.EINVAL
    assert lib.pepsvmc_sample_sweep(None, 1, None) == _lib.EINVAL
    assert lib.pepsvmc_n_params(None) == 0
    for name in ("pepsvmc_set_wait_budget", "pepsvmc_set_fused"):
        assert getattr(lib, name)(None, 0) == _lib.EINVAL
    assert lib.pepsvmc_finalize_sums(None) == _lib.EINVAL
    assert lib.pepsvmc_get_sums(None, None, None, None) == _lib.EINVAL
    assert lib.pepsvmc_set_sums(None, None, None, None) == _lib.EINVAL
    assert lib.pepsvmc_sums_device(None, None, None, None) == _lib.EINVAL


def test_config_layout_matches_header():
    """The ctypes mirror of pepsvmc_config has the C struct's field offsets."""
    offs = {name: getattr(_lib.Config, name).offset for name, _ in _lib.Config._fields_}
    assert offs["J1"] == 24 and offs["seed"] == 40 and offs["chi_measure"] == 52
    assert offs["wait_budget_cycles"] == 56 and offs["chain_offset"] == 64 and offs["symmetrize"] == 68
    assert offs["reserved"] == 72
    assert C.sizeof(_lib.Config) == 80
