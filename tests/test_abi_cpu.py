"""CPU-only checks of the C ABI library: it builds, loads, exports every symbol
that include/lbe.h declares, its integer shell tables match the oracle's bit for
bit, and without a usable sm_103a GPU it fails loudly (no CPU fallback)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1202_3842_gb300 import build as lbe_build
from paper_1202_3842_gb300 import lbe


@pytest.fixture(scope="module")
def L():
    lbe_build.build()
    return lbe.lib()


def test_every_declared_symbol_is_exported(L):
    names = lbe.declared_symbols()
    assert "lbe_step" in names and "lbe_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("sigma", [1, 2, 3, 4, 5, 6, 7, 8])
def test_shell_tables_match_oracle_bit_exact(L, sigma):
    mine = lbe.lbe_shell(sigma)
    ref = oracle.shell(sigma)
    assert mine.shape == ref.shape
    # same set and, both being listed z-major then y then x, the same order
    np.testing.assert_array_equal(mine, ref)


def test_status_strings(L):
    assert lbe.lbe_status_string(0) == "ok"
    assert lbe.lbe_status_string(5) == "diverged"


def test_non_integer_pair_diameter_is_rejected(L):
    with pytest.raises(lbe.LbeError):
        lbe.lbe_shell(3.5)


def test_create_without_gpu_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbe.LbeError) as ei:
        lbe.lbe_create((8, 8, 8))
    assert ei.value.status == 4  # LBE_ERR_CUDA


def test_bad_config_is_rejected_before_device_use(L):
    cfg = lbe.lbe_config()
    cfg.nx, cfg.ny, cfg.nz = 0, 4, 4
    cfg.nspecies = 1
    out = ctypes.c_void_p()
    assert L.lbe_create(ctypes.byref(cfg), None, None, ctypes.byref(out)) == 1
    cfg.nx = 4
    cfg.nspecies = 9
    assert L.lbe_create(ctypes.byref(cfg), None, None, ctypes.byref(out)) == 1
    cfg.nspecies = 1
    cfg.enable_visc = 1
    cfg.scheme = lbe.LBE_SD_EU  # the viscous force belongs to the DD-TR scheme
    assert L.lbe_create(ctypes.byref(cfg), None, None, ctypes.byref(out)) == 2


def test_scheme_config_is_checked_before_device_use(L):
    def create(**kw):
        cfg = lbe.lbe_config()
        cfg.nx, cfg.ny, cfg.nz = 4, 4, 4
        cfg.nspecies = kw.get("M", 1)
        cfg.precision = kw.get("prec", lbe.LBE_FP32)
        cfg.scheme = kw.get("scheme", lbe.LBE_DD_TR)
        cfg.consistent_moments = kw.get("consistent", 0)
        out = ctypes.c_void_p()
        return L.lbe_create(ctypes.byref(cfg), None, None, ctypes.byref(out))
    assert create(scheme=7) == 1                                          # unknown scheme
    assert create(scheme=lbe.LBE_SD_EU, prec=lbe.LBE_BF16_SHIFTED) == 2   # ablations: FP64/FP32 only
    assert create(scheme=lbe.LBE_SD_TR, M=3) == 2                         # ablations: one or two species
    assert create(scheme=lbe.LBE_DD_EU, consistent=1) == 1                # consistent recovery is DD-TR's
