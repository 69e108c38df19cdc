"""The C-ABI library builds, loads and exports every function include/lbm.h declares. No GPU: only
host-side calls that must fail cleanly (bad arguments) are made."""
import ctypes

import pytest

from paper_2309_08068_gb300 import build as lbm_build
from paper_2309_08068_gb300 import lbm


@pytest.fixture(scope="module")
def lib():
    lbm_build.build()
    return lbm.load_library()


def test_header_declares_the_boundary():
    names = lbm.header_functions()
    for required in ("lbm_create", "lbm_init_fields", "lbm_set_source", "lbm_step", "lbm_fields", "lbm_destroy",
                     "lbm_get_populations", "lbm_set_populations", "lbm_clear_sources", "lbm_last_error",
                     "lbm_time", "lbm_reduce", "lbm_check_finite"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lbm_build.LIB)
    missing = [name for name in lbm.header_functions() if not hasattr(raw, name)]
    assert missing == []


def test_population_counts(lib):
    # Section II: 2 x 2 x 3 x 4 + 2 = 50; Section III: 2 x 6 x 3 = 36.
    assert lib.lbm_num_populations(0) == 50
    assert lib.lbm_num_populations(1) == 36
    assert lib.lbm_num_populations(7) == -1


def test_create_rejects_bad_arguments_without_touching_a_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(5, 4, 4, 4, None, None, ctypes.byref(h)) == -1
    assert b"unknown model" in lib.lbm_last_error(None)
    assert lib.lbm_create(0, 0, 4, 4, None, None, ctypes.byref(h)) == -1
    assert lib.lbm_create(0, 65536, 65536, 2, None, None, ctypes.byref(h)) == -1
    opts = lbm._Options(0, None, 0, 1.0, 9.0, 0.0)
    assert lib.lbm_create(0, 4, 4, 4, None, ctypes.byref(opts), ctypes.byref(h)) == -6  # MM fixes eps0, mu0
    opts = lbm._Options(7, None, 0, 0.0, 0.0, 0.0)
    assert lib.lbm_create(1, 4, 4, 4, None, ctypes.byref(opts), ctypes.byref(h)) == -1  # unknown storage
    opts = lbm._Options(2, None, 0, 0.0, 0.0, 3.0)
    assert lib.lbm_create(1, 4, 4, 4, None, ctypes.byref(opts), ctypes.byref(h)) == -1  # scale not a power of 2
    assert b"power of two" in lib.lbm_last_error(None)
    assert lib.lbm_create(0, 4, 4, 4, None, None, None) == -1
    assert not h.value


def test_null_context_calls_are_rejected(lib):
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_sync(None) == -1
    assert lib.lbm_time(None) == -1
    assert lib.lbm_destroy(None) == 0
