"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/ntc.h declares; argument errors that are
decided before any CUDA call come back as statuses."""
import ctypes

import numpy as np
import pytest

from paper_2109_09534_gb300 import build as nbuild
from paper_2109_09534_gb300 import ntc


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return ntc.load()


def test_header_declares_the_boundary():
    names = ntc.declared_functions()
    for must in ["ntc_create", "ntc_set_param", "ntc_set_stream", "ntc_set_observed", "ntc_epoch",
                 "ntc_predict", "ntc_rmse", "ntc_cost", "ntc_get_factor", "ntc_set_factor",
                 "ntc_get_state", "ntc_set_state", "ntc_last_error", "ntc_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in ntc.declared_functions():
        assert hasattr(lib, name), name


def test_create_rejects_bad_arguments_without_gpu(lib):
    h = ctypes.c_void_p()
    dims = np.array([3, 4, 5], dtype=np.int64)
    P = dims.ctypes.data_as(ctypes.c_void_p)
    assert lib.ntc_create(1, P, 2, 0.1, ctypes.byref(h)) == ntc.NTC_ERR_ARG      # order < 2
    assert lib.ntc_create(9, P, 2, 0.1, ctypes.byref(h)) == ntc.NTC_ERR_ARG      # order > 8
    assert lib.ntc_create(3, P, 0, 0.1, ctypes.byref(h)) == ntc.NTC_ERR_ARG      # rank < 1
    assert lib.ntc_create(3, P, 65, 0.1, ctypes.byref(h)) == ntc.NTC_ERR_ARG     # rank > 64
    assert lib.ntc_create(3, P, 2, -1.0, ctypes.byref(h)) == ntc.NTC_ERR_ARG     # lambda < 0
    assert lib.ntc_create(3, P, 2, float("nan"), ctypes.byref(h)) == ntc.NTC_ERR_ARG
    bad = np.array([3, 0, 5], dtype=np.int64)
    assert lib.ntc_create(3, bad.ctypes.data_as(ctypes.c_void_p), 2, 0.1, ctypes.byref(h)) == ntc.NTC_ERR_ARG
    assert h.value is None
    assert lib.ntc_last_error(None) == b"null handle"
    lib.ntc_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    saved = ntc._lib
    try:
        ntc._lib = None
        with pytest.raises(OSError):
            ntc.load(str(tmp_path / "libntc_missing.so"))
    finally:
        ntc._lib = saved
