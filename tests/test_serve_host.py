"""Serving runtime, host side (no GPU): the job memory model behind admission
and the argument checks that come back before any CUDA call."""
import ctypes

import numpy as np
import pytest

from paper_2109_09534_gb300 import build as nbuild
from paper_2109_09534_gb300 import ntc


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return ntc.load()


def desc(dims=(300, 200, 100), rank=16, nnz=10_000, n_test=100, bf16=0, **kw):
    N = len(dims)
    arrays = dict(idx=np.zeros((nnz, N), np.int32), vals=np.zeros(nnz, np.float32),
                  test_idx=np.zeros((n_test, N), np.int32), test_vals=np.zeros(n_test, np.float32))
    d = ntc.job_desc(dims, rank, kw.get("lam", 1e-3), kw.get("c", 0.1), arrays["idx"], arrays["vals"],
                     arrays["test_idx"], arrays["test_vals"], kw.get("target", 0.01), kw.get("max_epochs", 5),
                     storage_bf16=bf16)
    return d, arrays


def test_job_bytes_covers_observations_and_factors(lib):
    d, _ = desc()
    b = ntc.job_bytes(d)
    N, nnz = 3, 10_000
    # at least the buckets (16-byte entries, one per mode) and the FP32 masters (R padded to 16)
    assert b >= N * nnz * 16 + (300 + 200 + 100) * 16 * 4
    # grows with observations, rank, BF16 copies and order-8 entries (32 bytes)
    d2, _ = desc(nnz=20_000)
    assert ntc.job_bytes(d2) - b >= N * 10_000 * 16
    d3, _ = desc(rank=64)
    assert ntc.job_bytes(d3) > b
    d4, _ = desc(bf16=1)
    assert ntc.job_bytes(d4) - b >= (300 + 200 + 100) * 16 * 2
    d5, _ = desc(dims=(10,) * 5)
    d6, _ = desc(dims=(10,) * 4)
    assert ntc.job_bytes(d5) - ntc.job_bytes(d6) >= 10_000 * (5 * 32 - 4 * 16)


@pytest.mark.parametrize("field,value", [("order", 1), ("order", 9), ("rank", 0), ("rank", 65), ("c", 0.0),
                                         ("c", 1.5), ("lam", -1.0), ("nnz", 0), ("n_test", 0), ("max_epochs", 0),
                                         ("target_rmse", -1.0)])
def test_job_bytes_rejects_invalid_descriptions(lib, field, value):
    d, _keep = desc()
    setattr(d, field, value)
    out = ctypes.c_int64(-7)
    assert lib.ntc_job_bytes(ctypes.byref(d), ctypes.byref(out)) == ntc.NTC_ERR_ARG
    assert out.value == -7
    d, _keep = desc()
    d.dims[1] = 0
    assert lib.ntc_job_bytes(ctypes.byref(d), ctypes.byref(out)) == ntc.NTC_ERR_ARG


def test_server_create_rejects_bad_arguments_without_gpu(lib):
    s = ctypes.c_void_p()
    assert lib.ntc_server_create(0.0, 4, ctypes.byref(s)) == ntc.NTC_ERR_ARG
    assert lib.ntc_server_create(-1.0, 4, ctypes.byref(s)) == ntc.NTC_ERR_ARG
    assert lib.ntc_server_create(1e9, 0, ctypes.byref(s)) == ntc.NTC_ERR_ARG
    assert lib.ntc_server_create(float("inf"), 4, ctypes.byref(s)) == ntc.NTC_ERR_ARG
    assert s.value is None
    assert lib.ntc_server_last_error(None) == b"null server"
    assert lib.ntc_server_now(None) == -1.0
    lib.ntc_server_destroy(None)
