"""ntc_rmse_noalloc: the RMSE entry point for callers that cannot allocate
device memory while they run (a serving process whose HBM is handed out up
front, or a framework whose caching allocator owns the device).  It must give
the same result as ntc_rmse on two calls in a row, allocate nothing, and
reject query counts beyond its fixed scratch.  This file is collected last."""
import ctypes

import numpy as np
import pytest

from paper_2109_09534_gb300 import ntc, synth

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu

LIMIT = 4096 * 2048


def test_rmse_noalloc_matches_rmse():
    torch = require_gpu()
    lib = ntc.load()
    f = lib.ntc_rmse_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    p = synth.planted_rank10_100cube()
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream)
    g.set_observed(p.idx_train, p.val_train)
    g.epoch(p.c, seed=4)
    want = g.rmse(p.idx_test, p.val_test)
    idx_d = torch.from_numpy(np.ascontiguousarray(p.idx_test)).cuda()
    val_d = torch.from_numpy(np.ascontiguousarray(p.val_test)).cuda()
    torch.cuda.synchronize()
    free = []
    for _ in range(3):
        out = ctypes.c_double(-1.0)
        st = f(g.h, idx_d.shape[0], idx_d.data_ptr(), val_d.data_ptr(), ctypes.byref(out))
        assert st == ntc.NTC_OK, lib.ntc_last_error(g.h)
        assert out.value == pytest.approx(want, rel=1e-4)
        free.append(torch.cuda.mem_get_info()[0])
    assert free[1] == free[2]   # after the one-time set-up, calls allocate nothing
    # a different, larger query set after the first: the shared scratch holds no stale state
    idx2 = torch.from_numpy(np.ascontiguousarray(p.idx_train)).cuda()
    val2 = torch.from_numpy(np.ascontiguousarray(p.val_train)).cuda()
    out = ctypes.c_double()
    assert f(g.h, idx2.shape[0], idx2.data_ptr(), val2.data_ptr(), ctypes.byref(out)) == ntc.NTC_OK
    assert out.value == pytest.approx(g.rmse(p.idx_train, p.val_train), rel=1e-4)
    # an index out of range: NTC_ERR_INDEX, found on the device without
    # reading a factor row; the next valid call starts from a clear flag
    bad = p.idx_test.copy()
    bad[17, 1] = p.dims[1]
    bad[40, 2] = -1
    bad_d = torch.from_numpy(np.ascontiguousarray(bad)).cuda()
    assert f(g.h, bad_d.shape[0], bad_d.data_ptr(), val_d.data_ptr(), ctypes.byref(out)) == ntc.NTC_ERR_INDEX
    assert b"out of range" in lib.ntc_last_error(g.h)
    out = ctypes.c_double(-1.0)
    assert f(g.h, idx_d.shape[0], idx_d.data_ptr(), val_d.data_ptr(), ctypes.byref(out)) == ntc.NTC_OK
    assert out.value == pytest.approx(want, rel=1e-4)
    # beyond the fixed scratch: a clear error, nothing launched
    st = f(g.h, LIMIT + 1, idx_d.data_ptr(), val_d.data_ptr(), ctypes.byref(out))
    assert st == ntc.NTC_ERR_ARG
    assert b"exceeds the limit" in lib.ntc_last_error(g.h)
    g.close()
