"""Full-size checks at the benchmark's workload and launch configuration
(Zipf(1.1) 10^4-cube, R = 32, 100M draws, c = 0.1): one Algorithm-1 call on
mode 0 through the C ABI, then every split row of the mode (about 1,700 rows
holding most of the observations), 200 random light rows and some skipped rows
recomputed one by one by the FP64 oracle from the same starting factors, each
row within 1e-5 relative; and properties that hold at any size after a full
epoch."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
from paper_2109_09534_gb300 import ntc, synth

from gpu_helpers import rel_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    torch = require_gpu()
    p = synth.zipf_1e4cube()
    return torch, p


def test_fullsize_rows_match_oracle(big):
    torch, p = big
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream)
    g.set_observed(p.idx_train, p.val_train)
    U0 = [g.get_factor(i).astype(np.float64) for i in range(3)]
    seed, mode = 4, 0
    g.snmc(mode, p.c, seed)
    U1 = g.get_factor(mode)
    st = g.stats()
    counts = np.bincount(p.idx_train[:, mode], minlength=p.dims[mode]).astype(np.int64)
    kp = np.floor(p.c * counts).astype(np.int64)
    assert st["visits"] == int(kp.sum())
    assert st["rows_skipped"] == int((kp == 0).sum())
    assert np.all(np.isfinite(U1)) and np.all(U1 >= 0)
    row_ptr = np.concatenate([[0], np.cumsum(counts)])
    bucket = np.argsort(p.idx_train[:, mode], kind="stable")   # bucket order = input order within a row
    heavy = np.flatnonzero(counts > 4096)
    light = np.flatnonzero((kp > 0) & (counts <= 4096))
    rng = np.random.default_rng(5)
    picks = list(heavy) + list(rng.choice(light, size=min(200, light.size), replace=False))
    assert heavy.size > 1000

    def check(r):
        sel = bucket[row_ptr[r]:row_ptr[r + 1]]
        res = oracle.row_update(mode, p.lam, U0, p.idx_train[sel], p.val_train[sel].astype(np.float64),
                                int(row_ptr[r]), p.c, seed, 0, 0, U0[mode][r], U0[mode][r])
        return r, res["k"], rel_err(U1[r], res["a"])

    worst = 0.0
    with cf.ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:   # the oracle releases the GIL
        for r, k, err in ex.map(check, picks):
            assert k == kp[r]
            assert err <= 1e-5, (r, counts[r], err)
            worst = max(worst, err)
    skipped = np.flatnonzero(kp == 0)
    for r in skipped[:20]:
        np.testing.assert_array_equal(U1[r], U0[mode][r].astype(np.float32))
    g.close()


def test_fullsize_epoch_properties(big):
    torch, p = big
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream)
    g.set_observed(p.idx_train, p.val_train)
    r0 = g.rmse(p.idx_test, p.val_test)
    g.epoch(p.c, seed=4)
    st = g.stats()
    assert g.ao_iter == 10
    assert st["fallback_rows"] <= 2
    for i in range(3):
        U = g.get_factor(i)
        assert np.all(np.isfinite(U)) and np.all(U >= 0)
    assert g.rmse(p.idx_test, p.val_test) < r0
    g.close()
