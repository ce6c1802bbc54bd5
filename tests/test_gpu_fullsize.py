"""Full-size checks at the benchmark's workload and launch configuration
(Zipf(1.1) 10^4-cube, R = 32, 100M draws, c = 0.1): one Algorithm-1 call on
mode 0 through the C ABI, then sampled rows -- the heaviest split row, a
middle split row, the lightest split row, light rows and a skipped row --
recomputed one by one by the FP64 oracle from the same starting factors; and
properties that hold at any size after a full epoch."""
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


def test_fullsize_sampled_rows_match_oracle(big):
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
    order = np.argsort(counts, kind="stable")
    heavy = [r for r in order if counts[r] > 4096]
    light = [r for r in order if 0 < kp[r] and counts[r] <= 4096]
    picks = [heavy[-1], heavy[len(heavy) // 2], heavy[0], light[-1], light[len(light) // 2], light[0]]
    skipped = [r for r in order if kp[r] == 0]
    col = p.idx_train[:, mode]
    for r in picks:
        sel = np.flatnonzero(col == r)           # bucket order = input order within the row
        res = oracle.row_update(mode, p.lam, U0, p.idx_train[sel], p.val_train[sel].astype(np.float64),
                                int(row_ptr[r]), p.c, seed, 0, 0, U0[mode][r], U0[mode][r])
        assert res["k"] == kp[r]
        assert rel_err(U1[r], res["a"]) <= 1e-5, (r, counts[r])
    for r in skipped[:3]:
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
