"""Full-size precision checks on the two workloads the BF16 storage contract is
stated for: the uniform 4-way tensor (10^5 x 5*10^4 x 2*10^4 x 10^3, R = 16,
200M draws, Gamma(2, 0.5) factors) and the rating-shaped tensor (10^6 x 5*10^5
x 200, R = 64, 500M draws, Zipf(1.2) users and items, values rounded to 1..5).

For each: (1) one Algorithm-1 call per checked mode from the same starting
factors, FP32 storage, with sampled rows -- split rows from the largest the
oracle recomputes in seconds down to the smallest, 100 random light rows and
skipped rows -- recomputed one by one by the FP64 oracle, each row within 1e-5
relative (with BF16 storage the oracle gathers the same BF16-rounded rows of
the other modes, so the bound is the same); (2) the held-out RMSE after four epochs with
BF16 factor storage within 1% of the plain FP32 method on the same seeds."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
from paper_2109_09534_gb300 import ntc, synth

from gpu_helpers import rel_err, require_gpu

pytestmark = pytest.mark.gpu

WORKLOADS = {
    "uniform4way_200M_R16": (lambda: synth.uniform_4way(), [0, 3]),
    "rating_500M_R64": (lambda: synth.rating_3way(), [0, 2]),
}
MAX_ORACLE_ROW = 3_000_000   # largest split row recomputed by the oracle


@pytest.fixture(scope="module", params=list(WORKLOADS))
def workload(request):
    torch = require_gpu()
    make, modes = WORKLOADS[request.param]
    return torch, make(), modes, request.param


def _handle(torch, p, bf16):
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream,
                storage_bf16=bf16, cache_staging=0)
    g.set_observed(p.idx_train, p.val_train)
    return g


def test_fullsize_rows_match_oracle(workload):
    torch, p, modes, name = workload
    rng = np.random.default_rng(11)
    for bf16 in (0, 1):
        g = _handle(torch, p, bf16)
        U0 = [g.get_factor(i).astype(np.float64) for i in range(p.order)]
        tol = 1e-5
        for mode in modes:
            g.snmc(mode, p.c, seed=6)
            U1 = g.get_factor(mode)
            g.set_factor(mode, U0[mode].astype(np.float32))   # the next mode starts from U0 as well
            counts = np.bincount(p.idx_train[:, mode], minlength=p.dims[mode]).astype(np.int64)
            kp = np.floor(p.c * counts).astype(np.int64)
            assert np.all(np.isfinite(U1)) and np.all(U1 >= 0)
            row_ptr = np.concatenate([[0], np.cumsum(counts)])
            bucket = np.argsort(p.idx_train[:, mode], kind="stable")
            heavy = np.flatnonzero((counts > 4096) & (counts <= MAX_ORACLE_ROW))
            heavy = heavy[np.argsort(counts[heavy], kind="stable")]
            light = np.flatnonzero((kp > 0) & (counts <= 4096))
            picks = []
            if heavy.size:
                picks += [int(heavy[-1]), int(heavy[heavy.size // 2]), int(heavy[0])]
            if light.size:
                picks += [int(r) for r in rng.choice(light, size=min(100, light.size), replace=False)]
            assert picks
            # the oracle gathers with the factors the GPU read: BF16-rounded copies under BF16 storage
            Ug = [u.astype(np.float32) for u in U0]
            if bf16:
                import torch as _t
                Ug = [_t.from_numpy(u).to(_t.bfloat16).float().numpy() for u in Ug]
            Uo = [u.astype(np.float64) for u in Ug]
            Uo[mode] = U0[mode]

            def check(r):
                sel = bucket[row_ptr[r]:row_ptr[r + 1]]
                res = oracle.row_update(mode, p.lam, Uo, p.idx_train[sel], p.val_train[sel].astype(np.float64),
                                        int(row_ptr[r]), p.c, 6, 0, 0, U0[mode][r], U0[mode][r])
                return r, res["k"], rel_err(U1[r], res["a"])

            with cf.ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
                for r, k, err in ex.map(check, picks):
                    assert k == kp[r]
                    assert err <= tol, (name, bf16, mode, r, counts[r], err)
            for r in np.flatnonzero(kp == 0)[:20]:
                np.testing.assert_array_equal(U1[r], U0[mode][r].astype(np.float32))
        g.close()


def test_fullsize_bf16_rmse_within_one_percent_of_fp32(workload):
    torch, p, _, name = workload
    res = {}
    for bf16 in (0, 1):
        g = _handle(torch, p, bf16)
        r0 = g.rmse(p.idx_test, p.val_test)
        for e in range(4):
            g.epoch(p.c, seed=500 + e)
        res[bf16] = g.rmse(p.idx_test, p.val_test)
        assert res[bf16] < r0
        assert g.stats()["wait_timeouts"] == 0
        g.close()
    assert abs(res[1] - res[0]) <= 0.01 * res[0], (name, res)
