"""bfloat16 factor storage (FP32 accumulation and FP32 masters): per-factor
error against the FP64 oracle after one epoch, and held-out RMSE against the
plain FP32 method after several epochs, on scaled-down versions of the 4-way
uniform (R = 16, Gamma(2, 0.5) factors) and rating-shaped (R = 64, Zipf(1.2)
users and items, values rounded to 1..5) workloads."""
import numpy as np
import pytest

from paper_2109_09534_gb300 import ntc, synth

from gpu_helpers import pair, rel_err, require_gpu

pytestmark = pytest.mark.gpu


def four_way():
    return synth.uniform_4way(nnz_total=3_000_000, dims=(2000, 1000, 400, 50), rank=16, seed=3)


def rating():
    return synth.rating_3way(nnz_total=4_000_000, dims=(20_000, 10_000, 200), rank=64, seed=3)


@pytest.mark.parametrize("make", [four_way, rating], ids=["uniform4way_R16", "rating3way_R64"])
def test_bf16_and_fp32_against_oracle_one_epoch(make):
    torch = require_gpu()
    p = make()
    U0 = synth.random_factors(p.dims, p.rank, 0.5, seed=17)
    g32, o = pair(p, torch, factors=U0, omp=True)
    g16, _ = pair(p, torch, factors=U0, gparams=dict(storage_bf16=1))
    del _
    o.epoch(p.c, seed=9)
    g32.epoch(p.c, seed=9)
    g16.epoch(p.c, seed=9)
    for m in range(p.order):
        want = o.get_factor(m)
        assert rel_err(g32.get_factor(m), want) <= 1e-5, m
        assert rel_err(g16.get_factor(m), want) <= 2e-2, m


@pytest.mark.parametrize("make,epochs", [(four_way, 6), (rating, 4)], ids=["uniform4way_R16", "rating3way_R64"])
def test_bf16_rmse_within_one_percent_of_fp32(make, epochs):
    torch = require_gpu()
    p = make()
    s = torch.cuda.current_stream().cuda_stream
    res = {}
    for bf in (0, 1):
        g = ntc.NTC(p.dims, p.rank, p.lam, stream=s, storage_bf16=bf)
        g.set_observed(p.idx_train, p.val_train)
        for e in range(epochs):
            g.epoch(p.c, seed=100 + e)
        res[bf] = g.rmse(p.idx_test, p.val_test)
        g.close()
    assert abs(res[1] - res[0]) <= 0.01 * res[0], res
