"""GPU parity of the tensor-core split-row Gram (tcgen05, TF32 operands split
into big + small parts) at padded rank 32, orders 2-4: one mode update (Alg. 1)
and one epoch against the FP64 oracle, and against the FP32 FMA Gram of the
same handle ("gram_tc" 0).  Ragged tiles, rank padding (R < 32), many tiles
per block and zero-visit blocks all occur in these cases."""
import numpy as np
import pytest

import oracle
from paper_2109_09534_gb300 import synth

from gpu_helpers import assert_factor_close, pair, rel_err, require_gpu, small_zipf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


CASES = {
    "order2_r32": lambda: synth.make_problem([400, 250], 32, 60_000, index_dist="zipf", sigma=0.01,
                                             test_frac=0.05, seed=21),
    "zipf2k_r32": lambda: small_zipf(),
    "zipf2k_r29": lambda: small_zipf(rank=29),
    "order4_r32": lambda: synth.make_problem([120, 90, 40, 30], 32, 120_000, index_dist="zipf", sigma=0.01,
                                             test_frac=0.05, seed=22),
}
# split thresholds: small chunks (ragged tiles, many blocks, some with no visits)
# and the default chunk (about 1600 visits, 26 tiles per block, at c = 0.1)
SPLITS = {"small": dict(heavy_rows=128, chunk=700), "default": dict(heavy_rows=128)}


def one_update(p, torch, gram_tc, split, c=0.1, bf16=False):
    g, o = pair(p, torch, gparams=dict(SPLITS[split], gram_tc=gram_tc, storage_bf16=int(bf16)))
    out = []
    for m in range(p.order):
        g.ao_iter = 2
        o.ao_iter = 2
        g.snmc(m, c, seed=77)
        o.snmc(m, c, seed=77)
        out.append((g.get_factor(m), o.get_factor(m)))
    st = g.stats()
    return out, st


@pytest.mark.parametrize("gram_tc", [1, 2], ids=["regrows", "tmagather"])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("split", list(SPLITS))
def test_single_update_tensor_gram(torch, case, split, gram_tc):
    """FP32 factors after one mode update: tensor-core Gram (rows gathered into
    registers, or by TMA gather4 in the warp-specialised form) vs FP64 within 1e-6."""
    p = CASES[case]()
    got, st = one_update(p, torch, gram_tc, split)
    assert st["visits_heavy"] > 0 and st["wait_timeouts"] == 0
    for m, (a, want) in enumerate(got):
        assert_factor_close(a, want, 1e-6, 1e-5, str((case, split, m, rel_err(a, want))))


@pytest.mark.parametrize("gram_tc", [1, 2], ids=["regrows", "tmagather"])
@pytest.mark.parametrize("case", ["zipf2k_r32", "order4_r32", "order2_r32"])
def test_tensor_gram_matches_fma_gram(torch, case, gram_tc):
    """The tensor-core and FP32 FMA Gram paths of one handle agree to FP32 rounding."""
    p = CASES[case]()
    tc, _ = one_update(p, torch, gram_tc, "small")
    fma, _ = one_update(p, torch, 0, "small")
    for m in range(p.order):
        assert_factor_close(tc[m][0], fma[m][0], 1e-6, 1e-5, str(m))


@pytest.mark.parametrize("gram_tc", [1, 2], ids=["regrows", "tmagather"])
def test_tensor_gram_bf16_storage(torch, gram_tc):
    p = CASES["zipf2k_r32"]()
    tc, st = one_update(p, torch, gram_tc, "small", bf16=True)
    fma, _ = one_update(p, torch, 0, "small", bf16=True)
    assert st["wait_timeouts"] == 0
    for m in range(p.order):
        assert rel_err(tc[m][0], tc[m][1]) <= 2e-2, m
        assert_factor_close(tc[m][0], fma[m][0], 1e-6, 1e-5, str(m))


@pytest.mark.parametrize("gram_tc", [1, 2], ids=["regrows", "tmagather"])
@pytest.mark.parametrize("c", [0.1, 1.0])
def test_epoch_tensor_gram(torch, c, gram_tc):
    """One epoch at c = 0.1 (10 AO iterations) and one full-gradient AO
    iteration at c = 1 (every visit of a split row, the longest blocks)."""
    p = small_zipf()
    g, o = pair(p, torch, gparams=dict(heavy_rows=128, gram_tc=gram_tc))
    g.epoch(c, seed=5)
    o.epoch(c, seed=5)
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, str(m))
    assert g.stats()["wait_timeouts"] == 0


@pytest.mark.parametrize("gram_tc", [1, 2], ids=["regrows", "tmagather"])
def test_wait_timeout_is_reported_and_the_handle_recovers(torch, gram_tc):
    """Test hook "test_gram_stall": block 0 of each tensor-core Gram launch
    waits up to 20,000 SM cycles on an mbarrier phase that no MMA was committed
    to, so its bounded wait gives up with nothing in flight.  The block frees its
    tensor memory, writes no partial and is counted; the next synchronising call
    reports the timeout once.  Afterwards the GPU and the library still work: a
    fresh handle matches the oracle."""
    from paper_2109_09534_gb300 import ntc
    p = small_zipf()
    split = dict(heavy_rows=128, chunk=700)
    g, _ = pair(p, torch, gparams=dict(split, gram_tc=gram_tc, test_gram_stall=20000))
    g.snmc(0, 0.1, seed=3)
    assert g.stats()["wait_timeouts"] == 1
    with pytest.raises(ntc.NTCError) as e:
        g.sync()
    assert e.value.status == ntc.NTC_ERR_CUDA and "gave up a bounded wait" in str(e.value)
    g.sync()   # reported once per new timeout
    g.ao_iter = 1
    g.snmc(1, 0.1, seed=3)
    with pytest.raises(ntc.NTCError) as e:
        g.get_factor(1)
    assert e.value.status == ntc.NTC_ERR_CUDA
    g.close()
    g2, o2 = pair(p, torch, gparams=dict(split, gram_tc=gram_tc))
    for m in range(3):
        g2.ao_iter = 2
        o2.ao_iter = 2
        g2.snmc(m, 0.1, seed=9)
        o2.snmc(m, 0.1, seed=9)
        assert_factor_close(g2.get_factor(m), o2.get_factor(m), 1e-6, 1e-5, str(m))
    assert g2.stats()["wait_timeouts"] == 0


# ---- padded rank 64: M = 128 = 2 R, N = 64 (gram_tc64.cuh) ----

CASES64 = {
    "zipf2k_r64": lambda: small_zipf(rank=64, nnz=150_000),
    "zipf2k_r40": lambda: small_zipf(rank=40, nnz=150_000),
    "order2_r64": lambda: synth.make_problem([400, 250], 64, 60_000, index_dist="zipf", sigma=0.01,
                                             test_frac=0.05, seed=23),
    "order4_r50": lambda: synth.make_problem([120, 90, 40, 30], 50, 100_000, index_dist="zipf", sigma=0.01,
                                             test_frac=0.05, seed=24),
}


@pytest.mark.parametrize("case", list(CASES64))
@pytest.mark.parametrize("split", list(SPLITS))
def test_single_update_tensor_gram_rank64(torch, case, split):
    """Padded rank 64: tensor-core Gram vs FP64 within 1e-6 after one mode
    update, and vs the FP32 FMA Gram of the same handle."""
    p = CASES64[case]()
    got, st = one_update(p, torch, 1, split)
    assert st["visits_heavy"] > 0 and st["wait_timeouts"] == 0
    fma, _ = one_update(p, torch, 0, split)
    for m, (a, want) in enumerate(got):
        assert_factor_close(a, want, 1e-6, 1e-5, str((case, split, m)))
        assert_factor_close(a, fma[m][0], 1e-6, 1e-5, str((case, split, m, "fma")))


def test_tensor_gram_rank64_bf16_and_epoch(torch):
    p = CASES64["zipf2k_r64"]()
    tc, st = one_update(p, torch, 1, "small", bf16=True)
    fma, _ = one_update(p, torch, 0, "small", bf16=True)
    assert st["wait_timeouts"] == 0
    for m in range(p.order):
        assert rel_err(tc[m][0], tc[m][1]) <= 2e-2, m
        assert_factor_close(tc[m][0], fma[m][0], 1e-6, 1e-5, str(m))
    g, o = pair(p, torch, gparams=dict(heavy_rows=128, gram_tc=1))
    g.epoch(0.1, seed=5)
    o.epoch(0.1, seed=5)
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, str(m))
    assert g.stats()["wait_timeouts"] == 0


def test_wait_timeout_rank64(torch):
    from paper_2109_09534_gb300 import ntc
    p = CASES64["zipf2k_r40"]()
    g, _ = pair(p, torch, gparams=dict(heavy_rows=128, chunk=700, test_gram_stall=20000))
    g.snmc(0, 0.1, seed=3)
    assert g.stats()["wait_timeouts"] == 1
    with pytest.raises(ntc.NTCError) as e:
        g.sync()
    assert e.value.status == ntc.NTC_ERR_CUDA
    g.close()
