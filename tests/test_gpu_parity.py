"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Bucketing and sampling are integer work and must match
bit for bit; factors must match within the tolerances of the method's
precision contract (FP32 accumulation: 1e-6 relative after one mode update,
1e-5 after one epoch; bfloat16 factor storage: 2e-2)."""
import numpy as np
import pytest

import oracle
from paper_2109_09534_gb300 import ntc, synth

from gpu_helpers import assert_factor_close, oracle_mask, pair, rel_err, require_gpu, small_zipf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


CASES = {
    "cube100": lambda: synth.planted_rank10_100cube(),
    "zipf2k": lambda: small_zipf(),
    "uni4way": lambda: synth.make_problem([300, 200, 60, 8], 16, 150_000, index_dist="uniform",
                                          factor_dist="gamma", sigma=0.05, test_frac=0.02, seed=5),
    "order2": lambda: synth.make_problem([500, 300], 5, 40_000, sigma=0.01, test_frac=0.05, seed=6),
    "order5": lambda: synth.make_problem([20, 12, 9, 7, 5], 4, 30_000, sigma=0.01, test_frac=0.05, seed=7),
}
# small thresholds so that even the small cases have split (heavy) rows and many chunks
SPLIT = dict(heavy_rows=128, chunk=700)
# every row of at most 4096 observations through the block-per-row kernel
# (none through the warp-per-row one)
LIGHT = dict(tiny_rows=0)
LAYOUTS = {"default": {}, "split": SPLIT, "light": LIGHT}


@pytest.mark.parametrize("case", list(CASES))
def test_bucket_bit_exact(torch, case):
    p = CASES[case]()
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream, keep_perm=1)
    g.set_observed(p.idx_train, p.val_train)
    for m in range(p.order):
        rp_o, perm_o = oracle.bucket(p.idx_train, m, p.dims[m])
        rp_g, perm_g = g.get_bucket(m, perm=True)
        np.testing.assert_array_equal(rp_g, rp_o)
        np.testing.assert_array_equal(perm_g, perm_o)


@pytest.mark.parametrize("case", ["cube100", "zipf2k", "uni4way", "order5"])
@pytest.mark.parametrize("c", [0.1, 0.37, 1.0])
@pytest.mark.parametrize("params", [{}, SPLIT, dict(SPLIT, bracket_z=0.0), dict(SPLIT, bracket_z=2.0),
                                    dict(SPLIT, bracket_z=1e5), LIGHT],
                         ids=["default", "split", "fallback", "narrow", "wide", "light"])
def test_sampler_bit_exact(torch, case, c, params):
    p = CASES[case]()
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream, **params)
    g.set_observed(p.idx_train, p.val_train)
    seed, it, inner = 12345, 7, 1
    for m in range(p.order):
        got = g.sample_mask(m, c, seed, it, inner, p.nnz)
        want = oracle_mask(p.idx_train, m, p.dims[m], c, seed, it, inner)
        np.testing.assert_array_equal(got, want)


def test_fallback_selector_is_counted(torch):
    """bracket_z = 0 leaves no candidates: a split row needs the exact fallback
    unless exactly k of its keys fall below the bracket."""
    p = small_zipf()
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream, bracket_z=0.0,
                heavy_rows=128, chunk=700)
    g.set_observed(p.idx_train, p.val_train)
    c, seed = 0.1, 1
    got = g.sample_mask(0, c, seed, 0, 0, p.nnz)
    np.testing.assert_array_equal(got, oracle_mask(p.idx_train, 0, p.dims[0], c, seed, 0, 0))
    row_ptr, _ = oracle.bucket(p.idx_train, 0, p.dims[0])
    want = 0
    for r in range(p.dims[0]):
        q0, n = int(row_ptr[r]), int(row_ptr[r + 1] - row_ptr[r])
        k = oracle.sample_count(c, n)
        if n <= 128 or k == 0 or k == n:
            continue
        lo = int(np.floor((k / n) * 4294967296.0))
        below = sum(oracle.sample_key(seed, 0, 0, 0, q) < lo for q in range(q0, q0 + n))
        want += below != k
    assert want > 0 and g.stats()["fallback_rows"] == want


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("layout", list(LAYOUTS))
def test_single_mode_update(torch, case, layout):
    """One call of Algorithm 1 from identical factors: FP32 vs FP64 within 1e-6."""
    p = CASES[case]()
    g, o = pair(p, torch, gparams=LAYOUTS[layout])
    for m in range(p.order):
        g.ao_iter = 3
        o.ao_iter = 3
        g.snmc(m, p.c, seed=99)
        o.snmc(m, p.c, seed=99)
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-6, 1e-5, f"{case} mode {m}")


@pytest.mark.parametrize("max_inner", [1, 3])
@pytest.mark.parametrize("split", [False, True])
def test_epoch_planted_cube(torch, max_inner, split):
    """One epoch (10 AO iterations at c = 0.1) of the 100^3 rank-10 problem: 1e-5."""
    p = synth.planted_rank10_100cube()
    gp = dict(SPLIT if split else {}, max_inner=max_inner)
    g, o = pair(p, torch, gparams=gp, oparams=dict(max_inner=max_inner))
    g.epoch(p.c, seed=4)
    o.epoch(p.c, seed=4)
    for m in range(p.order):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, f"mode {m}")
    assert g.ao_iter == o.ao_iter == 10


def test_epoch_zipf_split_rows_and_mode_order(torch):
    p = small_zipf()
    g, o = pair(p, torch, gparams=SPLIT)
    g.epoch(0.2, seed=8, mode_order=[2, 0, 1])
    o.epoch(0.2, seed=8, mode_order=[2, 0, 1])
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, f"mode {m}")
    st = g.stats()
    assert st["visits"] == o.visits and st["rows_skipped"] == o.rows_skipped


@pytest.mark.parametrize("rank", [10, 33])
def test_warm_power_method_epochs(torch, rank):
    """Warm-started power method (3 iterations from each row's last vector),
    light and split rows, two epochs, against the oracle's same reading."""
    p = synth.make_problem([60, 50, 40], rank, 30_000, sigma=0.01, test_frac=0.05, seed=40 + rank)
    params = dict(power_warm=1, power_iters=3)
    g, o = pair(p, torch, gparams=dict(params, heavy_rows=256, chunk=300), oparams=params)
    for e in range(2):
        g.epoch(0.25, seed=50 + e)
        o.epoch(0.25, seed=50 + e)
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, str((rank, m)))
    # new observations reset the kept vectors on both sides: the first epoch
    # after them matches a cold run with the same iteration count
    g2, o2 = pair(p, torch, gparams=dict(power_iters=3, heavy_rows=256, chunk=300), oparams=dict(power_iters=3))
    g.set_observed(p.idx_train, p.val_train)
    U0 = [g2.get_factor(m) for m in range(3)]
    for m in range(3):
        g.set_factor(m, U0[m])
    g.set_param("power_warm", 1)
    g.snmc(0, 0.25, seed=9)
    g2.snmc(0, 0.25, seed=9)
    np.testing.assert_array_equal(g.get_factor(0), g2.get_factor(0))


@pytest.mark.parametrize("rank", [1, 3, 8, 10, 16, 17, 31, 33, 64])
def test_ranks(torch, rank):
    p = synth.make_problem([60, 50, 40], rank, 30_000, sigma=0.01, test_frac=0.05, seed=rank)
    g, o = pair(p, torch, gparams=dict(heavy_rows=256, chunk=300))
    g.epoch(0.25, seed=rank)
    o.epoch(0.25, seed=rank)
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, str((rank, m)))


def test_bf16_storage_epoch(torch):
    p = synth.planted_rank10_100cube()
    g, o = pair(p, torch, gparams=dict(storage_bf16=1))
    g.epoch(p.c, seed=4)
    o.epoch(p.c, seed=4)
    for m in range(3):
        assert rel_err(g.get_factor(m), o.get_factor(m)) <= 2e-2, m


def test_predict_rmse_cost(torch):
    p = synth.planted_rank10_100cube()
    g, o = pair(p, torch)
    g.epoch(p.c, seed=4)
    o.epoch(p.c, seed=4)
    np.testing.assert_allclose(g.predict(p.idx_test), o.predict(p.idx_test), rtol=2e-5, atol=1e-6)
    assert g.rmse(p.idx_test, p.val_test) == pytest.approx(o.rmse(p.idx_test, p.val_test), rel=1e-4)
    assert g.cost() == pytest.approx(o.cost(), rel=1e-4)
    # device-pointer queries: an index out of range gives NaN and reads no factor row
    q = p.idx_test[:64].copy()
    q[5, 0] = p.dims[0]
    q[9, 2] = -3
    qd = torch.from_numpy(q).cuda()
    out = torch.empty(64, dtype=torch.float32, device="cuda")
    g.predict_dev(64, qd.data_ptr(), out.data_ptr())
    got = out.cpu().numpy()
    assert np.isnan(got[5]) and np.isnan(got[9])
    keep = np.ones(64, bool)
    keep[[5, 9]] = False
    np.testing.assert_allclose(got[keep], o.predict(q[keep]), rtol=2e-5, atol=1e-6)


def test_init_factors_match_oracle_rule(torch):
    p = synth.planted_rank10_100cube()
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream, init_seed=3)
    g.set_observed(p.idx_train, p.val_train)
    o = oracle.Oracle(p.dims, p.rank, p.lam)
    o.set_observed(p.idx_train, p.val_train.astype(np.float64))
    o.init_factors(3)
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-6, 1e-5)


def test_deterministic_and_resumable(torch):
    p = small_zipf()
    runs = []
    for _ in range(2):
        g, _o = pair(p, torch, gparams=SPLIT)
        g.epoch(0.1, seed=4)
        g.epoch(0.1, seed=5)
        runs.append(g.factors())
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)
    # checkpoint after one epoch, resume in a fresh handle
    g, _o = pair(p, torch, gparams=SPLIT)
    g.epoch(0.1, seed=4)
    ck = (g.factors(), g.ao_iter)
    h, _o2 = pair(p, torch, factors=[f.astype(np.float64) for f in ck[0]], gparams=SPLIT)
    h.ao_iter = ck[1]
    h.epoch(0.1, seed=5)
    for a, b in zip(h.factors(), runs[0]):
        np.testing.assert_array_equal(a, b)


def test_error_statuses_leave_handle_usable(torch):
    p = synth.planted_rank10_100cube()
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(ntc.NTCError) as e:
        g.epoch(0.1, seed=1)
    assert e.value.status == ntc.NTC_ERR_STATE
    g.set_observed(p.idx_train, p.val_train)
    bad = p.idx_train.copy()
    bad[5, 1] = 100
    with pytest.raises(ntc.NTCError) as e:
        g.set_observed(bad, p.val_train)
    assert e.value.status == ntc.NTC_ERR_INDEX
    for c in (0.0, -0.1, 1.5, float("nan")):
        with pytest.raises(ntc.NTCError) as e:
            g.epoch(c, seed=1)
        assert e.value.status == ntc.NTC_ERR_ARG
    with pytest.raises(ntc.NTCError):
        g.epoch(0.1, seed=1, mode_order=[0, 0, 1])
    with pytest.raises(ntc.NTCError):
        g.set_factor(0, -np.ones((100, 10), dtype=np.float32))
    with pytest.raises(ntc.NTCError):
        g.set_param("no_such_key", 1)
    with pytest.raises(ntc.NTCError) as e:
        g.predict(bad[:10])
    assert e.value.status == ntc.NTC_ERR_INDEX
    # the earlier observations are still in place: one epoch still matches the oracle
    U0 = synth.random_factors(p.dims, p.rank, 0.7, seed=101)
    o = oracle.Oracle(p.dims, p.rank, p.lam)
    o.set_observed(p.idx_train, p.val_train.astype(np.float64))
    for i, u in enumerate(U0):
        g.set_factor(i, u.astype(np.float32))
        o.set_factor(i, u)
    g.epoch(0.1, seed=2)
    o.epoch(0.1, seed=2)
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4)


def test_edge_cases(torch):
    # empty observation set: nothing to update, factors unchanged
    p = synth.make_problem([7, 5, 3], 4, 0, test_frac=0.0, seed=1)
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream)
    g.set_observed(p.idx_train, p.val_train)
    U = [np.full((d, 4), 0.5, np.float32) for d in p.dims]
    for i, u in enumerate(U):
        g.set_factor(i, u)
    g.epoch(0.5, seed=1)
    for a, b in zip(g.factors(), U):
        np.testing.assert_array_equal(a, b)
    assert g.stats()["visits"] == 0
    assert g.cost() == pytest.approx(0.5 * p.lam * sum((u.astype(np.float64) ** 2).sum() for u in U))
    # single-row modes, empty rows, duplicates, lambda = 0, c = 1, heavy rows with k = n
    rng = np.random.default_rng(2)
    idx = np.stack([rng.integers(0, 1, 5000), rng.integers(0, 40, 5000), rng.integers(0, 3, 5000) * 7],
                   1).astype(np.int32)
    idx[:50] = idx[0]
    vals = rng.random(5000).astype(np.float32)
    q = synth.Problem(dims=[1, 45, 21], rank=6, lam=0.0, c=1.0, factors=[], idx_train=idx, val_train=vals,
                      idx_test=idx[:10], val_test=vals[:10], val_test_clean=vals[:10].astype(np.float64),
                      sigma=0.0)
    for c in (1.0, 0.3):
        g, o = pair(q, torch, gparams=dict(heavy_rows=64, chunk=512))
        g.epoch(c, seed=3)
        o.epoch(c, seed=3)
        for m in range(3):
            assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, str((c, m)))


# ---- epoch-permutation sampling variant --------------------------------------------

def perm_mask(idx, mode, dim, c, seed, ao_iter, inner, max_inner=1):
    """The variant's sample of every row of `mode`, as a mask over bucket positions (oracle)."""
    row_ptr, _ = oracle.bucket(idx, mode, dim)
    T = int(np.ceil(1.0 / c - 1e-12))
    epoch, slot = ao_iter // T, (ao_iter % T) * max_inner + inner
    mask = np.zeros(idx.shape[0], dtype=np.uint8)
    for r in range(dim):
        q0, n = int(row_ptr[r]), int(row_ptr[r + 1] - row_ptr[r])
        k = oracle.sample_count(c, n)
        for j in range(k):
            mask[q0 + oracle.perm_index(seed, mode, epoch, r, n, (slot * k + j) % n)] = 1
    return mask


@pytest.mark.parametrize("split", [False, True])
def test_epoch_permutation_sampler_bit_exact(torch, split):
    p = small_zipf(nnz=60_000, dim=400)
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream, sampler=1,
                **(dict(heavy_rows=128, chunk=300) if split else {}))
    g.set_observed(p.idx_train, p.val_train)
    c, seed = 0.25, 4242
    for m in range(3):
        epoch_total = np.zeros(p.nnz, np.int32)
        for it in range(4, 8):                       # AO iterations 4..7 = epoch 1 (T = 4)
            got = g.sample_mask(m, c, seed, it, 0, p.nnz)
            np.testing.assert_array_equal(got, perm_mask(p.idx_train, m, p.dims[m], c, seed, it, 0))
            epoch_total += got
        assert epoch_total.max() == 1                # the epoch's minibatches are disjoint


@pytest.mark.parametrize("split", [False, True])
def test_epoch_permutation_epoch_parity(torch, split):
    p = small_zipf(nnz=120_000, dim=600)
    gp = dict(sampler=1, **(dict(heavy_rows=128, chunk=700) if split else {}))
    g, o = pair(p, torch, gparams=gp, oparams=dict(sampler=1))
    for e in range(2):
        g.epoch(0.2, seed=31 + e)
        o.epoch(0.2, seed=31 + e)
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, str(m))


@pytest.mark.parametrize("sampler", [0, 1], ids=["independent", "perm"])
@pytest.mark.parametrize("storage_bf16", [0, 1], ids=["fp32", "bf16"])
def test_light_rows_rank16_epochs(torch, sampler, storage_bf16):
    """Every row through the block-per-row kernel at R_pad = 16 (its
    shuffle-based Gram), both samplers and both storage forms, two epochs
    against the FP64 oracle."""
    p = small_zipf(nnz=120_000, dim=600, rank=12, seed=9)
    g, o = pair(p, torch, gparams=dict(tiny_rows=0, sampler=sampler, storage_bf16=storage_bf16),
                oparams=dict(sampler=sampler))
    for e in range(2):
        g.epoch(0.2, seed=51 + e)
        o.epoch(0.2, seed=51 + e)
    tol = (2e-2, 5e-2) if storage_bf16 else (1e-5, 1e-4)
    for m in range(3):
        assert_factor_close(g.get_factor(m), o.get_factor(m), *tol, str(m))


@pytest.mark.parametrize("overlap", [1, 2])
def test_light_rows_on_a_side_stream(torch, overlap):
    """overlap 1 / 2: light rows run on a second stream beside the split rows'
    sampler / Gram of the same mode update; the result is the same as in
    stream order."""
    p = small_zipf()
    g, o = pair(p, torch, gparams=dict(SPLIT, overlap=overlap))
    g2, _ = pair(p, torch, gparams=dict(SPLIT, overlap=0))
    for e in range(2):
        g.epoch(0.2, seed=61 + e)
        g2.epoch(0.2, seed=61 + e)
        o.epoch(0.2, seed=61 + e)
    for m in range(3):
        np.testing.assert_array_equal(g.get_factor(m), g2.get_factor(m))
        assert_factor_close(g.get_factor(m), o.get_factor(m), 1e-5, 1e-4, str(m))


def test_pipelined_sampling_matches_stream_order(torch):
    """pipeline = 1 (default): the next update's split-row sampling runs on its
    own stream with a second scratch set; results equal stream order bit for
    bit, also with the permutation sampler and after a change of c."""
    p = small_zipf()
    for extra in (dict(), dict(sampler=1)):
        a, _ = pair(p, torch, gparams=dict(SPLIT, **extra))
        b, _ = pair(p, torch, gparams=dict(SPLIT, pipeline=0, overlap=0, **extra))
        for c, seed in ((0.2, 71), (0.1, 72), (0.2, 73)):
            a.epoch(c, seed=seed)
            b.epoch(c, seed=seed)
        for m in range(3):
            np.testing.assert_array_equal(a.get_factor(m), b.get_factor(m))
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream)
    g.set_observed(p.idx_train, p.val_train)
    with pytest.raises(ntc.NTCError) as e:
        g.set_param("pipeline", 0)
    assert e.value.status == ntc.NTC_ERR_STATE


# ---- rows of at most 509 observations: one warp from sample to update ----

def _tiny_problem(order, rank, seed):
    """Rows of a few to a few hundred observations (Zipf skew), some above the
    one-warp limit and some split, so that all three row paths meet in an epoch."""
    dims = {2: [3000, 400], 3: [2000, 900, 300], 4: [900, 600, 200, 40]}[order]
    return synth.make_problem(dims, rank, 150_000, index_dist="zipf", zipf_s=1.0, sigma=0.02,
                              test_frac=0.05, seed=seed)


@pytest.mark.parametrize("order,rank,extra", [
    (3, 8, {}), (3, 16, {}), (3, 32, {}), (3, 64, {}), (3, 5, {}), (2, 24, {}), (4, 40, {}),
    (3, 32, dict(storage_bf16=1)), (3, 20, dict(max_inner=3)), (3, 12, dict(power_warm=1, power_iters=3)),
    (3, 32, dict(sampler=1)), (3, 64, dict(storage_bf16=1)), (3, 48, dict(power_warm=1, power_iters=3)),
    (3, 56, dict(max_inner=3)), (2, 64, {}), (4, 64, dict(sampler=1))],
    ids=["r8", "r16", "r32", "r64", "r5", "o2r24", "o4r40", "bf16", "inner3", "warm", "perm", "r64bf16",
         "r48warm", "r56inner3", "o2r64", "o4r64perm"])
def test_tiny_rows_epoch(torch, order, rank, extra):
    """Epoch parity with the one-warp kernel on, and the same epoch through the
    block-per-row kernel (tiny_rows 0): both against the FP64 oracle, and the
    sampled masks of both paths bit-exact."""
    p = _tiny_problem(order, rank, seed=70 + rank + order)
    oparams = {k: v for k, v in extra.items() if k in ("max_inner", "power_warm", "power_iters", "sampler")}
    tol = (2e-2, 5e-2) if extra.get("storage_bf16") else (1e-5, 1e-4)
    for tiny in (1, 0):
        g, o = pair(p, torch, gparams=dict(extra, tiny_rows=tiny, heavy_rows=1024, chunk=2048), oparams=oparams)
        g.epoch(0.2, seed=11)
        o.epoch(0.2, seed=11)
        for m in range(order):
            assert_factor_close(g.get_factor(m), o.get_factor(m), *tol, f"tiny={tiny} mode {m}")
        if not extra:
            for m in range(order):
                got = g.sample_mask(m, 0.2, 13, 3, 0, p.nnz)
                np.testing.assert_array_equal(got, oracle_mask(p.idx_train, m, p.dims[m], 0.2, 13, 3, 0))
        g.close()


@pytest.mark.parametrize("rank", [16, 64])
def test_tiny_rows_ties_and_full_rows(torch, rank):
    """c = 1 (every position of every row) and c = 0.999 (k = n - 1 for rows
    below 1000 observations): the bisection selects all but the largest key.
    At rank 64 the rows of at most 32 visits take the K-only launch."""
    p = _tiny_problem(3, rank, seed=5)
    for c in (1.0, 0.999, 0.5):
        g, o = pair(p, torch, gparams=dict(heavy_rows=1024, chunk=2048))
        g.snmc(1, c, seed=3)
        o.snmc(1, c, seed=3)
        assert_factor_close(g.get_factor(1), o.get_factor(1), 1e-6, 1e-5, f"c={c}")
        got = g.sample_mask(2, c, 7, 1, 0, p.nnz)
        np.testing.assert_array_equal(got, oracle_mask(p.idx_train, 2, p.dims[2], c, 7, 1, 0))
        g.close()
