"""Oracle pins: Philox4x32-10, per-mode bucketing and per-row sampling.

Each test pins the oracle to something other than itself: published
known-answer vectors, numpy's stable argsort, order properties of the
selected subset and the uniform distribution of k-subsets (Sec. II-B:
"sample, uniformly at random, B_{l,p} nonzero elements").
"""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(oracle_mod):
    for ctr, key, out in _kat():
        got = oracle_mod.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == out


def test_sample_key_is_word_q_mod_4_of_block_q_div_4(oracle_mod):
    seed = 0x0123456789ABCDEF
    for mode, k, l, q in [(0, 0, 0, 0), (0, 0, 0, 3), (2, 7, 1, 12345), (2, 7, 1, 12346),
                          (3, 2**31 + 5, 4, 2**31 - 1), (1, 9, 0, 2**31 - 4)]:
        w = oracle_mod.philox4x32_10([mode, k & 0xFFFFFFFF, l, q // 4], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle_mod.sample_key(seed, mode, k, l, q) == int(w[q % 4])


def test_keys_of_one_block_are_jointly_uniform(oracle_mod):
    """The four positions that share a Philox block: the joint histogram of the
    top 3 bits of the keys of positions 4g + j and 4g + j + 1 over 8192 blocks
    is flat (chi2, 63 dof), for each neighbouring pair of words."""
    for j in range(3):
        a = np.array([oracle_mod.sample_key(11, 2, 5, 0, 4 * g + j) for g in range(8192)], dtype=np.uint64)
        b = np.array([oracle_mod.sample_key(11, 2, 5, 0, 4 * g + j + 1) for g in range(8192)], dtype=np.uint64)
        cell = ((a >> 29) * 8 + (b >> 29)).astype(np.int64)
        h = np.bincount(cell, minlength=64)
        chi2 = ((h - 128.0) ** 2 / 128.0).sum()
        assert chi2 < 110.0  # p ~ 2e-4 at 63 dof


def test_philox_uniformity(oracle_mod):
    # 4096 consecutive counters: word-0 top-4-bit histogram is flat (chi2, 15 dof)
    keys = np.array([oracle_mod.sample_key(7, 1, 3, 0, q) for q in range(4096)], dtype=np.uint64)
    h = np.bincount((keys >> 28).astype(np.int64), minlength=16)
    chi2 = ((h - 256.0) ** 2 / 256.0).sum()
    assert chi2 < 45.0  # p ~ 1e-4 at 15 dof


@pytest.mark.parametrize("nnz,dim,order,mode", [(0, 5, 3, 0), (1, 1, 2, 1), (1000, 17, 3, 1),
                                                 (5000, 300, 4, 3)])
def test_bucket_matches_stable_argsort(oracle_mod, nnz, dim, order, mode):
    rng = np.random.default_rng(nnz + dim)
    idx = rng.integers(0, dim, size=(nnz, order)).astype(np.int32)
    row_ptr, perm = oracle_mod.bucket(idx, mode, dim)
    assert row_ptr[0] == 0 and row_ptr[-1] == nnz
    np.testing.assert_array_equal(np.diff(row_ptr), np.bincount(idx[:, mode], minlength=dim))
    np.testing.assert_array_equal(perm, np.argsort(idx[:, mode], kind="stable"))


def test_bucket_rejects_out_of_range(oracle_mod):
    idx = np.array([[0, 1], [3, 0]], dtype=np.int32)
    with pytest.raises(IndexError):
        oracle_mod.bucket(idx, 0, 3)


def test_sample_count_floor(oracle_mod):
    assert oracle_mod.sample_count(0.1, 9) == 0
    assert oracle_mod.sample_count(0.1, 10) == 1
    assert oracle_mod.sample_count(0.1, 19) == 1
    assert oracle_mod.sample_count(1.0, 17) == 17
    assert oracle_mod.sample_count(0.3, 10) == 3  # 0.3*10 = 3.0000000000000004 in IEEE
    assert oracle_mod.sample_count(0.7, 10) == 7  # 0.7*10 = 7.000000000000001
    assert oracle_mod.sample_count(0.29, 100) == 28  # 0.29*100 = 28.999999999999996


@pytest.mark.parametrize("n,k", [(1, 1), (5, 0), (9, 3), (64, 6), (1000, 100), (333, 333)])
def test_sample_is_k_smallest(oracle_mod, n, k):
    seed, mode, it, inner, q0 = 99, 1, 5, 0, 1234
    sel = oracle_mod.sample_row(seed, mode, it, inner, q0, n, k)
    assert len(sel) == k and len(set(sel.tolist())) == k
    assert np.all((sel >= q0) & (sel < q0 + n))
    keys = {q: oracle_mod.sample_key(seed, mode, it, inner, q) for q in range(q0, q0 + n)}
    chosen = set(sel.tolist())
    if 0 < k < n:
        worst_in = max((keys[q], q) for q in chosen)
        best_out = min((keys[q], q) for q in range(q0, q0 + n) if q not in chosen)
        assert worst_in < best_out


def test_sample_subsets_uniform(oracle_mod):
    # every 2-subset of 5 positions equally likely (10 cells), and 3-of-7 marginals
    n, k, T = 5, 2, 6000
    counts = {}
    for t in range(T):
        s = tuple(sorted(oracle_mod.sample_row(3, 0, t, 0, 40, n, k).tolist()))
        counts[s] = counts.get(s, 0) + 1
    assert set(counts) == set(itertools.combinations(range(40, 45), 2))
    exp = T / 10.0
    chi2 = sum((v - exp) ** 2 / exp for v in counts.values())
    assert chi2 < 33.7  # 9 dof, p ~ 1e-4
    n, k = 7, 3
    freq = np.zeros(n)
    for t in range(T):
        for q in oracle_mod.sample_row(11, 2, 0, t, 0, n, k):
            freq[q] += 1
    exp = T * k / n
    assert ((freq - exp) ** 2 / exp).sum() < 27.9  # 6 dof, p ~ 1e-4


def test_sample_streams_independent_across_mode_iter_inner(oracle_mod):
    base = oracle_mod.sample_row(5, 0, 0, 0, 0, 200, 20)
    for args in [(5, 1, 0, 0), (5, 0, 1, 0), (5, 0, 0, 1), (6, 0, 0, 0)]:
        other = oracle_mod.sample_row(*args, 0, 200, 20)
        assert set(other.tolist()) != set(base.tolist())


# ---- epoch-permutation sampling variant ------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 31, 32, 33, 100, 257, 1000, 4097])
def test_epoch_permutation_is_a_bijection(oracle_mod, n):
    oracle = oracle_mod
    for (seed, mode, epoch, row) in [(1, 0, 0, 0), (2, 1, 5, 7), (2 ** 40 + 3, 2, 9, 123456)]:
        img = [oracle.perm_index(seed, mode, epoch, row, n, i) for i in range(n)]
        assert sorted(img) == list(range(n))


@pytest.mark.parametrize("n,c", [(100, 0.1), (97, 0.2), (1000, 0.05), (64, 0.25), (10, 0.3)])
def test_epoch_slots_are_disjoint_stretches(oracle_mod, n, c):
    oracle = oracle_mod
    k = oracle.sample_count(c, n)
    T = int(np.ceil(1.0 / c - 1e-12))
    seen = []
    for s in range(T):
        seen += [oracle.perm_index(9, 0, 4, 11, n, (s * k + j) % n) for j in range(k)]
    if T * k <= n:
        assert len(set(seen)) == T * k                       # one epoch reads an entry at most once
    else:
        assert len(set(seen)) == n                           # ... and every entry when slots wrap around


def test_epoch_permutation_is_uniform_and_varies_with_its_counter(oracle_mod):
    oracle = oracle_mod
    n, trials = 10, 20000
    first = np.bincount([oracle.perm_index(3, 0, e, 0, n, 0) for e in range(trials)], minlength=n)
    chi2 = ((first - trials / n) ** 2 / (trials / n)).sum()
    assert chi2 < 27.9                                       # chi^2_9 at p = 0.001
    # pairs (pi(0), pi(1)) cover the 90 ordered pairs evenly
    pairs = np.zeros((n, n))
    for e in range(trials):
        pairs[oracle.perm_index(3, 0, e, 1, n, 0), oracle.perm_index(3, 0, e, 1, n, 1)] += 1
    cells = pairs[~np.eye(n, dtype=bool)]
    chi2 = ((cells - trials / 90) ** 2 / (trials / 90)).sum()
    assert chi2 < 137.2                                      # chi^2_89 at p = 0.001
    base = [oracle.perm_index(3, 0, 0, 0, 1000, i) for i in range(50)]
    for kw in [dict(seed=4), dict(mode=1), dict(epoch=1), dict(row=1)]:
        a = dict(seed=3, mode=0, epoch=0, row=0)
        a.update(kw)
        other = [oracle.perm_index(a["seed"], a["mode"], a["epoch"], a["row"], 1000, i) for i in range(50)]
        assert other != base, kw
