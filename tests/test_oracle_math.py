"""Oracle pins for the NMC row update (Sec. II-B, Algorithm 1) and the AO loop
(Algorithm 2), each against an independent statement of the mathematics:
dense Khatri-Rao / Kronecker formulas built with numpy, finite differences of
the cost, numpy eigvalsh, closed forms, scipy's NNLS, and monotone descent."""
import numpy as np
import pytest

from paper_2109_09534_gb300 import synth


def khatri_rao(mats):
    """Column-wise Kronecker product, last matrix's row index fastest."""
    out = mats[0]
    for m in mats[1:]:
        out = (out[:, None, :] * m[None, :, :]).reshape(-1, out.shape[1])
    return out


def unfold(X, n):
    """Mode-n unfolding with the lowest remaining mode varying fastest (Sec. II)."""
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def kr_for_mode(U, n):
    """K for mode n: U^(N) kr ... kr U^(n+1) kr U^(n-1) kr ... kr U^(1)."""
    others = [U[j] for j in range(len(U)) if j != n]
    return khatri_rao(others[::-1])


def dense(U):
    X = np.einsum("ir,jr,kr->ijk", *U) if len(U) == 3 else None
    return X


def full_cells(dims):
    g = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1)
    return g.reshape(-1, len(dims)).astype(np.int32)


def make_oracle(oracle_mod, dims, R, lam, idx, vals, U, **params):
    o = oracle_mod.Oracle(dims, R, lam)
    for k, v in params.items():
        o.set_param(k, v)
    o.set_observed(idx, vals)
    for i, u in enumerate(U):
        o.set_factor(i, u)
    return o


@pytest.fixture
def tiny_full():
    rng = np.random.default_rng(0)
    dims, R = [4, 5, 6], 3
    U = [rng.random((d, R)) + 0.1 for d in dims]
    X = dense(U) + 0.3 * rng.random(dims)
    idx = full_cells(dims)
    vals = X[tuple(idx.T)]
    return dims, R, U, X, idx, vals


def test_dense_gradient_full_observation(oracle_mod, tiny_full):
    """c = 1 on a fully observed tensor: grad = U (K^T K) - X_(n) K + lambda U (eq. gradient_F)."""
    dims, R, U, X, idx, vals = tiny_full
    lam = 0.05
    for n in range(3):
        o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U, debug=1)
        o.snmc(n, 1.0, seed=1)
        K = kr_for_mode(U, n)
        G = U[n] @ (K.T @ K) - unfold(X, n) @ K + lam * U[n]
        for p in range(dims[n]):
            np.testing.assert_allclose(o.debug_row(p)["grad"], G[p], rtol=1e-12, atol=1e-12)


def test_hessian_block_matches_kronecker_form(oracle_mod):
    """H_p is the row-p diagonal block of (B^T kron I_P) diag(vec M) (B kron I_P) + lambda I (eq. hessian_F)."""
    rng = np.random.default_rng(1)
    dims, R, lam = [3, 4, 5], 2, 0.2
    U = [rng.random((d, R)) for d in dims]
    cells = full_cells(dims)
    keep = rng.random(len(cells)) < 0.6
    idx = cells[keep]
    vals = rng.random(idx.shape[0])
    M = np.zeros(dims)
    M[tuple(idx.T)] = 1.0
    n = 1
    o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U, debug=1)
    o.snmc(n, 1.0, seed=2)
    B = kr_for_mode(U, n)
    P = dims[n]
    Mn = unfold(M, n)
    Hfull = np.kron(B.T, np.eye(P)) @ np.diag(Mn.flatten(order="F")) @ np.kron(B, np.eye(P)) \
        + lam * np.eye(P * R)
    for p in range(P):
        sl = [p + P * r for r in range(R)]
        d = o.debug_row(p)
        if d["kp"] == 0:
            continue
        np.testing.assert_allclose(d["H"], Hfull[np.ix_(sl, sl)], rtol=1e-12, atol=1e-12)


def test_gradient_matches_finite_differences_of_cost(oracle_mod):
    """c = 1: the row gradient is the derivative of eq. 3's cost (central differences)."""
    rng = np.random.default_rng(2)
    dims, R, lam = [5, 4, 3], 3, 0.03
    U = [rng.random((d, R)) + 0.2 for d in dims]
    cells = full_cells(dims)
    idx = cells[rng.random(len(cells)) < 0.7]
    vals = rng.random(idx.shape[0]) * 2
    n, p = 0, 2
    o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U, debug=1)
    o.snmc(n, 1.0, seed=3)
    g = o.debug_row(p)["grad"]
    h = 1e-6
    fd = np.zeros(R)
    for r in range(R):
        vals_c = []
        for s in (+1, -1):
            V = [u.copy() for u in U]
            V[n][p, r] += s * h
            q = make_oracle(oracle_mod, dims, R, lam, idx, vals, V)
            vals_c.append(q.cost())
        fd[r] = (vals_c[0] - vals_c[1]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-8)


def test_lmax_eigvalsh_and_power_gap(oracle_mod):
    p = synth.planted_rank10_100cube()
    rng = np.random.default_rng(5)
    U = [rng.random((d, p.rank)) for d in p.dims]
    o = make_oracle(oracle_mod, p.dims, p.rank, p.lam, p.idx_train, p.val_train, U, debug=1)
    o.snmc(0, p.c, seed=4)
    gaps = []
    for row in range(p.dims[0]):
        d = o.debug_row(row)
        if d["kp"] == 0:
            continue
        ev = np.linalg.eigvalsh(d["H"])[-1]
        assert d["L_exact"] == pytest.approx(ev, rel=1e-12)
        assert d["L"] <= ev * (1 + 1e-12)
        gaps.append((ev - d["L"]) / ev)
    assert max(gaps) <= 1e-6


def test_lmax_closed_forms(oracle_mod):
    rng = np.random.default_rng(3)
    R = 6
    k = rng.random(R)
    H = np.outer(k, k) + 0.01 * np.eye(R)          # one sample: ||k||^2 + lambda
    assert oracle_mod.jacobi_lmax(H) == pytest.approx(k @ k + 0.01, rel=1e-13)
    assert oracle_mod.power_lmax(H, 10) == pytest.approx(k @ k + 0.01, rel=1e-12)
    ks = rng.random(9)                               # R = 1: sum k^2 + lambda
    H1 = np.array([[ks @ ks + 0.5]])
    assert oracle_mod.power_lmax(H1, 10) == pytest.approx(ks @ ks + 0.5, rel=1e-15)
    assert oracle_mod.jacobi_lmax(H1) == pytest.approx(ks @ ks + 0.5, rel=1e-15)


def test_rank1_single_entry_step_is_ridge_minimizer(oracle_mod):
    """R = 1, one observation per row, c = 1: one step with L = k^2 + lambda lands
    on the 1-D ridge solution (x k / (k^2 + lambda))_+ (Alg. 1 lines 6-11)."""
    dims, lam = [3, 1], 0.25
    idx = np.array([[0, 0], [1, 0], [2, 0]], dtype=np.int32)
    vals = np.array([2.0, 0.5, 0.0])
    U = [np.array([[0.7], [0.1], [0.9]]), np.array([[1.5]])]
    o = make_oracle(oracle_mod, dims, 1, lam, idx, vals, U)
    o.snmc(0, 1.0, seed=0)
    kk = 1.5
    want = np.maximum(0, vals * kk / (kk * kk + lam))
    np.testing.assert_allclose(o.get_factor(0)[:, 0], want, rtol=1e-14, atol=1e-15)


def test_nonnegativity_beta_range_and_skips(oracle_mod):
    p = synth.planted_rank10_100cube()
    rng = np.random.default_rng(6)
    U = [rng.random((d, p.rank)) * 3 for d in p.dims]   # far from the data: steps hit the bound
    o = make_oracle(oracle_mod, p.dims, p.rank, p.lam, p.idx_train, p.val_train, U,
                    debug=1, max_inner=3)
    o.snmc(2, 0.05, seed=9)
    A = o.get_factor(2)
    assert np.all(A >= 0) and np.any(A == 0)
    for row in range(p.dims[2]):
        d = o.debug_row(row)
        if d["kp"]:
            assert 0 <= d["beta"] < 1
    # rows with fewer than 1/c observations are skipped and keep their values
    idx = p.idx_train
    counts = np.bincount(idx[:, 2], minlength=p.dims[2])
    o2 = make_oracle(oracle_mod, p.dims, p.rank, p.lam, idx, p.val_train, U)
    o2.snmc(2, 0.5 / counts.min(), seed=1)   # k_p = floor(c n_p): the smallest rows get 0
    skipped = np.floor((0.5 / counts.min()) * counts) == 0
    assert skipped.any() and o2.rows_skipped == skipped.sum()
    np.testing.assert_array_equal(o2.get_factor(2)[skipped], U[2][skipped])


def test_cost_nonincreasing_full_batch_exact_L(oracle_mod):
    """c = 1, MAX_INNER = 1, L_p = lambda_max(H_p): each row update is a projected
    gradient step with step 1/L_p on its own separable subproblem, so the cost of
    eq. 3 never increases (Sec. II-B, step-size motivation)."""
    rng = np.random.default_rng(7)
    dims, R, lam = [12, 10, 8], 4, 1e-2
    cells = full_cells(dims)
    idx = cells[rng.random(len(cells)) < 0.3]
    Ut = [rng.random((d, R)) for d in dims]
    vals = np.einsum("er,er,er->e", Ut[0][idx[:, 0]], Ut[1][idx[:, 1]], Ut[2][idx[:, 2]])
    vals = vals + 0.05 * rng.standard_normal(len(vals))
    U = [rng.random((d, R)) for d in dims]
    o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U, lp_exact=1)
    prev = o.cost()
    for it in range(6):
        for n in (2, 0, 1):
            o.snmc(n, 1.0, seed=it)
            cur = o.cost()
            assert cur <= prev * (1 + 1e-13)
            prev = cur


def test_ao_iteration_matches_dense_recomputation(oracle_mod):
    """Algorithm 2 with c = 1, MAX_INNER = 1, exact L_p and a permuted mode
    order, replayed with dense numpy formulas (eq. gradient_F, hessian_F) and
    Gauss-Seidel use of the factors already updated (K_k^(i) definition)."""
    rng = np.random.default_rng(8)
    dims, R, lam = [5, 6, 4], 3, 0.02
    cells = full_cells(dims)
    idx = cells[rng.random(len(cells)) < 0.5]
    vals = rng.random(idx.shape[0])
    U = [rng.random((d, R)) for d in dims]
    order = [2, 0, 1]
    o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U, lp_exact=1)
    o.epoch(1.0, seed=5, mode_order=order)
    M = np.zeros(dims)
    M[tuple(idx.T)] = 1
    X = np.zeros(dims)
    X[tuple(idx.T)] = vals
    V = [u.copy() for u in U]
    for n in order:
        K = kr_for_mode(V, n)
        Mn, Xn = unfold(M, n), unfold(X, n)
        grad = -(Mn * Xn - Mn * (V[n] @ K.T)) @ K + lam * V[n]
        new = V[n].copy()
        for p in range(dims[n]):
            if Mn[p].sum() == 0:
                continue
            H = K.T @ np.diag(Mn[p]) @ K + lam * np.eye(R)
            L = np.linalg.eigvalsh(H)[-1]
            new[p] = np.maximum(0, V[n][p] - grad[p] / L)
        V[n] = new
    for n in range(3):
        np.testing.assert_allclose(o.get_factor(n), V[n], rtol=1e-11, atol=1e-13)
    assert o.ao_iter == 1


def test_minibatch_update_matches_dense_masked_formula(oracle_mod):
    """c = 0.5: the row update uses M_hat_l (eq. M_hat_def) in place of M; M_hat is
    rebuilt from the pinned sampler and bucket, the step from dense formulas."""
    rng = np.random.default_rng(9)
    dims, R, lam = [6, 5, 4], 3, 0.05
    cells = full_cells(dims)
    idx = cells[rng.random(len(cells)) < 0.8]
    vals = rng.random(idx.shape[0])
    U = [rng.random((d, R)) for d in dims]
    n, c, seed = 0, 0.5, 77
    o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U, lp_exact=1)
    o.ao_iter = 3
    o.snmc(n, c, seed)
    row_ptr, perm = oracle_mod.bucket(idx, n, dims[n])
    Mh = np.zeros(dims)
    for p in range(dims[n]):
        cnt = row_ptr[p + 1] - row_ptr[p]
        k = oracle_mod.sample_count(c, cnt)
        for q in oracle_mod.sample_row(seed, n, 3, 0, row_ptr[p], cnt, k):
            Mh[tuple(idx[perm[q]])] = 1
    X = np.zeros(dims)
    X[tuple(idx.T)] = vals
    K = kr_for_mode(U, n)
    Mn, Xn = unfold(Mh, n), unfold(X, n)
    grad = -(Mn * Xn - Mn * (U[n] @ K.T)) @ K + lam * U[n]
    want = U[n].copy()
    for p in range(dims[n]):
        if Mn[p].sum() == 0:
            continue
        H = K.T @ np.diag(Mn[p]) @ K + lam * np.eye(R)
        want[p] = np.maximum(0, U[n][p] - grad[p] / np.linalg.eigvalsh(H)[-1])
    np.testing.assert_allclose(o.get_factor(n), want, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("lp_exact", [1, 0])
def test_inner_loop_converges_to_ridge_nnls(oracle_mod, lp_exact):
    """One row, c = 1, MAX_INNER = 2000: Algorithm 1 converges to the minimizer of
    1/2||x - K y||^2 + lambda/2 ||y||^2 over y >= 0 (eq. matrix_NMC), which
    scipy's NNLS gives for the stacked system [K; sqrt(lambda) I] y = [x; 0]."""
    from scipy.optimize import nnls
    rng = np.random.default_rng(10)
    Q, R, lam = 40, 4, 0.05
    K = rng.random((Q, R))
    x = rng.random(Q) * 2 - 0.3          # some targets push coordinates to the bound
    x[::3] = -0.5
    idx = np.stack([np.zeros(Q, np.int32), np.arange(Q, dtype=np.int32)], 1)
    o = make_oracle(oracle_mod, [1, Q], R, lam, idx, x, [np.full((1, R), 0.3), K],
                    max_inner=2000, lp_exact=lp_exact)
    o.snmc(0, 1.0, seed=0)
    y_ref, _ = nnls(np.vstack([K, np.sqrt(lam) * np.eye(R)]), np.concatenate([x, np.zeros(R)]))
    np.testing.assert_allclose(o.get_factor(0)[0], y_ref, atol=1e-8)


def test_predict_rmse_cost_against_dense(oracle_mod, tiny_full):
    dims, R, U, X, idx, vals = tiny_full
    lam = 0.1
    o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U)
    model = dense(U)
    q = idx[::7]
    np.testing.assert_allclose(o.predict(q), model[tuple(q.T)], rtol=1e-13)
    want_rmse = np.sqrt(np.mean((vals[::7] - model[tuple(q.T)]) ** 2))
    assert o.rmse(q, vals[::7]) == pytest.approx(want_rmse, rel=1e-12)
    want_cost = 0.5 * np.sum((X - model) ** 2) + 0.5 * lam * sum((u * u).sum() for u in U)
    assert o.cost() == pytest.approx(want_cost, rel=1e-12)


def test_init_factors_scale_and_range(oracle_mod):
    p = synth.planted_rank10_100cube()
    o = oracle_mod.Oracle(p.dims, p.rank, p.lam)
    o.set_observed(p.idx_train, p.val_train)
    o.init_factors(3)
    a = (np.mean(p.val_train.astype(np.float64)) / p.rank) ** (1 / 3)
    for U in o.factors():
        assert U.min() > 0 and U.max() < 2 * a
        assert abs(U.mean() - a) < 0.1 * a  # 5 standard errors of a 1000-sample mean


def test_planted_recovery_small(oracle_mod):
    """Planted rank-10 100^3 tensor, 5% observed, sigma = 0.01 (high SNR):
    at c = 0.1 the held-out RMSE reaches the noise floor (1.5 sigma, a
    constant calibrated on this oracle: the paper prints no value) within 80
    epochs, and after 20 epochs the small minibatch is ahead of the full batch,
    the high-SNR trend of Sec. IV-B.  (Over ten sample streams the RMSE after
    40 epochs ranges from 2.0 to 6.1 sigma, so the epoch budget leaves room for
    the stream's variance.)"""
    p = synth.planted_rank10_100cube()

    def run(c, epochs):
        o = oracle_mod.Oracle(p.dims, p.rank, p.lam)
        o.set_observed(p.idx_train, p.val_train)
        o.init_factors(3)
        r0 = o.rmse(p.idx_test, p.val_test)
        out = []
        for ep in range(epochs):
            o.epoch(c, seed=4 + ep)
            out.append(o.rmse(p.idx_test, p.val_test))
        return r0, out

    r0, small = run(0.1, 80)
    _, full = run(1.0, 20)
    assert small[19] < 0.5 * full[19]
    assert small[-1] < 0.1 * r0
    assert small[-1] < 1.5 * p.sigma


# ---- warm-started power method (the cheaper-L_p topic of Sec. II-B) ----------

def test_warm_power_method_continues_the_cold_iteration_exactly(oracle_mod):
    oracle = oracle_mod
    rng = np.random.default_rng(11)
    for R in (1, 3, 8, 17):
        A = rng.random((R, R + 3))
        H = A @ A.T + 1e-3 * np.eye(R)
        for t1, t2 in ((1, 9), (4, 6), (9, 1)):
            mu1, v1 = oracle.power_lmax_v(H, t1)
            mu2, v2 = oracle.power_lmax_v(H, t2, v1)
            assert mu2 == oracle.power_lmax(H, t1 + t2)
            assert abs(np.linalg.norm(v2) - 1.0) < 1e-12


def test_warm_start_tracks_a_slowly_changing_matrix_better_than_cold(oracle_mod):
    oracle = oracle_mod
    rng = np.random.default_rng(12)
    R = 16
    A = rng.random((R, 40))
    v = None
    warm_err, cold_err = [], []
    for _ in range(30):
        A = A + 0.02 * rng.random(A.shape)         # the next minibatch's H is close to the last
        H = A @ A.T + 1e-3 * np.eye(R)
        exact = np.linalg.eigvalsh(H)[-1]
        mu_w, v = oracle.power_lmax_v(H, 2, v)
        warm_err.append((exact - mu_w) / exact)
        cold_err.append((exact - oracle.power_lmax(H, 2)) / exact)
    assert np.all(np.array(warm_err) >= -1e-12)    # Rayleigh quotients never exceed lambda_max
    assert np.mean(warm_err[5:]) < 0.1 * np.mean(cold_err[5:])


def test_oracle_warm_start_begins_cold_and_then_differs(oracle_mod):
    oracle = oracle_mod
    p = synth.planted_rank10_100cube()
    runs = []
    for warm in (0, 1):
        o = oracle.Oracle(p.dims, p.rank, p.lam)
        o.set_param("power_warm", warm)
        o.set_param("power_iters", 3)
        o.set_observed(p.idx_train, p.val_train.astype(np.float64))
        o.init_factors(3)
        o.snmc(0, p.c, seed=5)
        first = o.get_factor(0).copy()
        o.ao_iter = 1
        o.snmc(0, p.c, seed=5)
        runs.append((first, o.get_factor(0).copy()))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])   # first call: v0 = ones/sqrt(R) both ways
    assert not np.array_equal(runs[0][1], runs[1][1])       # second call starts from the kept vector


# ---- epoch-permutation sampling variant (Sec. IV epoch) ----

def test_epoch_permutation_update_matches_dense_masked_formula(oracle_mod):
    """sampler = 1, c = 0.5, AO iteration 3 = slot 1 of epoch 1 (T = 2): M_hat
    is rebuilt from the permutation's stretch, the step from dense formulas."""
    rng = np.random.default_rng(19)
    dims, R, lam = [6, 5, 4], 3, 0.05
    cells = full_cells(dims)
    idx = cells[rng.random(len(cells)) < 0.8]
    vals = rng.random(idx.shape[0])
    U = [rng.random((d, R)) for d in dims]
    n, c, seed = 1, 0.5, 78
    o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U, lp_exact=1, sampler=1)
    o.ao_iter = 3
    o.snmc(n, c, seed)
    row_ptr, perm = oracle_mod.bucket(idx, n, dims[n])
    Mh = np.zeros(dims)
    for p in range(dims[n]):
        cnt = row_ptr[p + 1] - row_ptr[p]
        k = oracle_mod.sample_count(c, cnt)
        for j in range(k):
            q = row_ptr[p] + oracle_mod.perm_index(seed, n, 1, p, cnt, (1 * k + j) % cnt)
            Mh[tuple(idx[perm[q]])] = 1
    X = np.zeros(dims)
    X[tuple(idx.T)] = vals
    K = kr_for_mode(U, n)
    Mn, Xn = unfold(Mh, n), unfold(X, n)
    grad = -(Mn * Xn - Mn * (U[n] @ K.T)) @ K + lam * U[n]
    want = U[n].copy()
    for p in range(dims[n]):
        if Mn[p].sum() == 0:
            continue
        H = K.T @ np.diag(Mn[p]) @ K + lam * np.eye(R)
        want[p] = np.maximum(0, U[n][p] - grad[p] / np.linalg.eigvalsh(H)[-1])
    np.testing.assert_allclose(o.get_factor(n), want, rtol=1e-11, atol=1e-13)


# ---- momentum and extrapolation (Alg. 1 lines 12-13) and the epoch length ----

@pytest.mark.parametrize("c", [1.0, 0.5])
def test_inner_iterations_match_dense_momentum_replay(oracle_mod, c):
    """MAX_INNER = 3 on one mode with exact L_p, replayed densely: each inner
    iteration l rebuilds M_hat_l from the pinned sampler (inner counter l), takes
    the gradient at the extrapolated point Y_l (lines 6-8 with Y_l, not A_l),
    A_{l+1} = (Y_l - grad / L_p)_+ (line 11), beta = (sqrt(L_p) - sqrt(lambda)) /
    (sqrt(L_p) + sqrt(lambda)) (line 12) and Y_{l+1} = A_{l+1} + beta (A_{l+1} -
    A_l) (line 13).  Rows with k_p = 0 keep A and Y.  Iterations 2 and 3 start
    from Y_1 and Y_2, so a wrong beta or a wrong extrapolation changes A_3."""
    rng = np.random.default_rng(21 if c == 1.0 else 22)
    dims, R, lam = [7, 5, 4], 3, 0.04
    cells = full_cells(dims)
    idx = cells[rng.random(len(cells)) < 0.7]
    vals = rng.random(idx.shape[0]) * 1.5
    U = [rng.random((d, R)) + 0.05 for d in dims]
    n, seed, k_ao, inner = 0, 31, 5, 3
    o = make_oracle(oracle_mod, dims, R, lam, idx, vals, U, lp_exact=1, max_inner=inner, debug=1)
    o.ao_iter = k_ao
    o.snmc(n, c, seed)
    row_ptr, perm = oracle_mod.bucket(idx, n, dims[n])
    X = np.zeros(dims)
    X[tuple(idx.T)] = vals
    Xn = unfold(X, n)
    K = kr_for_mode(U, n)
    A, Y = U[n].copy(), U[n].copy()
    beta_last = np.zeros(dims[n])
    for l in range(inner):
        Mh = np.zeros(dims)
        for p in range(dims[n]):
            cnt = row_ptr[p + 1] - row_ptr[p]
            k = oracle_mod.sample_count(c, cnt)
            for q in oracle_mod.sample_row(seed, n, k_ao, l, row_ptr[p], cnt, k):
                Mh[tuple(idx[perm[q]])] = 1
        Mn = unfold(Mh, n)
        A_new, Y_new = A.copy(), Y.copy()
        for p in range(dims[n]):
            if Mn[p].sum() == 0:
                continue
            grad = -(Mn[p] * Xn[p]) @ K + (Mn[p] * (Y[p] @ K.T)) @ K + lam * Y[p]
            H = K.T @ np.diag(Mn[p]) @ K + lam * np.eye(R)
            L = np.linalg.eigvalsh(H)[-1]
            a_next = np.maximum(0.0, Y[p] - grad / L)
            beta = (np.sqrt(L) - np.sqrt(lam)) / (np.sqrt(L) + np.sqrt(lam))
            A_new[p] = a_next
            Y_new[p] = a_next + beta * (a_next - A[p])
            beta_last[p] = beta
        A, Y = A_new, Y_new
    np.testing.assert_allclose(o.get_factor(n), A, rtol=1e-11, atol=1e-13)
    for p in range(dims[n]):
        d = o.debug_row(p)
        if d["kp"] > 0:
            assert d["beta"] == pytest.approx(beta_last[p], rel=1e-11)
    # the replay is not vacuous: the extrapolated points moved the result
    assert np.abs(A - U[n]).max() > 1e-3


@pytest.mark.parametrize("c,T", [(0.1, 10), (0.3, 4), (0.37, 3), (1.0 / 3.0, 3), (0.25, 4), (1.0, 1)])
def test_epoch_runs_ceil_one_over_c_ao_iterations(oracle_mod, c, T):
    """An epoch is the number of AO iterations that touches every observation
    once on average (Sec. IV): ceil(1/c - 1e-12), so that a 1/c that rounding
    left just above an integer counts as that integer (c = 1/3 gives 3)."""
    rng = np.random.default_rng(23)
    dims, R = [6, 5, 4], 2
    cells = full_cells(dims)
    idx = cells[rng.random(len(cells)) < 0.9]
    vals = rng.random(idx.shape[0])
    o = make_oracle(oracle_mod, dims, R, 0.01, idx, vals, [rng.random((d, R)) for d in dims])
    o.ao_iter = 7
    o.epoch(c, seed=3)
    assert o.ao_iter == 7 + T
    # every AO iteration updated every mode: the visits are T times one
    # iteration's sum over the modes of floor(c n_p)
    per_iter = 0
    for m in range(3):
        counts = np.bincount(idx[:, m], minlength=dims[m])
        per_iter += int(np.floor(c * counts.astype(np.float64)).sum())
    assert o.visits == T * per_iter
