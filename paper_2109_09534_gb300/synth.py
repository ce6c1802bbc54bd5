"""Seeded synthetic tensor-completion inputs.

This module only manufactures inputs: planted nonnegative CPD factors, observed
index sets (uniform cells without replacement, or uniform / Zipf multisets over
a seeded row permutation), noisy observed values and a held-out test split.
It is shared by the tests, the benchmark and the oracle legs; it implements no
step of the completion method.  Planted values are evaluated in double
precision from the planted factors (eq. 1) purely to synthesize data.

The workloads mirror the paper's experiments (Sec. IV): planted rank-R
factors with i.i.d. U[0, 1] entries and additive Gaussian noise, and
MovieLens- / Uber-shaped skew stand-ins; none of the paper's datasets is used.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

CHUNK = 1 << 21


@dataclasses.dataclass
class Problem:
    dims: List[int]
    rank: int
    lam: float
    c: float
    factors: List[np.ndarray]          # planted factors, float64 [I_i][R]
    idx_train: np.ndarray              # int32 [n_train][N], row-major COO
    val_train: np.ndarray              # float32 [n_train]
    idx_test: np.ndarray               # int32 [n_test][N]
    val_test: np.ndarray               # float32 [n_test] (noisy)
    val_test_clean: np.ndarray         # float64 [n_test] (planted model)
    sigma: float
    name: str = ""

    @property
    def order(self) -> int:
        return len(self.dims)

    @property
    def nnz(self) -> int:
        return int(self.val_train.shape[0])


def _zipf_cdf(n: int, s: float) -> np.ndarray:
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    return cdf / cdf[-1]


def _draw_mode(rng: np.random.Generator, n: int, dim: int, kind: str, s: float,
               perm: Optional[np.ndarray], cdf: Optional[np.ndarray]) -> np.ndarray:
    if kind == "uniform":
        return rng.integers(0, dim, size=n, dtype=np.int64).astype(np.int32)
    if kind == "zipf":
        import torch
        u = torch.from_numpy(rng.random(n))
        rank = torch.searchsorted(torch.from_numpy(cdf), u, right=True).numpy()
        np.minimum(rank, dim - 1, out=rank)
        return perm[rank].astype(np.int32)
    raise ValueError(kind)


def planted_values(factors: Sequence[np.ndarray], idx: np.ndarray) -> np.ndarray:
    """Planted CPD model values (eq. 1) at idx: float32 products of the
    (float32-representable) planted factors, summed over r in float64.
    Evaluated in chunks with torch's CPU threads, only to synthesize data."""
    import torch
    n = idx.shape[0]
    out = np.empty(n, dtype=np.float64)
    F = [torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)) for f in factors]
    step = 4 * CHUNK
    for s0 in range(0, n, step):
        s1 = min(n, s0 + step)
        it = torch.from_numpy(np.ascontiguousarray(idx[s0:s1]).astype(np.int64))
        prod = torch.index_select(F[0], 0, it[:, 0])
        for i in range(1, len(F)):
            prod.mul_(torch.index_select(F[i], 0, it[:, i]))
        out[s0:s1] = prod.sum(dim=1, dtype=torch.float64).numpy()
    return out


def make_problem(dims: Sequence[int], rank: int, nnz_total: int, *, lam: float = 1e-3,
                 c: float = 0.1, index_dist: Sequence[str] | str = "uniform",
                 zipf_s: Sequence[float] | float = 1.1, without_replacement: bool = False,
                 factor_dist: str = "uniform", factor_scale: float = 1.0,
                 sigma: float = 0.01, test_frac: float = 0.1, round_clamp: bool = False,
                 seed: int = 1, name: str = "") -> Problem:
    """Planted nonnegative rank-R tensor, observed on nnz_total cells.

    factor_dist: "uniform" -> U[0, factor_scale]; "gamma" -> Gamma(2, 0.5).
    index_dist: per mode "uniform" or "zipf" (rank r has weight r^-s over a
    seeded permutation of the rows).  without_replacement draws distinct cells
    uniformly (only for small tensors).  The last test_frac of the draws (which
    are exchangeable) form the test split.
    """
    dims = [int(d) for d in dims]
    N = len(dims)
    rng = np.random.default_rng(seed)
    if factor_dist == "uniform":
        factors = [rng.random((d, rank)) * factor_scale for d in dims]
    elif factor_dist == "gamma":
        factors = [rng.gamma(2.0, 0.5, size=(d, rank)) for d in dims]
    else:
        raise ValueError(factor_dist)
    factors = [f.astype(np.float32).astype(np.float64) for f in factors]
    kinds = [index_dist] * N if isinstance(index_dist, str) else list(index_dist)
    ss = [zipf_s] * N if isinstance(zipf_s, (int, float)) else list(zipf_s)
    perms = [rng.permutation(d) if k == "zipf" else None for d, k in zip(dims, kinds)]
    cdfs = [_zipf_cdf(d, s) if k == "zipf" else None for d, k, s in zip(dims, kinds, ss)]

    idx = np.empty((nnz_total, N), dtype=np.int32)
    if without_replacement:
        total = math.prod(dims)
        assert nnz_total <= total
        cells = rng.choice(total, size=nnz_total, replace=False)
        coords = np.unravel_index(cells, dims)
        for i in range(N):
            idx[:, i] = coords[i]
    else:
        for s0 in range(0, nnz_total, CHUNK):
            s1 = min(nnz_total, s0 + CHUNK)
            for i in range(N):
                idx[s0:s1, i] = _draw_mode(rng, s1 - s0, dims[i], kinds[i], ss[i], perms[i], cdfs[i])

    clean = planted_values(factors, idx)
    vals = np.empty(nnz_total, dtype=np.float32)
    for s0 in range(0, nnz_total, CHUNK):
        s1 = min(nnz_total, s0 + CHUNK)
        v = clean[s0:s1]
        if round_clamp:
            v = np.clip(np.rint(v), 1.0, 5.0)
        elif sigma > 0:
            v = v + sigma * rng.standard_normal(s1 - s0)
        vals[s0:s1] = v
    n_test = int(round(test_frac * nnz_total))
    n_train = nnz_total - n_test
    return Problem(dims=dims, rank=rank, lam=lam, c=c, factors=factors,
                   idx_train=idx[:n_train], val_train=vals[:n_train],
                   idx_test=np.ascontiguousarray(idx[n_train:]), val_test=vals[n_train:],
                   val_test_clean=clean[n_train:], sigma=sigma, name=name)


# ---- the workloads -----------------------------------------------------------

def planted_rank10_100cube(seed: int = 1) -> Problem:
    """100x100x100, R = 10, U[0,1] factors, 50,000 distinct cells, sigma = 0.01,
    10% test, lambda = 1e-3, c = 0.1 (the small parity workload)."""
    return make_problem([100, 100, 100], 10, 50_000, lam=1e-3, c=0.1,
                        without_replacement=True, sigma=0.01, test_frac=0.1,
                        seed=seed, name="planted-100^3-R10-50k")


def zipf_1e4cube(nnz_total: int = 100_000_000, dim: int = 10_000, rank: int = 32,
                 seed: int = 1) -> Problem:
    """10^4 x 10^4 x 10^4, R = 32, Zipf(1.1) indices over permuted rows,
    U[0,1] factors, sigma = 0.01, 2% test."""
    return make_problem([dim] * 3, rank, nnz_total, lam=1e-3, c=0.1, index_dist="zipf",
                        zipf_s=1.1, sigma=0.01, test_frac=0.02, seed=seed,
                        name=f"zipf1.1-{dim}^3-R{rank}-{nnz_total}")


def uniform_4way(nnz_total: int = 200_000_000, dims=(100_000, 50_000, 20_000, 1_000),
                 rank: int = 16, seed: int = 1) -> Problem:
    """4-way 1e5 x 5e4 x 2e4 x 1e3, R = 16, uniform indices, Gamma(2, 0.5)
    factors, sigma = 0.05, 2% test."""
    return make_problem(list(dims), rank, nnz_total, lam=1e-3, c=0.1, index_dist="uniform",
                        factor_dist="gamma", sigma=0.05, test_frac=0.02, seed=seed,
                        name=f"uniform-4way-R{rank}-{nnz_total}")


def rating_3way(nnz_total: int = 500_000_000, dims=(1_000_000, 500_000, 200), rank: int = 64,
                seed: int = 1) -> Problem:
    """User x item x time 1e6 x 5e5 x 200, R = 64, Zipf(1.2) users and items,
    uniform time, planted U[0, 2a] with a = (3/64)^(1/3), values rounded and
    clamped to 1..5, 1% test."""
    a = (3.0 / rank) ** (1.0 / 3.0)
    return make_problem(list(dims), rank, nnz_total, lam=1e-3, c=0.1,
                        index_dist=["zipf", "zipf", "uniform"], zipf_s=[1.2, 1.2, 1.0],
                        factor_dist="uniform", factor_scale=2 * a, sigma=0.0,
                        round_clamp=True, test_frac=0.01, seed=seed,
                        name=f"rating-3way-R{rank}-{nnz_total}")


def random_factors(dims: Sequence[int], rank: int, scale: float, seed: int) -> List[np.ndarray]:
    """Seeded nonnegative starting factors, rounded to float32 values so that a
    float32 and a float64 implementation start from identical numbers."""
    rng = np.random.default_rng(seed)
    return [(rng.random((d, rank)) * scale).astype(np.float32).astype(np.float64) for d in dims]


# ---- the serving stream ------------------------------------------------------

@dataclasses.dataclass
class JobSpec:
    """One job of a serving stream; its data come from make_problem(seed=data_seed)."""
    arrival: float
    dims: List[int]
    rank: int
    nnz: int
    storage_bf16: int
    data_seed: int


def serving_stream(n_jobs: int = 256, rate: float = 4.0, dim_range=(1_000, 200_000),
                   nnz_range=(1_000_000, 50_000_000), ranks=(8, 16, 32, 64), orders=(3, 4),
                   seed: int = 5) -> List[JobSpec]:
    """Poisson arrivals (mean `rate` jobs/s) of completion jobs: order drawn
    from `orders`, each mode size log-uniform in dim_range, rank from `ranks`,
    observation count log-uniform in nnz_range, FP32 and BF16 storage
    alternating (half each)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for j in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(orders))
        lo, hi = math.log(dim_range[0]), math.log(dim_range[1])
        dims = [int(round(math.exp(rng.uniform(lo, hi)))) for _ in range(N)]
        rank = int(rng.choice(ranks))
        nnz = int(round(math.exp(rng.uniform(math.log(nnz_range[0]), math.log(nnz_range[1])))))
        out.append(JobSpec(arrival=t, dims=dims, rank=rank, nnz=nnz, storage_bf16=j % 2,
                           data_seed=seed * 1_000_003 + j))
    return out


def serving_job(spec: JobSpec, sigma: float = 0.01, test_frac: float = 0.01) -> Problem:
    """Planted U[0,1] factors of the spec's rank, uniform observed indices,
    Gaussian noise sigma, lambda = 1e-3, c = 0.1."""
    return make_problem(spec.dims, spec.rank, spec.nnz, lam=1e-3, c=0.1, index_dist="uniform",
                        sigma=sigma, test_frac=test_frac, seed=spec.data_seed,
                        name=f"job-{len(spec.dims)}way-R{spec.rank}-{spec.nnz}")


def serving_job_device(spec: JobSpec, sigma: float = 0.01, test_frac: float = 0.01, device: str = "cuda",
                       chunk: int = 1 << 22) -> Problem:
    """The job of serving_job's recipe (planted U[0,1] factors of the spec's
    rank, uniform indices, Gaussian noise sigma, lambda = 1e-3, c = 0.1) drawn
    with torch's generator on `device`, for streams whose jobs are too large to
    draw on the host in time: seeded by the spec (the same job on the same
    device and torch version), not the same draws as serving_job.  Planted
    values are float32 products summed in float64, as in planted_values.  The
    arrays are returned on the host; the planted factors are not kept."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(spec.data_seed))
    dims, R, n = [int(d) for d in spec.dims], int(spec.rank), int(spec.nnz)
    F = [torch.rand(d, R, generator=g, device=device, dtype=torch.float32) for d in dims]
    idx = torch.empty(n, len(dims), dtype=torch.int32, device=device)
    for i, d in enumerate(dims):
        idx[:, i] = torch.randint(0, d, (n,), generator=g, device=device, dtype=torch.int32)
    vals = torch.empty(n, dtype=torch.float32, device=device)
    clean = torch.empty(n, dtype=torch.float64, device=device)
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        ix = idx[s0:s1].long()
        prod = F[0].index_select(0, ix[:, 0])
        for i in range(1, len(dims)):
            prod.mul_(F[i].index_select(0, ix[:, i]))
        c = prod.sum(dim=1, dtype=torch.float64)
        clean[s0:s1] = c
        noise = torch.randn(s1 - s0, generator=g, device=device, dtype=torch.float64)
        vals[s0:s1] = (c + sigma * noise).to(torch.float32)
    n_test = int(round(test_frac * n))
    n_train = n - n_test
    idx_h, vals_h, clean_h = idx.cpu().numpy(), vals.cpu().numpy(), clean.cpu().numpy()
    return Problem(dims=dims, rank=R, lam=1e-3, c=0.1, factors=[], idx_train=idx_h[:n_train],
                   val_train=vals_h[:n_train], idx_test=np.ascontiguousarray(idx_h[n_train:]),
                   val_test=vals_h[n_train:], val_test_clean=clean_h[n_train:], sigma=sigma,
                   name=f"job-{len(dims)}way-R{R}-{n}-device")


def uber_twin(seed: int = 1) -> Problem:
    """Uber-Pickups-shaped timing twin (Sec. IV-C): 183 x 24 x 1140 x 1717,
    3,309,490 uniform draws of a planted rank-10 tensor with U[0,1] factors,
    noiseless, c = 0.5, 2% held out.  The fitted rank is the caller's."""
    return make_problem([183, 24, 1140, 1717], 10, 3_309_490, lam=1e-3, c=0.5, index_dist="uniform",
                        sigma=0.0, test_frac=0.02, seed=seed, name="uber-twin-4way-planted-R10")
