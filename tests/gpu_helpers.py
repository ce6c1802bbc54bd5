"""Helpers shared by the GPU tests: build/load the library, run the oracle on
the same seeded inputs, and compare."""
import numpy as np
import pytest

import oracle
from paper_2109_09534_gb300 import build as nbuild
from paper_2109_09534_gb300 import ntc, synth


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbuild.build()
    ntc.load()
    return torch


def gpu_problem(p, torch, **params):
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=torch.cuda.current_stream().cuda_stream, **params)
    return g


def pair(p, torch, factors=None, gparams=None, oparams=None, omp=False):
    """A GPU handle and an oracle on the same observations and starting factors."""
    g = gpu_problem(p, torch, **(gparams or {}))
    o = oracle.Oracle(p.dims, p.rank, p.lam, omp=omp)
    for k, v in (oparams or {}).items():
        o.set_param(k, v)
    g.set_observed(p.idx_train, p.val_train)
    o.set_observed(p.idx_train, p.val_train.astype(np.float64))
    if factors is None:
        factors = synth.random_factors(p.dims, p.rank, 0.7, seed=101)
    for i, u in enumerate(factors):
        g.set_factor(i, u.astype(np.float32))
        o.set_factor(i, u)
    return g, o


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def max_row_err(a, b, floor_frac=1e-3):
    """Largest per-row relative error max_r ||a_r - b_r|| / ||b_r|| over the
    factor's rows, every row included (light and split alike).  A row whose
    oracle norm is below floor_frac of the factor's RMS row norm (a row the
    projection drove to or near zero) is measured against that floor instead,
    so that the bound stays relative to the factor's scale."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b, axis=1)
    rms = np.sqrt(np.mean(nb ** 2)) if nb.size else 0.0
    den = np.maximum(nb, floor_frac * rms if rms > 0 else 1.0)
    return float(np.max(np.linalg.norm(a - b, axis=1) / den)) if nb.size else 0.0


def assert_factor_close(a, b, frob, row, what=""):
    """Per-factor Frobenius bound and per-row bound (element-wise parity)."""
    fe, re_ = rel_err(a, b), max_row_err(a, b)
    assert fe <= frob, f"{what}: Frobenius relative error {fe:.3e} > {frob:g}"
    assert re_ <= row, f"{what}: largest row relative error {re_:.3e} > {row:g}"


def oracle_mask(idx, mode, dim, c, seed, ao_iter, inner):
    """Sample of every row of `mode` by the oracle, as a mask over bucket positions."""
    row_ptr, _ = oracle.bucket(idx, mode, dim)
    mask = np.zeros(idx.shape[0], dtype=np.uint8)
    for r in range(dim):
        n = int(row_ptr[r + 1] - row_ptr[r])
        k = oracle.sample_count(c, n)
        if k:
            mask[oracle.sample_row(seed, mode, ao_iter, inner, int(row_ptr[r]), n, k)] = 1
    return mask


def small_zipf(nnz=200_000, dim=2_000, rank=32, seed=3):
    return synth.make_problem([dim] * 3, rank, nnz, lam=1e-3, c=0.1, index_dist="zipf", zipf_s=1.1,
                              sigma=0.01, test_frac=0.02, seed=seed, name="small-zipf")
