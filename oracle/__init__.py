"""FP64 CPU oracle for AO accelerated stochastic nonnegative tensor completion.

TEST INFRASTRUCTURE ONLY.  The C source (``ntc_oracle.c``) restates the
paper's equations and Algorithms 1-2 in plain double precision.  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and imports nothing from it.

Functions whose result cannot be pinned to anything but the oracle itself
are marked "parity unpinned" in their docstrings (none at present).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntc_oracle.c")
_LIBS = {False: os.path.join(_HERE, "libntc_oracle.so"),
         True: os.path.join(_HERE, "libntc_oracle_omp.so")}
_lock = threading.Lock()
_loaded: dict = {}


def build(force: bool = False) -> None:
    """Compile the oracle twice: single-threaded and with OpenMP (Alg. 3)."""
    for omp, out in _LIBS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ntc_oracle.h"))):
            continue
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", out + ".tmp", "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.check_call(cmd)
        os.replace(out + ".tmp", out)


def _lib(omp: bool = False):
    with _lock:
        if omp in _loaded:
            return _loaded[omp]
        build()
        L = ctypes.CDLL(_LIBS[omp])
        P = ctypes.c_void_p
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        L.orc_sample_key.restype = ctypes.c_uint32
        L.orc_sample_key.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_int64]
        L.orc_sample_count.restype = ctypes.c_int64
        L.orc_sample_count.argtypes = [ctypes.c_double, ctypes.c_int64]
        L.orc_sample_row.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, i64p]
        L.orc_bucket.argtypes = [ctypes.c_int, ctypes.c_int64, P, ctypes.c_int,
                                 ctypes.c_int64, P, P]
        L.orc_power_lmax.restype = ctypes.c_double
        L.orc_power_lmax.argtypes = [ctypes.c_int, P, ctypes.c_int]
        L.orc_perm_index.restype = ctypes.c_int64
        L.orc_perm_index.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_int64, ctypes.c_int64]
        L.orc_power_lmax_v.restype = ctypes.c_double
        L.orc_power_lmax_v.argtypes = [ctypes.c_int, P, ctypes.c_int, P]
        L.orc_jacobi_lmax.restype = ctypes.c_double
        L.orc_jacobi_lmax.argtypes = [ctypes.c_int, P]
        L.orc_row_update.restype = ctypes.c_int64
        L.orc_row_update.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, P, ctypes.c_int64, P, P,
                                     ctypes.c_int64, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_uint64, ctypes.c_int, P, P, P, P, P, P, P, P, P]
        L.orc_create.restype = P
        L.orc_create.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_double]
        L.orc_destroy.argtypes = [P]
        L.orc_set_param.argtypes = [P, ctypes.c_char_p, ctypes.c_double]
        L.orc_set_observed.argtypes = [P, ctypes.c_int64, P, P]
        L.orc_set_factor.argtypes = [P, ctypes.c_int, P]
        L.orc_get_factor.argtypes = [P, ctypes.c_int, P]
        L.orc_init_factors.argtypes = [P, ctypes.c_uint64]
        L.orc_get_ao_iter.restype = ctypes.c_uint64
        L.orc_get_ao_iter.argtypes = [P]
        L.orc_set_ao_iter.argtypes = [P, ctypes.c_uint64]
        L.orc_snmc.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_uint64]
        L.orc_epoch.argtypes = [P, P, ctypes.c_double, ctypes.c_uint64]
        L.orc_predict.argtypes = [P, ctypes.c_int64, P, P]
        L.orc_rmse.restype = ctypes.c_double
        L.orc_rmse.argtypes = [P, ctypes.c_int64, P, P]
        L.orc_cost.restype = ctypes.c_double
        L.orc_cost.argtypes = [P]
        L.orc_debug_row.argtypes = [P, ctypes.c_int64, P, P, P, P, P, P]
        L.orc_get_bucket.argtypes = [P, ctypes.c_int, P, P]
        L.orc_rows_skipped.restype = ctypes.c_int64
        L.orc_rows_skipped.argtypes = [P]
        L.orc_visits.restype = ctypes.c_int64
        L.orc_visits.argtypes = [P]
        _loaded[omp] = L
        return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11, Sec. 4.2)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    _lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def sample_key(seed: int, mode: int, ao_iter: int, inner: int, q: int) -> int:
    """Sample key of bucket position q (Sec. II-B sampling reading): word
    q mod 4 of the Philox4x32-10 block with counter {mode, ao_iter, inner, q // 4}."""
    return int(_lib().orc_sample_key(seed, mode, ao_iter, inner, q))


def sample_count(c: float, n: int) -> int:
    """B_{l,p} = floor(c * n_p) (Sec. II-B)."""
    return int(_lib().orc_sample_count(c, n))


def sample_row(seed, mode, ao_iter, inner, q0, n, k) -> np.ndarray:
    """Absolute bucket positions of the row's sample, in (key, position) order."""
    out = np.zeros(max(k, 1), dtype=np.int64)
    rc = _lib().orc_sample_row(seed, mode, ao_iter, inner, q0, n, k,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise ValueError("bad sample arguments")
    return out[:k]


def bucket(idx: np.ndarray, mode: int, dim: int):
    """Stable counting sort by the mode index (rows of X_(i), Sec. II)."""
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    nnz, order = idx.shape
    row_ptr = np.zeros(dim + 1, dtype=np.int64)
    perm = np.zeros(max(nnz, 1), dtype=np.int64)
    if _lib().orc_bucket(order, nnz, _ptr(idx), mode, dim, _ptr(row_ptr), _ptr(perm)) != 0:
        raise IndexError("index out of range")
    return row_ptr, perm[:nnz]


def power_lmax(H: np.ndarray, iters: int = 10) -> float:
    """Power-method estimate of max eig(H) (Alg. 1 line 10, Sec. II-B item 4)."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    return float(_lib().orc_power_lmax(H.shape[0], _ptr(H), iters))


def perm_index(seed: int, mode: int, epoch: int, row: int, n: int, i: int) -> int:
    """Epoch-permutation sampling: image of i under row `row`'s permutation of
    [0, n) in epoch `epoch`."""
    return int(_lib().orc_perm_index(seed, mode, epoch, row, n, i))


def power_lmax_v(H: np.ndarray, iters: int, v: np.ndarray = None):
    """Power method from start vector v (None: ones/sqrt(R)); returns
    (estimate, last normalised iterate)."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    R = H.shape[0]
    vv = np.full(R, 1.0 / np.sqrt(R)) if v is None else np.array(v, dtype=np.float64)
    mu = float(_lib().orc_power_lmax_v(R, _ptr(H), iters, _ptr(vv)))
    return mu, vv


def jacobi_lmax(H: np.ndarray) -> float:
    """Exact max eig(H) by cyclic Jacobi rotations."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    return float(_lib().orc_jacobi_lmax(H.shape[0], _ptr(H)))


def row_update(mode: int, lam: float, factors, idx: np.ndarray, vals: np.ndarray, q0: int,
               c: float, seed: int, ao_iter: int, inner: int, y: np.ndarray, a: np.ndarray,
               power_iters: int = 10, lp_exact: bool = False) -> dict:
    """Alg. 1 lines 5-13 for one row given its observations in bucket order."""
    L = _lib()
    fac = [np.ascontiguousarray(f, dtype=np.float64) for f in factors]
    order, R = len(fac), fac[0].shape[1]
    arr = (ctypes.c_void_p * order)(*[f.ctypes.data for f in fac])
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    a_out, y_out, H, g = np.zeros(R), np.zeros(R), np.zeros((R, R)), np.zeros(R)
    Lp, Lx, beta = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    k = L.orc_row_update(order, mode, R, lam, power_iters, int(lp_exact), ctypes.cast(arr, ctypes.c_void_p),
                         vals.shape[0], _ptr(idx), _ptr(vals), q0, c, seed, ao_iter, inner, _ptr(y),
                         _ptr(a), _ptr(a_out), _ptr(y_out), _ptr(H), _ptr(g), ctypes.byref(Lp),
                         ctypes.byref(Lx), ctypes.byref(beta))
    return dict(k=int(k), a=a_out, y=y_out, H=H, grad=g, L=Lp.value, L_exact=Lx.value, beta=beta.value)


class Oracle:
    """Whole-problem oracle: Algorithm 2 around Algorithm 1, FP64."""

    def __init__(self, dims, rank: int, lam: float, omp: bool = False):
        self.L = _lib(omp)
        self.dims = [int(d) for d in dims]
        self.order = len(self.dims)
        self.rank = int(rank)
        d = np.array(self.dims, dtype=np.int64)
        self.h = self.L.orc_create(self.order, _ptr(d), self.rank, float(lam))
        if not self.h:
            raise ValueError("bad problem arguments")
        self.nnz = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    def set_param(self, key: str, value: float) -> None:
        if self.L.orc_set_param(self.h, key.encode(), float(value)) != 0:
            raise ValueError(f"bad parameter {key}={value}")

    def set_observed(self, idx: np.ndarray, vals: np.ndarray) -> None:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        assert idx.shape == (vals.shape[0], self.order)
        if self.L.orc_set_observed(self.h, vals.shape[0], _ptr(idx), _ptr(vals)) != 0:
            raise IndexError("index out of range")
        self.nnz = vals.shape[0]

    def set_factor(self, mode: int, U: np.ndarray) -> None:
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (self.dims[mode], self.rank)
        if self.L.orc_set_factor(self.h, mode, _ptr(U)) != 0:
            raise ValueError("factor must be >= 0")

    def get_factor(self, mode: int) -> np.ndarray:
        U = np.zeros((self.dims[mode], self.rank), dtype=np.float64)
        self.L.orc_get_factor(self.h, mode, _ptr(U))
        return U

    def factors(self):
        return [self.get_factor(i) for i in range(self.order)]

    def init_factors(self, init_seed: int) -> None:
        self.L.orc_init_factors(self.h, init_seed)

    @property
    def ao_iter(self) -> int:
        return int(self.L.orc_get_ao_iter(self.h))

    @ao_iter.setter
    def ao_iter(self, k: int) -> None:
        self.L.orc_set_ao_iter(self.h, k)

    def snmc(self, mode: int, c: float, seed: int) -> None:
        if self.L.orc_snmc(self.h, mode, float(c), seed) != 0:
            raise ValueError("snmc failed")

    def epoch(self, c: float, seed: int, mode_order=None) -> None:
        mo = None
        if mode_order is not None:
            mo_arr = np.ascontiguousarray(mode_order, dtype=np.int32)
            mo = _ptr(mo_arr)
        if self.L.orc_epoch(self.h, mo, float(c), seed) != 0:
            raise ValueError("epoch failed")

    def predict(self, idx: np.ndarray) -> np.ndarray:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        out = np.zeros(idx.shape[0], dtype=np.float64)
        if self.L.orc_predict(self.h, idx.shape[0], _ptr(idx), _ptr(out)) != 0:
            raise IndexError("index out of range")
        return out

    def rmse(self, idx: np.ndarray, vals: np.ndarray) -> float:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        return float(self.L.orc_rmse(self.h, idx.shape[0], _ptr(idx), _ptr(vals)))

    def cost(self) -> float:
        return float(self.L.orc_cost(self.h))

    def debug_row(self, row: int):
        R = self.rank
        H = np.zeros((R, R))
        g = np.zeros(R)
        L = ctypes.c_double()
        Lx = ctypes.c_double()
        b = ctypes.c_double()
        kp = ctypes.c_int64()
        if self.L.orc_debug_row(self.h, row, _ptr(H), _ptr(g), ctypes.byref(L),
                                ctypes.byref(Lx), ctypes.byref(b), ctypes.byref(kp)) != 0:
            raise ValueError("no debug data (set_param('debug', 1) before snmc)")
        return dict(H=H, grad=g, L=L.value, L_exact=Lx.value, beta=b.value, kp=kp.value)

    def get_bucket(self, mode: int):
        rp = np.zeros(self.dims[mode] + 1, dtype=np.int64)
        pm = np.zeros(max(self.nnz, 1), dtype=np.int64)
        if self.L.orc_get_bucket(self.h, mode, _ptr(rp), _ptr(pm)) != 0:
            raise ValueError("no bucket")
        return rp, pm[:self.nnz]

    @property
    def rows_skipped(self) -> int:
        return int(self.L.orc_rows_skipped(self.h))

    @property
    def visits(self) -> int:
        return int(self.L.orc_visits(self.h))
