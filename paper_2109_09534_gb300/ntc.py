"""Thin ctypes binding of the C ABI in ``include/ntc.h`` and ``include/ntc_serve.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``libntc.so``.  The functions keep the C names; :class:`NTC` wraps a handle
for convenience.  Host arrays are numpy arrays; ``*_dev`` calls take device
pointers (for example ``torch.Tensor.data_ptr()``).  There is no fallback: if
the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import glob
import os
import re
from typing import Optional, Sequence

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "ntc.h")
HEADERS = sorted(glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h")))

NTC_OK, NTC_ERR_ARG, NTC_ERR_INDEX, NTC_ERR_OOM, NTC_ERR_STATE, NTC_ERR_CUDA = range(6)
KERNELS = ["light", "heavy_sample", "heavy_resolve", "heavy_gram", "finish"]
_STATUS = {0: "NTC_OK", 1: "NTC_ERR_ARG", 2: "NTC_ERR_INDEX", 3: "NTC_ERR_OOM", 4: "NTC_ERR_STATE",
           5: "NTC_ERR_CUDA"}


class NTCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class ntc_stats(ctypes.Structure):
    _fields_ = [("visits", ctypes.c_int64), ("visits_heavy", ctypes.c_int64),
                ("rows_updated", ctypes.c_int64), ("rows_skipped", ctypes.c_int64),
                ("fallback_rows", ctypes.c_int64), ("alg_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("wait_timeouts", ctypes.c_int64)]


class ntc_job_desc(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("dims", ctypes.c_int64 * 8), ("rank", ctypes.c_int),
                ("lam", ctypes.c_double), ("c", ctypes.c_double), ("storage_bf16", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("init_seed", ctypes.c_uint64), ("nnz", ctypes.c_int64),
                ("idx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("n_test", ctypes.c_int64),
                ("test_idx", ctypes.c_void_p), ("test_vals", ctypes.c_void_p),
                ("target_rmse", ctypes.c_double), ("max_epochs", ctypes.c_int), ("arrival", ctypes.c_double)]


class ntc_job_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("reached", ctypes.c_int), ("epochs", ctypes.c_int),
                ("rmse", ctypes.c_double), ("rmse0", ctypes.c_double), ("t_arrival", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("bytes", ctypes.c_int64)]


class ntc_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ["submitted", "queued", "running", "done", "failed", "bytes_in_use", "peak_bytes", "peak_running",
                 "epochs", "entries", "predict_calls", "predict_queries", "predict_launches"]]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = range(4)

_lib = None


def declared_functions() -> list:
    """Names of the functions declared in include/*.h."""
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(ntc_[a-z_]+)\s*\(", src))
    return sorted(names)


def load(path: Optional[str] = None):
    """Load libntc.so (built in-tree by build.py).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    P, i64, u64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
    sig = {
        "ntc_create": [i32, P, i32, dbl, ctypes.POINTER(P)],
        "ntc_set_param": [P, ctypes.c_char_p, dbl],
        "ntc_set_stream": [P, P],
        "ntc_set_observed": [P, i64, P, P],
        "ntc_set_observed_dev": [P, i64, P, P],
        "ntc_epoch": [P, P, dbl, u64],
        "ntc_snmc": [P, i32, dbl, u64],
        "ntc_predict": [P, i64, P, P],
        "ntc_predict_dev": [P, i64, P, P],
        "ntc_rmse": [P, i64, P, P, ctypes.POINTER(dbl)],
        "ntc_cost": [P, ctypes.POINTER(dbl)],
        "ntc_get_factor": [P, i32, P],
        "ntc_set_factor": [P, i32, P],
        "ntc_get_state": [P, ctypes.POINTER(u64)],
        "ntc_set_state": [P, u64],
        "ntc_sync": [P],
        "ntc_get_stats": [P, ctypes.POINTER(ntc_stats)],
        "ntc_get_bucket": [P, i32, P, P],
        "ntc_sample_mask": [P, i32, dbl, u64, u64, i32, P],
        "ntc_get_profile": [P, i32, ctypes.POINTER(dbl), ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "ntc_measure_fp32_peak": [P, ctypes.POINTER(dbl)],
        "ntc_job_bytes": [ctypes.POINTER(ntc_job_desc), ctypes.POINTER(i64)],
        "ntc_server_create": [dbl, i32, ctypes.POINTER(P)],
        "ntc_server_submit": [P, ctypes.POINTER(ntc_job_desc), ctypes.POINTER(i64)],
        "ntc_server_set_param": [P, ctypes.c_char_p, dbl],
        "ntc_server_step": [P, ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "ntc_server_sync": [P],
        "ntc_server_job_info": [P, i64, ctypes.POINTER(ntc_job_info)],
        "ntc_server_predict": [P, i64, P, P, P],
        "ntc_server_get_factor": [P, i64, i32, P],
        "ntc_server_stats_get": [P, ctypes.POINTER(ntc_server_stats)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.ntc_last_error.argtypes = [P]
    L.ntc_last_error.restype = ctypes.c_char_p
    L.ntc_destroy.argtypes = [P]
    L.ntc_destroy.restype = None
    L.ntc_server_now.argtypes = [P]
    L.ntc_server_now.restype = dbl
    L.ntc_server_last_error.argtypes = [P]
    L.ntc_server_last_error.restype = ctypes.c_char_p
    L.ntc_server_destroy.argtypes = [P]
    L.ntc_server_destroy.restype = None
    _lib = L
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(h, status: int) -> None:
    if status != NTC_OK:
        msg = load().ntc_last_error(h) if h else b""
        raise NTCError(status, (msg or b"").decode())


def measure_fp32_peak(stream: int = 0) -> float:
    """FP32 FMA throughput of the current device, TFLOP/s."""
    out = ctypes.c_double()
    _check(None, load().ntc_measure_fp32_peak(ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


class NTC:
    """One completion problem on the current CUDA device (a C handle)."""

    def __init__(self, dims: Sequence[int], rank: int, lam: float, stream: Optional[int] = None,
                 **params):
        L = load()
        self.dims = [int(d) for d in dims]
        self.order = len(self.dims)
        self.rank = int(rank)
        d = np.ascontiguousarray(self.dims, dtype=np.int64)
        h = ctypes.c_void_p()
        st = L.ntc_create(self.order, _ptr(d), self.rank, float(lam), ctypes.byref(h))
        if st != NTC_OK:
            raise NTCError(st, "ntc_create failed")
        self.h = h
        self.L = L
        if stream is not None:
            _check(self.h, L.ntc_set_stream(self.h, ctypes.c_void_p(stream)))
        for k, v in params.items():
            self.set_param(k, v)

    def close(self) -> None:
        if getattr(self, "h", None):
            self.L.ntc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_param(self, key: str, value: float) -> None:
        _check(self.h, self.L.ntc_set_param(self.h, key.encode(), float(value)))

    def set_stream(self, stream: int) -> None:
        _check(self.h, self.L.ntc_set_stream(self.h, ctypes.c_void_p(stream)))

    def set_observed(self, idx: np.ndarray, vals: np.ndarray) -> None:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        if idx.shape != (vals.shape[0], self.order):
            raise ValueError("idx must be [nnz][order] and vals [nnz]")
        _check(self.h, self.L.ntc_set_observed(self.h, vals.shape[0], _ptr(idx), _ptr(vals)))

    def set_observed_ptr(self, nnz: int, idx_ptr: int, vals_ptr: int, device: bool) -> None:
        f = self.L.ntc_set_observed_dev if device else self.L.ntc_set_observed
        _check(self.h, f(self.h, int(nnz), ctypes.c_void_p(idx_ptr), ctypes.c_void_p(vals_ptr)))

    def epoch(self, c: float, seed: int, mode_order: Optional[Sequence[int]] = None) -> None:
        mo = None
        if mode_order is not None:
            self._mo = np.ascontiguousarray(mode_order, dtype=np.int32)
            mo = _ptr(self._mo)
        _check(self.h, self.L.ntc_epoch(self.h, mo, float(c), int(seed)))

    def snmc(self, mode: int, c: float, seed: int) -> None:
        _check(self.h, self.L.ntc_snmc(self.h, int(mode), float(c), int(seed)))

    def predict(self, idx: np.ndarray) -> np.ndarray:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        out = np.zeros(idx.shape[0], dtype=np.float32)
        _check(self.h, self.L.ntc_predict(self.h, idx.shape[0], _ptr(idx), _ptr(out)))
        return out

    def predict_dev(self, n: int, idx_ptr: int, out_ptr: int) -> None:
        _check(self.h, self.L.ntc_predict_dev(self.h, int(n), ctypes.c_void_p(idx_ptr),
                                              ctypes.c_void_p(out_ptr)))

    def rmse(self, idx: np.ndarray, vals: np.ndarray) -> float:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        out = ctypes.c_double()
        _check(self.h, self.L.ntc_rmse(self.h, idx.shape[0], _ptr(idx), _ptr(vals), ctypes.byref(out)))
        return out.value

    def cost(self) -> float:
        out = ctypes.c_double()
        _check(self.h, self.L.ntc_cost(self.h, ctypes.byref(out)))
        return out.value

    def get_factor(self, mode: int) -> np.ndarray:
        out = np.zeros((self.dims[mode], self.rank), dtype=np.float32)
        _check(self.h, self.L.ntc_get_factor(self.h, int(mode), _ptr(out)))
        return out

    def set_factor(self, mode: int, U: np.ndarray) -> None:
        U = np.ascontiguousarray(U, dtype=np.float32)
        if U.shape != (self.dims[mode], self.rank):
            raise ValueError("factor shape")
        _check(self.h, self.L.ntc_set_factor(self.h, int(mode), _ptr(U)))

    def factors(self):
        return [self.get_factor(i) for i in range(self.order)]

    @property
    def ao_iter(self) -> int:
        v = ctypes.c_uint64()
        _check(self.h, self.L.ntc_get_state(self.h, ctypes.byref(v)))
        return int(v.value)

    @ao_iter.setter
    def ao_iter(self, k: int) -> None:
        _check(self.h, self.L.ntc_set_state(self.h, int(k)))

    def sync(self) -> None:
        _check(self.h, self.L.ntc_sync(self.h))

    def stats(self) -> dict:
        s = ntc_stats()
        _check(self.h, self.L.ntc_get_stats(self.h, ctypes.byref(s)))
        return {k: int(getattr(s, k)) for k, _ in ntc_stats._fields_}

    def profile(self) -> dict:
        """Per kernel class: summed event ms, launches, algorithmic bytes (then cleared)."""
        out = {}
        for kind, name in enumerate(KERNELS):
            ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
            _check(self.h, self.L.ntc_get_profile(self.h, kind, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)))
            out[name] = dict(ms=ms.value, launches=int(n.value), alg_bytes=int(b.value))
        return out

    def get_bucket(self, mode: int, perm: bool = False):
        rp = np.zeros(self.dims[mode] + 1, dtype=np.int64)
        pm = None
        if perm:
            pm = np.zeros(max(self._nnz_hint(rp, mode), 1), dtype=np.int64)
        _check(self.h, self.L.ntc_get_bucket(self.h, int(mode), _ptr(rp), _ptr(pm) if pm is not None else None))
        if pm is not None:
            pm = pm[:rp[-1]]
        return rp, pm

    def _nnz_hint(self, rp, mode):
        _check(self.h, self.L.ntc_get_bucket(self.h, int(mode), _ptr(rp), None))
        return int(rp[-1])

    def sample_mask(self, mode: int, c: float, seed: int, ao_iter: int, inner: int, nnz: int) -> np.ndarray:
        m = np.zeros(max(nnz, 1), dtype=np.uint8)
        _check(self.h, self.L.ntc_sample_mask(self.h, int(mode), float(c), int(seed), int(ao_iter),
                                              int(inner), _ptr(m)))
        return m[:nnz]


# ---------------------------------------------------------------------------
# Completion server (include/ntc_serve.h)

def job_desc(dims, rank, lam, c, idx, vals, test_idx, test_vals, target_rmse, max_epochs, arrival=0.0,
             seed=1, init_seed=3, storage_bf16=0) -> ntc_job_desc:
    """An ntc_job_desc over numpy arrays (the caller keeps them alive)."""
    d = ntc_job_desc()
    d.order = len(dims)
    for i, n in enumerate(dims):
        d.dims[i] = int(n)
    d.rank, d.lam, d.c, d.storage_bf16 = int(rank), float(lam), float(c), int(storage_bf16)
    d.seed, d.init_seed = int(seed), int(init_seed)
    d.nnz, d.idx, d.vals = len(vals), idx.ctypes.data, vals.ctypes.data
    d.n_test, d.test_idx, d.test_vals = len(test_vals), test_idx.ctypes.data, test_vals.ctypes.data
    d.target_rmse, d.max_epochs, d.arrival = float(target_rmse), int(max_epochs), float(arrival)
    return d


def job_bytes(d: ntc_job_desc) -> int:
    out = ctypes.c_int64()
    _check(None, load().ntc_job_bytes(ctypes.byref(d), ctypes.byref(out)))
    return out.value


class Server:
    """Continuous-batching completion server on the current CUDA device."""

    def __init__(self, hbm_budget: float, max_running: int = 64):
        L = load()
        self._s = ctypes.c_void_p()
        st = L.ntc_server_create(float(hbm_budget), int(max_running), ctypes.byref(self._s))
        if st != NTC_OK:
            raise NTCError(st, "ntc_server_create failed")
        self._keep = {}

    def _check(self, status: int) -> None:
        if status != NTC_OK:
            raise NTCError(status, (load().ntc_server_last_error(self._s) or b"").decode())

    def close(self) -> None:
        if self._s:
            load().ntc_server_destroy(self._s)
            self._s = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        self.close()

    def set_param(self, key: str, value: float) -> None:
        self._check(load().ntc_server_set_param(self._s, key.encode(), float(value)))

    def submit(self, dims, rank, lam, c, idx, vals, test_idx, test_vals, target_rmse, max_epochs,
               arrival=0.0, seed=1, init_seed=3, storage_bf16=0) -> int:
        arrays = [np.ascontiguousarray(idx, dtype=np.int32), np.ascontiguousarray(vals, dtype=np.float32),
                  np.ascontiguousarray(test_idx, dtype=np.int32), np.ascontiguousarray(test_vals, dtype=np.float32)]
        d = job_desc(dims, rank, lam, c, *arrays, target_rmse, max_epochs, arrival, seed, init_seed, storage_bf16)
        jid = ctypes.c_int64()
        self._check(load().ntc_server_submit(self._s, ctypes.byref(d), ctypes.byref(jid)))
        self._keep[jid.value] = arrays   # read at admission
        return jid.value

    def step(self):
        r, q = ctypes.c_int64(), ctypes.c_int64()
        self._check(load().ntc_server_step(self._s, ctypes.byref(r), ctypes.byref(q)))
        for jid in [j for j in self._keep if self.job_info(j)["state"] != JOB_QUEUED]:
            del self._keep[jid]
        return r.value, q.value

    def sync(self) -> None:
        self._check(load().ntc_server_sync(self._s))

    def now(self) -> float:
        return load().ntc_server_now(self._s)

    def job_info(self, jid: int) -> dict:
        out = ntc_job_info()
        self._check(load().ntc_server_job_info(self._s, int(jid), ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in ntc_job_info._fields_}

    def predict(self, job_ids, idx) -> np.ndarray:
        """idx: [n][order] (padded to 8 columns here) for the jobs named in job_ids."""
        job_ids = np.ascontiguousarray(job_ids, dtype=np.int64)
        idx = np.asarray(idx, dtype=np.int32)
        q = np.zeros((len(job_ids), 8), dtype=np.int32)
        q[:, :idx.shape[1]] = idx
        out = np.empty(len(job_ids), dtype=np.float32)
        self._check(load().ntc_server_predict(self._s, len(job_ids), _ptr(job_ids), _ptr(q), _ptr(out)))
        return out

    def get_factor(self, jid: int, mode: int, rows: int, rank: int) -> np.ndarray:
        out = np.empty((rows, rank), dtype=np.float32)
        self._check(load().ntc_server_get_factor(self._s, int(jid), int(mode), _ptr(out)))
        return out

    def stats(self) -> dict:
        out = ntc_server_stats()
        self._check(load().ntc_server_stats_get(self._s, ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in ntc_server_stats._fields_}
