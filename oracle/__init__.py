"""CPU oracle for the KS change-point path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with the CUDA library: ``ks_oracle.c`` is plain single-pass C
written from the paper's definitions (Sec. II-C-1: D = max_x |F(x) - G(x)|; Eq. 1: the
Kolmogorov critical value; Sec. IV-B-1 step (4): every index is a candidate change point;
Eq. 2: the geometric-mapping reduction).  Every function here cites the passage it follows
in its docstring; the C file's header states the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ks_oracle.c")
_LIB = os.path.join(_HERE, "libks_oracle.so")
_lib = None

OK, EINVAL, ECAPACITY, ENOMEM = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.oracle_sort_series.argtypes = [vp, i32, i32, vp, vp]
        L.oracle_scan_segment.argtypes = [vp, vp, i64, i32, i32, i32, i32, vp, vp, vp]
        L.oracle_kolmogorov_q.argtypes = [dbl]
        L.oracle_kolmogorov_q.restype = dbl
        L.oracle_lambda.argtypes = [i64, i64, i64]
        L.oracle_lambda.restype = dbl
        L.oracle_pvalue.argtypes = [i64, i64, i64]
        L.oracle_pvalue.restype = dbl
        L.oracle_critical_value.argtypes = [dbl, i64, i64]
        L.oracle_critical_value.restype = dbl
        L.oracle_reduce_series.argtypes = [vp, i32, i32, vp]
        L.oracle_ks_scan.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int]
        L.oracle_ks_segment.argtypes = [vp, vp, vp, i64, dbl, i32, i32, vp, vp, vp, vp, vp, ctypes.c_int,
                                        ctypes.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def sort_series(x: np.ndarray):
    """Values of one [T, m] series sorted ascending, equal values in step order, with step labels."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    T, m = x.shape
    sv = np.empty(T * m, np.uint32)
    st = np.empty(T * m, np.int32)
    rc = _load().oracle_sort_series(_p(x), T, m, _p(sv), _p(st))
    assert rc == OK
    return sv, st


def scan_segment(x: np.ndarray, lo: int, hi: int, min_seg: int = 1):
    """Best split of steps [lo, hi) of one [T, m] series: (k, num, den) with D = num/den exact
    (Sec. II-C-1 definition of D; every index a candidate, Sec. IV-B-1 step (4))."""
    T, m = x.shape
    sv, st = sort_series(x)
    k = np.zeros(1, np.int32)
    num = np.zeros(1, np.int64)
    den = np.zeros(1, np.int64)
    rc = _load().oracle_scan_segment(_p(sv), _p(st), T * m, m, lo, hi, min_seg, _p(k), _p(num), _p(den))
    if rc != OK:
        raise ValueError(f"oracle_scan_segment rc={rc}")
    return int(k[0]), int(num[0]), int(den[0])


def kolmogorov_q(lam: float) -> float:
    """Asymptotic Kolmogorov survival function Q(lambda) (the distribution behind Eq. 1)."""
    return float(_load().oracle_kolmogorov_q(float(lam)))


def lam(num: int, den: int, N: int) -> float:
    return float(_load().oracle_lambda(num, den, N))


def pvalue(num: int, den: int, N: int) -> float:
    """p = Q(num / sqrt(N den)) for a split with D = num/den over N pooled samples."""
    return float(_load().oracle_pvalue(num, den, N))


def critical_value(alpha: float, n: int, m: int) -> float:
    """Eq. 1 read with the natural log and the minus sign: sqrt(-1/2 ln(alpha/2) (n+m)/(n m))."""
    return float(_load().oracle_critical_value(alpha, n, m))


def reduce_series(x: np.ndarray) -> np.ndarray:
    """Eq. 2: S_t = sqrt(sum_j (r_tj - min r)^2), min r the series' global minimum."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    T, m = x.shape
    S = np.empty(T, np.float64)
    assert _load().oracle_reduce_series(_p(x), T, m, _p(S)) == OK
    return S


def ks_scan(samples, offsets, steps, reduced: bool = False, nthreads: int = 1):
    """Top-level scan (all k in [1, T-1]) of every series; returns (k, num, den, p)."""
    samples = np.ascontiguousarray(samples, dtype=np.uint32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    steps = np.ascontiguousarray(steps, dtype=np.int32)
    S = steps.shape[0]
    k = np.zeros(S, np.int32)
    num = np.zeros(S, np.int64)
    den = np.zeros(S, np.int64)
    p = np.zeros(S, np.float64)
    rc = _load().oracle_ks_scan(_p(samples), _p(offsets), _p(steps), S, _p(k), _p(num), _p(den), _p(p),
                                int(reduced), nthreads)
    if rc != OK:
        raise ValueError(f"oracle_ks_scan rc={rc}")
    return k, num, den, p


def ks_segment(samples, offsets, steps, alpha: float, min_seg: int = 1, max_cp: int = 16,
               reduced: bool = False, nthreads: int = 1):
    """Binary segmentation of every series (split if p <= alpha, recurse left then right).

    Returns (rc, count, idx, num, den, p); idx/num/den/p are [S, max_cp] with unused slots
    -1/0/0/1.0; rc is ECAPACITY when some series has more than max_cp change points.
    """
    samples = np.ascontiguousarray(samples, dtype=np.uint32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    steps = np.ascontiguousarray(steps, dtype=np.int32)
    S = steps.shape[0]
    cnt = np.zeros(S, np.int32)
    idx = np.zeros((S, max_cp), np.int32)
    num = np.zeros((S, max_cp), np.int64)
    den = np.zeros((S, max_cp), np.int64)
    p = np.zeros((S, max_cp), np.float64)
    rc = _load().oracle_ks_segment(_p(samples), _p(offsets), _p(steps), S, alpha, min_seg, max_cp, _p(cnt),
                                   _p(idx), _p(num), _p(den), _p(p), int(reduced), nthreads)
    if rc not in (OK, ECAPACITY):
        raise ValueError(f"oracle_ks_segment rc={rc}")
    return rc, cnt, idx, num, den, p


def latency_stats(samples, offsets, steps):
    """Load-latency statistics of each series (Sec. IV-C: the average as the main result, plus
    p50, p95 and the standard deviation), over all T*m samples of the series.

    Readings (the paper names the statistics but not their estimators):
      mean = (sum x) / N, the exact integer sum rounded once to FP64, then one FP64 division;
      p50, p95 = nearest-rank order statistics, sorted[ceil(q N) - 1] with ceil(q N) taken
          exactly (q = 50/100 and 95/100);
      std = sqrt(var), var = (N sum x^2 - (sum x)^2) / N^2 (population variance): the exact
          integer numerator rounded once to FP64, divided by the FP64 product N * N.
    Returns (mean, p50, p95, std) arrays of length S.
    """
    samples = np.asarray(samples, dtype=np.uint32)
    offsets = np.asarray(offsets, dtype=np.int64)
    S = len(offsets) - 1
    mean = np.empty(S, np.float64)
    std = np.empty(S, np.float64)
    p50 = np.empty(S, np.uint32)
    p95 = np.empty(S, np.uint32)
    for s in range(S):
        x = samples[offsets[s]:offsets[s + 1]]
        N = int(x.size)
        sx = int(x.astype(np.uint64).sum())
        sxx = sum(int(v) * int(v) for v in x.tolist())
        mean[s] = float(sx) / float(N)
        std[s] = math.sqrt(float(N * sxx - sx * sx) / (float(N) * float(N)))
        xs = np.sort(x)
        p50[s] = xs[(50 * N + 99) // 100 - 1]
        p95[s] = xs[(95 * N + 99) // 100 - 1]
    return mean, p50, p95, std
