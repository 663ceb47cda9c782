"""Seeded synthetic latency-series inputs shared by the oracle, the tests and the benchmark.

The generator (``gen.c``) holds no arithmetic of the change-point method; it only draws
series of uint32 cycle counts shaped like the size benchmarks' 2D result array (one row
per array-size step, the first m latencies of each kept; paper Sec. IV-B-1, step (4)).
Series are stored step-major, ``samples[offsets[s] + t*m_s + j]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libmt4g_synth.so")
MAX_CP = 8
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libmt4g_synth.so (plain gcc, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.mt4g_synth_params.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                          i32p, i32p, i32p, i32p]
        lib.mt4g_synth_params.restype = ctypes.c_int
        lib.mt4g_synth_fill.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_int]
        lib.mt4g_synth_fill.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


@dataclass
class Batch:
    """A batch of series: step-major samples plus shapes and the generator's truth."""
    samples: np.ndarray   # uint32 [offsets[-1]]
    offsets: np.ndarray   # int64 [S+1]
    steps: np.ndarray     # int32 [S]  (T_s)
    m: np.ndarray         # int32 [S]
    ncp: np.ndarray       # int32 [S]  true number of change points
    cps: np.ndarray       # int32 [S, MAX_CP], -1 padded

    @property
    def S(self) -> int:
        return int(self.steps.shape[0])

    def series(self, s: int) -> np.ndarray:
        """Series s as a [T, m] view."""
        return self.samples[self.offsets[s]:self.offsets[s + 1]].reshape(int(self.steps[s]), int(self.m[s]))


def params(cfg: int, seed: int, count: int, series_begin: int = 0):
    lib = _load()
    T = np.zeros(count, np.int32)
    m = np.zeros(count, np.int32)
    ncp = np.zeros(count, np.int32)
    cps = np.zeros((count, MAX_CP), np.int32)
    rc = lib.mt4g_synth_params(cfg, seed, series_begin, count, _ptr(T, ctypes.c_int32), _ptr(m, ctypes.c_int32),
                               _ptr(ncp, ctypes.c_int32), _ptr(cps, ctypes.c_int32))
    if rc != 0:
        raise ValueError(f"unknown workload {cfg}")
    return T, m, ncp, cps


def generate(cfg: int, seed: int, count: int, series_begin: int = 0, nthreads: int | None = None,
             out: np.ndarray | None = None) -> Batch:
    """Generate series [series_begin, series_begin+count) of workload ``cfg``.

    ``out`` may be a preallocated (e.g. pinned) uint32 array of at least the batch's size.
    """
    lib = _load()
    T, m, ncp, cps = params(cfg, seed, count, series_begin)
    offsets = np.zeros(count + 1, np.int64)
    np.cumsum(T.astype(np.int64) * m.astype(np.int64), out=offsets[1:])
    total = int(offsets[-1])
    if out is None:
        samples = np.empty(total, np.uint32)
    else:
        assert out.dtype == np.uint32 and out.size >= total
        samples = out[:total]
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib.mt4g_synth_fill(cfg, seed, series_begin, count, _ptr(offsets, ctypes.c_int64),
                             samples.ctypes.data_as(ctypes.c_void_p), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"mt4g_synth_fill failed ({rc})")
    return Batch(samples, offsets, T, m, ncp, cps)


def tiny_random(rng: np.random.Generator, S: int, T_range=(2, 8), m_range=(1, 4), vmax: int = 5) -> Batch:
    """Small random series with heavy ties (values in 0..vmax) for exhaustive checks."""
    T = rng.integers(T_range[0], T_range[1] + 1, size=S).astype(np.int32)
    m = rng.integers(m_range[0], m_range[1] + 1, size=S).astype(np.int32)
    offsets = np.zeros(S + 1, np.int64)
    np.cumsum(T.astype(np.int64) * m, out=offsets[1:])
    samples = rng.integers(0, vmax + 1, size=int(offsets[-1])).astype(np.uint32)
    return Batch(samples, offsets, T, m, np.zeros(S, np.int32), -np.ones((S, MAX_CP), np.int32))


def from_arrays(series_list) -> Batch:
    """Pack a list of [T, m] uint32 arrays into one step-major batch."""
    T = np.array([a.shape[0] for a in series_list], np.int32)
    m = np.array([a.shape[1] for a in series_list], np.int32)
    offsets = np.zeros(len(series_list) + 1, np.int64)
    np.cumsum(T.astype(np.int64) * m, out=offsets[1:])
    samples = np.concatenate([np.ascontiguousarray(a, dtype=np.uint32).ravel() for a in series_list]) \
        if series_list else np.zeros(0, np.uint32)
    S = len(series_list)
    return Batch(samples, offsets, T, m, np.zeros(S, np.int32), -np.ones((S, MAX_CP), np.int32))


# ----------------------------------------------------------------------------- GPU twin

_SRC_GPU = os.path.join(_HERE, "gen_gpu.cu")
_LIB_GPU = os.path.join(_HERE, "libmt4g_synth_gpu.so")
_lib_gpu = None


def build_gpu(force: bool = False) -> str:
    """Compile gen_gpu.cu (the FP32 GPU twin of the generator) for sm_103a."""
    if force or not os.path.exists(_LIB_GPU) or os.path.getmtime(_LIB_GPU) < os.path.getmtime(_SRC_GPU):
        tmp = _LIB_GPU + f".tmp{os.getpid()}"
        subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared", "-o", tmp, _SRC_GPU,
                               "-Xlinker", "-rpath,/usr/local/cuda/lib64"])
        os.replace(tmp, _LIB_GPU)
    return _LIB_GPU


def _load_gpu():
    global _lib_gpu
    if _lib_gpu is None:
        build_gpu()
        lib = ctypes.CDLL(_LIB_GPU)
        lib.mt4g_synth_fill_gpu.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.mt4g_synth_fill_gpu.restype = ctypes.c_int
        _lib_gpu = lib
    return _lib_gpu


def generate_gpu(cfg: int, seed: int, count: int, series_begin: int = 0, device="cuda", stream=None):
    """Generate series on the GPU (same recipe and seeds as generate(), FP32 draws, so values differ).

    Returns (samples as a device int32 tensor holding the uint32 bits, Batch with host shapes and
    truth; its .samples is None).
    """
    import torch
    T, m, ncp, cps = params(cfg, seed, count, series_begin)
    offsets = np.zeros(count + 1, np.int64)
    np.cumsum(T.astype(np.int64) * m.astype(np.int64), out=offsets[1:])
    d_off = torch.from_numpy(offsets).to(device)
    samples = torch.empty(int(offsets[-1]), dtype=torch.int32, device=device)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = _load_gpu().mt4g_synth_fill_gpu(cfg, seed, series_begin, count, int(T.max()),
                                         ctypes.c_void_p(d_off.data_ptr()), ctypes.c_void_p(samples.data_ptr()),
                                         ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"mt4g_synth_fill_gpu failed ({rc})")
    return samples, Batch(None, offsets, T, m, ncp, cps)
