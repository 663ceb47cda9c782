"""Python binding of libmt4g, the B300 Kolmogorov-Smirnov change-point engine.

Argument marshalling only: every step of the path (sort, scan, p-value, segmentation) runs in
the CUDA kernels of ``libmt4g.so`` behind the C ABI declared in ``include/mt4g.h``.  PyTorch is
used for device memory and streams.  There is no CPU fallback: if the library is missing or no
CUDA device is usable, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import NamedTuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmt4g.so")

OK, EINVAL, ECAPACITY, ENOMEM, ECUDA, ETIMEOUT, ECHECK = 0, -1, -2, -3, -4, -5, -6
MODE_FULL, MODE_LEARNED, MODE_REDUCED = 0, 1, 2
OPT_WAIT_LIMIT_NS = 1
OPT_STAGE_TIMING = 2
OPT_SCAN_KPT = 3
OPT_WINDOWS = 4
OPT_HALF_WIDTH = 5
OPT_CONF_MIN_PPM = 6
OPT_GRAPH = 7
OPT_CHECKS = 8
OPT_SWEEP_SKIP = 9
OPT_LEARNED_WINDOWS = 10
SCAN_SWEEP = 8  # MT4G_OPT_SCAN_KPT value of the run sweep
MAX_STEPS = 32768
FEAT_CHANNELS = 18
CNN_PARAMS = 13377

_lib = None


class Mt4gError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mt4g error {code}: {msg}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile libmt4g.so for sm_103a (nvcc) if any source is newer than it."""
    from . import buildlib
    return buildlib.build(force=force)


def load_library():
    """Load libmt4g.so (built in-tree by build()); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise Mt4gError(ECUDA, f"CUDA library not built: {LIB_PATH} is missing (run build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.mt4g_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    L.mt4g_destroy.argtypes = [vp]
    L.mt4g_destroy.restype = None
    L.mt4g_last_error.argtypes = [vp]
    L.mt4g_last_error.restype = ctypes.c_char_p
    L.mt4g_wait.argtypes = [vp]
    L.mt4g_set_option.argtypes = [vp, ctypes.c_int, i64]
    L.mt4g_ks_scan.argtypes = [vp, vp, vp, vp, i64, i32, vp, vp, vp, vp, vp]
    L.mt4g_ks_segment.argtypes = [vp, vp, vp, vp, i64, dbl, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mt4g_learned_stats.argtypes = [vp, vp]
    L.mt4g_last_sweep.argtypes = [vp, vp]
    L.mt4g_ks_scan_noalloc.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp, vp]
    L.mt4g_selftest_wait_timeout.argtypes = [vp, i64, vp]
    L.mt4g_autotune.argtypes = [vp, vp, vp, vp, i64, vp]
    L.mt4g_autotune_save.argtypes = [vp, ctypes.c_char_p]
    L.mt4g_autotune_load.argtypes = [vp, ctypes.c_char_p]
    L.mt4g_autotune_get.argtypes = [vp, i32, i32]
    L.mt4g_critical_value.argtypes = [dbl, i64, i64]
    L.mt4g_critical_value.restype = dbl
    L.mt4g_stage_times.argtypes = [vp, vp, i32]
    L.mt4g_int32_peak.argtypes = [ctypes.c_int, vp]
    L.mt4g_latency_stats.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp, vp]
    L.mt4g_ks_segment_host.argtypes = [vp, vp, vp, vp, i64, dbl, i32, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp,
                                       vp]
    L.mt4g_last_work.argtypes = [vp, vp]
    L.mt4g_summaries.argtypes = [vp, vp, vp, vp, i64, vp, vp]
    L.mt4g_cnn_init.argtypes = [vp, ctypes.c_uint64]
    L.mt4g_cnn_get_params.argtypes = [vp, vp]
    L.mt4g_cnn_set_params.argtypes = [vp, vp]
    L.mt4g_cnn_save.argtypes = [vp, ctypes.c_char_p]
    L.mt4g_cnn_load.argtypes = [vp, ctypes.c_char_p]
    L.mt4g_cnn_forward.argtypes = [vp, vp, vp, i64, vp, vp]
    L.mt4g_cnn_grads.argtypes = [vp, vp, i32, i64, vp, vp, i32, vp, vp, vp]
    L.mt4g_cnn_train_step.argtypes = [vp, vp, i32, i64, vp, vp, i32, ctypes.c_float, vp, vp]
    L.mt4g_propose.argtypes = [vp, vp, vp, vp, i64, i32, i32, vp, vp, vp]
    _lib = L
    return L


def exported_symbols():
    """Names the header declares; the tests check the library exports each of them."""
    return ["mt4g_create", "mt4g_destroy", "mt4g_last_error", "mt4g_wait", "mt4g_set_option",
            "mt4g_ks_scan", "mt4g_ks_segment", "mt4g_stage_times", "mt4g_last_work",
            "mt4g_summaries", "mt4g_cnn_init", "mt4g_cnn_get_params", "mt4g_cnn_set_params", "mt4g_cnn_save",
            "mt4g_cnn_load", "mt4g_cnn_forward", "mt4g_cnn_grads", "mt4g_cnn_train_step", "mt4g_propose",
            "mt4g_learned_stats", "mt4g_ks_scan_noalloc", "mt4g_selftest_wait_timeout", "mt4g_critical_value",
            "mt4g_autotune", "mt4g_autotune_save", "mt4g_autotune_load", "mt4g_autotune_get",
            "mt4g_int32_peak", "mt4g_latency_stats", "mt4g_ks_segment_host", "mt4g_last_sweep"]


class ScanResult(NamedTuple):
    k: "torch.Tensor"
    dnum: "torch.Tensor"
    dden: "torch.Tensor"
    p: "torch.Tensor"


class SegmentResult(NamedTuple):
    rc: int
    count: "torch.Tensor"   # [S]
    idx: "torch.Tensor"     # [S, max_cp]
    dnum: "torch.Tensor"
    dden: "torch.Tensor"
    p: "torch.Tensor"
    fallback: "torch.Tensor"  # [S], 1 where a learned call took the full scan
    crit: "torch.Tensor"      # [S, max_cp], Eq. 1 critical value of each change point's split


def _host_tables(offsets, steps):
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    steps = np.ascontiguousarray(steps, dtype=np.int32)
    if offsets.ndim != 1 or steps.ndim != 1 or offsets.shape[0] != steps.shape[0] + 1:
        raise Mt4gError(EINVAL, "offsets must have S+1 entries and steps S entries")
    return offsets, steps


def _dev_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise Mt4gError(EINVAL, f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise Mt4gError(EINVAL, f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Engine:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0):
        import torch
        L = load_library()
        self.device = device
        torch.cuda.set_device(device)
        h = ctypes.c_void_p()
        rc = L.mt4g_create(ctypes.byref(h), device)
        if rc != OK:
            raise Mt4gError(rc, "mt4g_create failed (no usable CUDA device?)")
        self._h = h
        self._L = L

    def close(self):
        if getattr(self, "_h", None):
            self._L.mt4g_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise Mt4gError(rc, self._L.mt4g_last_error(self._h).decode())

    def last_error(self) -> str:
        return self._L.mt4g_last_error(self._h).decode()

    def wait(self) -> int:
        """Synchronise the last call's stream; returns its device-side status code."""
        return int(self._L.mt4g_wait(self._h))

    def set_option(self, option: int, value: int):
        self._check(self._L.mt4g_set_option(self._h, option, int(value)))

    def stage_times(self, max_calls: int = 1) -> np.ndarray:
        """[n, 5] ms per call (upload, sort, proposals, queue kernel, collect), last n <= 64 calls."""
        buf = np.zeros((max_calls, 5), np.float64)
        n = self._L.mt4g_stage_times(self._h, buf.ctypes.data_as(ctypes.c_void_p), max_calls)
        if n < 0:
            self._check(n)
        return buf[:n]

    def learned_stats(self) -> dict:
        """Certification counters of the last learned call (valid after wait())."""
        v = np.zeros(3, np.int64)
        self._check(self._L.mt4g_learned_stats(self._h, v.ctypes.data_as(ctypes.c_void_p)))
        return {"certified": int(v[0]), "refined": int(v[1]), "probe_groups": int(v[2])}

    def last_sweep(self) -> dict:
        """Run-sweep counters of the last call (valid after wait()): segments swept, samples ranked,
        samples sorted by counting, series the sweep does not take."""
        v = np.zeros(4, np.int64)
        self._check(self._L.mt4g_last_sweep(self._h, v.ctypes.data_as(ctypes.c_void_p)))
        return {"swept_segments": int(v[0]), "ranked_samples": int(v[1]), "counted_samples": int(v[2]),
                "unswept_series": int(v[3])}

    def selftest_wait_timeout(self, limit_ns: int = 10_000_000, stream=None) -> int:
        """Run the queue kernel on a queue whose pending item never comes; returns mt4g_wait()'s code."""
        self._check(self._L.mt4g_selftest_wait_timeout(self._h, int(limit_ns), _stream_handle(stream)))
        return self.wait()

    def autotune(self, samples, offsets, steps, stream=None):
        """Time each scan tile per (log2 T, log2 m) bucket of the batch and keep the fastest."""
        offsets, steps = _host_tables(offsets, steps)
        self._check(self._L.mt4g_autotune(self._h, _dev_ptr(samples, "samples"), offsets.ctypes.data_as(ctypes.c_void_p),
                                          steps.ctypes.data_as(ctypes.c_void_p), steps.shape[0],
                                          _stream_handle(stream)))

    def autotune_save(self, path: str):
        self._check(self._L.mt4g_autotune_save(self._h, os.fsencode(path)))

    def autotune_load(self, path: str):
        self._check(self._L.mt4g_autotune_load(self._h, os.fsencode(path)))

    def autotune_get(self, T: int, m: int) -> int:
        v = int(self._L.mt4g_autotune_get(self._h, int(T), int(m)))
        if v < 0:
            self._check(v)
        return v

    def last_work(self) -> int:
        """(split, distinct value) pairs evaluated by the last call (valid after wait())."""
        v = np.zeros(1, np.int64)
        self._check(self._L.mt4g_last_work(self._h, v.ctypes.data_as(ctypes.c_void_p)))
        return int(v[0])

    def ks_scan(self, samples, offsets, steps, mode: int = MODE_FULL, stream=None, out=None,
                sync: bool = True) -> ScanResult:
        import torch
        offsets, steps = _host_tables(offsets, steps)
        S = steps.shape[0]
        dev = samples.device
        if out is None:
            out = ScanResult(torch.empty(S, dtype=torch.int32, device=dev), torch.empty(S, dtype=torch.int64, device=dev),
                             torch.empty(S, dtype=torch.int64, device=dev), torch.empty(S, dtype=torch.float64, device=dev))
        rc = self._L.mt4g_ks_scan(self._h, _dev_ptr(samples, "samples"), offsets.ctypes.data_as(ctypes.c_void_p),
                                  steps.ctypes.data_as(ctypes.c_void_p), S, mode, _dev_ptr(out.k, "k"),
                                  _dev_ptr(out.dnum, "dnum"), _dev_ptr(out.dden, "dden"), _dev_ptr(out.p, "p"),
                                  _stream_handle(stream))
        self._check(rc)
        if sync:
            self._check(self.wait())
        return out

    def ks_segment(self, samples, offsets, steps, alpha: float, min_seg: int = 1, max_cp: int = 16,
                   mode: int = MODE_FULL, stream=None, out=None, sync: bool = True) -> SegmentResult:
        import torch
        offsets, steps = _host_tables(offsets, steps)
        S = steps.shape[0]
        dev = samples.device
        if out is None:
            out = SegmentResult(0, torch.empty(S, dtype=torch.int32, device=dev),
                                torch.empty((S, max_cp), dtype=torch.int32, device=dev),
                                torch.empty((S, max_cp), dtype=torch.int64, device=dev),
                                torch.empty((S, max_cp), dtype=torch.int64, device=dev),
                                torch.empty((S, max_cp), dtype=torch.float64, device=dev),
                                torch.empty(S, dtype=torch.int32, device=dev),
                                torch.empty((S, max_cp), dtype=torch.float64, device=dev))
        rc = self._L.mt4g_ks_segment(self._h, _dev_ptr(samples, "samples"), offsets.ctypes.data_as(ctypes.c_void_p),
                                     steps.ctypes.data_as(ctypes.c_void_p), S, float(alpha), int(min_seg),
                                     int(max_cp), mode, _dev_ptr(out.count, "count"), _dev_ptr(out.idx, "idx"),
                                     _dev_ptr(out.dnum, "dnum"), _dev_ptr(out.dden, "dden"), _dev_ptr(out.p, "p"),
                                     _dev_ptr(out.fallback, "fallback"), _dev_ptr(out.crit, "crit"),
                                     _stream_handle(stream))
        self._check(rc)
        status = OK
        if sync:
            status = self.wait()
            if status not in (OK, ECAPACITY):
                self._check(status)
        return out._replace(rc=status)

    def ks_segment_host(self, samples_host, offsets, steps, alpha: float, min_seg: int = 1, max_cp: int = 16,
                        mode: int = MODE_FULL, chunk_samples: int = 0, stream=None, out=None, device=None,
                        sync: bool = True) -> SegmentResult:
        """mt4g_ks_segment_host: samples in host memory (a CPU tensor, page-locked for overlap, or a
        numpy array), copied chunk by chunk while earlier chunks are segmented.  Outputs on the
        device; samples_host must stay alive until wait()."""
        import torch
        offsets, steps = _host_tables(offsets, steps)
        S = steps.shape[0]
        if isinstance(samples_host, np.ndarray):
            if samples_host.dtype not in (np.uint32, np.int32) or not samples_host.flags.c_contiguous:
                raise Mt4gError(EINVAL, "host samples must be a contiguous uint32 array")
            ptr = samples_host.ctypes.data_as(ctypes.c_void_p)
        else:
            if not isinstance(samples_host, torch.Tensor) or samples_host.is_cuda or not samples_host.is_contiguous():
                raise Mt4gError(EINVAL, "host samples must be a contiguous CPU tensor or numpy array")
            ptr = ctypes.c_void_p(samples_host.data_ptr())
        dev = torch.device("cuda", self.device) if device is None else device
        if out is None:
            out = SegmentResult(0, torch.empty(S, dtype=torch.int32, device=dev),
                                torch.empty((S, max_cp), dtype=torch.int32, device=dev),
                                torch.empty((S, max_cp), dtype=torch.int64, device=dev),
                                torch.empty((S, max_cp), dtype=torch.int64, device=dev),
                                torch.empty((S, max_cp), dtype=torch.float64, device=dev),
                                torch.empty(S, dtype=torch.int32, device=dev),
                                torch.empty((S, max_cp), dtype=torch.float64, device=dev))
        rc = self._L.mt4g_ks_segment_host(self._h, ptr, offsets.ctypes.data_as(ctypes.c_void_p),
                                          steps.ctypes.data_as(ctypes.c_void_p), S, float(alpha), int(min_seg),
                                          int(max_cp), mode, int(chunk_samples), _dev_ptr(out.count, "count"),
                                          _dev_ptr(out.idx, "idx"), _dev_ptr(out.dnum, "dnum"),
                                          _dev_ptr(out.dden, "dden"), _dev_ptr(out.p, "p"),
                                          _dev_ptr(out.fallback, "fallback"), _dev_ptr(out.crit, "crit"),
                                          _stream_handle(stream))
        self._check(rc)
        status = OK
        if sync:
            status = self.wait()
            if status not in (OK, ECAPACITY):
                self._check(status)
        return out._replace(rc=status)


def int32_peak(device: int = 0) -> float:
    """Measured rate (10^12 ops/s) of the scan's integer step mix on every SM (mt4g_int32_peak)."""
    v = np.zeros(1, np.float64)
    rc = load_library().mt4g_int32_peak(int(device), v.ctypes.data_as(ctypes.c_void_p))
    if rc != OK:
        raise Mt4gError(rc, "mt4g_int32_peak failed")
    return float(v[0])


def critical_value(alpha: float, n_left: int, n_right: int) -> float:
    """Eq. 1 critical value of D (host computation in the library)."""
    return float(load_library().mt4g_critical_value(float(alpha), int(n_left), int(n_right)))


def feature_rows(steps) -> int:
    """Rows of the padded feature layout: sum over series of T_s + 4."""
    steps = np.asarray(steps, np.int64)
    return int(steps.sum() + 4 * steps.shape[0])


def _mixin_learned(cls):
    """Learned-proposal calls of Engine (kept apart for readability)."""

    def summaries(self, samples, offsets, steps, stream=None, out=None, sync=True):
        import torch
        offsets, steps = _host_tables(offsets, steps)
        rows = feature_rows(steps)
        if out is None:
            out = torch.empty((rows, FEAT_CHANNELS), dtype=torch.int16, device=samples.device)
        self._check(self._L.mt4g_summaries(self._h, _dev_ptr(samples, "samples"),
                                           offsets.ctypes.data_as(ctypes.c_void_p),
                                           steps.ctypes.data_as(ctypes.c_void_p), steps.shape[0],
                                           _dev_ptr(out, "feat"), _stream_handle(stream)))
        if sync:
            self._check(self.wait())
        return out

    def latency_stats(self, samples, offsets, steps, stream=None, sync=True):
        """mt4g_latency_stats: per-series (mean, p50, p95, std) device tensors.  mean and std are
        float64; p50 and p95 hold the uint32 sample values in int32 tensors (bit patterns: view
        them as uint32 on the host, e.g. t.cpu().numpy().view(np.uint32))."""
        import torch
        offsets, steps = _host_tables(offsets, steps)
        S = steps.shape[0]
        dev = samples.device
        mean = torch.empty(S, dtype=torch.float64, device=dev)
        std = torch.empty(S, dtype=torch.float64, device=dev)
        p50 = torch.empty(S, dtype=torch.int32, device=dev)
        p95 = torch.empty(S, dtype=torch.int32, device=dev)
        self._check(self._L.mt4g_latency_stats(self._h, _dev_ptr(samples, "samples"),
                                               offsets.ctypes.data_as(ctypes.c_void_p),
                                               steps.ctypes.data_as(ctypes.c_void_p), S, _dev_ptr(mean, "mean"),
                                               _dev_ptr(p50, "p50"), _dev_ptr(p95, "p95"), _dev_ptr(std, "std"),
                                               _stream_handle(stream)))
        if sync:
            self._check(self.wait())
        return mean, p50, p95, std

    def cnn_init(self, seed: int):
        self._check(self._L.mt4g_cnn_init(self._h, int(seed)))

    def cnn_get_params(self) -> np.ndarray:
        w = np.zeros(CNN_PARAMS, np.float32)
        self._check(self._L.mt4g_cnn_get_params(self._h, w.ctypes.data_as(ctypes.c_void_p)))
        return w

    def cnn_set_params(self, w: np.ndarray):
        w = np.ascontiguousarray(w, np.float32)
        assert w.shape == (CNN_PARAMS,)
        self._check(self._L.mt4g_cnn_set_params(self._h, w.ctypes.data_as(ctypes.c_void_p)))

    def cnn_save(self, path: str):
        self._check(self._L.mt4g_cnn_save(self._h, os.fsencode(path)))

    def cnn_load(self, path: str):
        self._check(self._L.mt4g_cnn_load(self._h, os.fsencode(path)))

    def cnn_forward(self, feat, steps, stream=None, out=None):
        import torch
        steps = np.ascontiguousarray(steps, np.int32)
        if out is None:
            out = torch.zeros(feature_rows(steps), dtype=torch.float32, device=feat.device)
        self._check(self._L.mt4g_cnn_forward(self._h, _dev_ptr(feat, "feat"), steps.ctypes.data_as(ctypes.c_void_p),
                                             steps.shape[0], _dev_ptr(out, "logits"), _stream_handle(stream)))
        return out

    def cnn_grads(self, feat, T, B, cp_count, cp_idx, stream=None):
        import torch
        grad = torch.zeros(CNN_PARAMS, dtype=torch.float32, device=feat.device)
        loss = torch.zeros(1, dtype=torch.float32, device=feat.device)
        self._check(self._L.mt4g_cnn_grads(self._h, _dev_ptr(feat, "feat"), int(T), int(B),
                                           _dev_ptr(cp_count, "cp_count"), _dev_ptr(cp_idx, "cp_idx"),
                                           int(cp_idx.shape[-1]), _dev_ptr(grad, "grad"), _dev_ptr(loss, "loss"),
                                           _stream_handle(stream)))
        return grad, loss

    def cnn_train_step(self, feat, T, B, cp_count, cp_idx, lr=1e-3, loss=None, stream=None):
        self._check(self._L.mt4g_cnn_train_step(self._h, _dev_ptr(feat, "feat"), int(T), int(B),
                                                _dev_ptr(cp_count, "cp_count"), _dev_ptr(cp_idx, "cp_idx"),
                                                int(cp_idx.shape[-1]), ctypes.c_float(lr),
                                                _dev_ptr(loss, "loss") if loss is not None else None,
                                                _stream_handle(stream)))

    def propose(self, samples, offsets, steps, n_win=3, half_width=16, stream=None, sync=True):
        import torch
        offsets, steps = _host_tables(offsets, steps)
        S = steps.shape[0]
        win = torch.empty((S, n_win), dtype=torch.int32, device=samples.device)
        conf = torch.empty(S, dtype=torch.float32, device=samples.device)
        self._check(self._L.mt4g_propose(self._h, _dev_ptr(samples, "samples"),
                                         offsets.ctypes.data_as(ctypes.c_void_p),
                                         steps.ctypes.data_as(ctypes.c_void_p), S, int(n_win), int(half_width),
                                         _dev_ptr(win, "win"), _dev_ptr(conf, "conf"), _stream_handle(stream)))
        if sync:
            self._check(self.wait())
        return win, conf

    for name, fn in list(locals().items()):
        if callable(fn) and not name.startswith("_"):
            setattr(cls, name, fn)
    return cls


Engine = _mixin_learned(Engine)


NOALLOC_MAX_SERIES, NOALLOC_MAX_SAMPLES, NOALLOC_MAX_STEPS = 4096, 1 << 19, 1 << 16


def ks_scan_noalloc(samples, offsets, steps, out, stream=None) -> int:
    """mt4g_ks_scan_noalloc: the top-level scan without any allocation by the library.

    For callers that cannot allocate device memory: code running inside a memory pool or
    arena that someone else owns, or a process that forbids allocation after start-up.
    ``out`` must be a ScanResult of preallocated device tensors (int32, int64, int64,
    float64, at least S elements each) on the device of ``samples``; returns the C status
    code.  Runs on the device of ``samples`` and synchronises ``stream``.  Limits:
    NOALLOC_MAX_SERIES series, NOALLOC_MAX_SAMPLES samples, NOALLOC_MAX_STEPS steps in total.
    """
    import torch
    L = load_library()
    offsets, steps = _host_tables(offsets, steps)
    S = steps.shape[0]
    want = (("k", out.k, torch.int32), ("dnum", out.dnum, torch.int64), ("dden", out.dden, torch.int64),
            ("p", out.p, torch.float64))
    ptrs = [_dev_ptr(samples, "samples")] + [_dev_ptr(t, name) for name, t, _ in want]
    if samples.dtype not in (torch.int32, torch.uint32):
        raise Mt4gError(EINVAL, "samples must hold 32-bit words (int32 or uint32)")
    if S and samples.numel() < int(offsets[-1]):
        raise Mt4gError(EINVAL, "samples holds fewer elements than offsets[-1]")
    for name, t, dt in want:
        if t.dtype != dt:
            raise Mt4gError(EINVAL, f"out.{name} must be {dt}")
        if t.numel() < S:
            raise Mt4gError(EINVAL, f"out.{name} holds fewer than S elements")
        if t.device != samples.device:
            raise Mt4gError(EINVAL, f"out.{name} is not on the device of samples")
    with torch.cuda.device(samples.device):
        return int(L.mt4g_ks_scan_noalloc(ptrs[0], offsets.ctypes.data_as(ctypes.c_void_p),
                                          steps.ctypes.data_as(ctypes.c_void_p), S, *ptrs[1:],
                                          _stream_handle(stream)))


def to_device_samples(samples: np.ndarray, device="cuda"):
    """Copy uint32 host samples to a device tensor (stored as int32 bits)."""
    import torch
    a = np.ascontiguousarray(samples, dtype=np.uint32).view(np.int32)
    return torch.from_numpy(a).to(device)
