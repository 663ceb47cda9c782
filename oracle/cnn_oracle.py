"""CPU oracle for the learned change-point proposal — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
module.  The paper's evaluation scans every index (Sec. IV-B-1 (4)) and mentions that change
points may be shortlisted first to save computation (Sec. IV-B-1, after step (4)); this module
defines the shortlisting network exactly, in plain numpy fp64, so the CUDA kernels can be checked
against it:

Per-step summary (17 channels) of a series with T steps and m samples per step:
    channel i < 16: log2(q_i) - log2(med), q_i = sorted_step[min(m-1, floor((i + 0.5) m / 16))],
                    med = sorted_series[N // 2] (upper median of all N = T m samples)
    channel 16:     log2(1024 + 32 t) - 10   (the array size of step t, fetch-granularity steps
                    from 1 KiB, Sec. IV-B-1 (2); shifted so step 0 is 0)
    zero samples are read as 1 (log2 of a cycle count >= 1).
Network: 4 one-dimensional convolutions over the step axis, width 5, zero padding 2,
    17 -> 32 -> 32 -> 32 -> 1 channels, ReLU after the first three; the output is one logit per
    step.  Weights W_l[o, i, d] (d = 0..4 covers t-2..t+2), biases b_l[o].
Precision: the input, the weights and the three hidden activations are rounded to bfloat16
    (round to nearest even) where the GPU stores them; sums are exact here (fp64) and fp32 on
    the GPU.
Loss: softmax over the T steps; cross-entropy against the distribution uniform over the
    series' change points (series without change points are masked out); mean over the
    series that carry a target.
Adam (Kingma & Ba): lr, beta1, beta2, eps with bias correction on fp32 master weights.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, WIDTH = 17, 32, 5
LAYERS = [(N_IN, N_HID), (N_HID, N_HID), (N_HID, N_HID), (N_HID, 1)]


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def n_params() -> int:
    return sum(o * i * WIDTH + o for i, o in LAYERS)


# ----------------------------------------------------------------------------- summaries

def summaries(x2d: np.ndarray) -> np.ndarray:
    """17 x T feature matrix of one [T, m] series (float64, before bf16 rounding)."""
    x2d = np.asarray(x2d, np.uint32)
    T, m = x2d.shape
    flat = np.sort(x2d.ravel())
    med = float(max(int(flat[flat.size // 2]), 1))
    srt = np.sort(x2d, axis=1)
    idx = np.minimum(m - 1, np.floor((np.arange(16) + 0.5) * m / 16).astype(np.int64))
    q = np.maximum(srt[:, idx].astype(np.float64), 1.0)  # [T, 16]
    feat = np.empty((N_IN, T), np.float64)
    feat[:16] = (np.log2(q) - np.log2(med)).T
    feat[16] = np.log2(1024.0 + 32.0 * np.arange(T)) - 10.0
    return feat


# ----------------------------------------------------------------------------- network

def conv1d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[o, t] = b[o] + sum_{i, d} W[o, i, d] x[i, t + d - 2], zero padding (x: [Cin, T])."""
    Cin, T = x.shape
    xp = np.zeros((Cin, T + 4), np.float64)
    xp[:, 2:T + 2] = x
    y = np.repeat(b[:, None].astype(np.float64), T, axis=1)
    for d in range(WIDTH):
        y += W[:, :, d].astype(np.float64) @ xp[:, d:d + T]
    return y


def forward(params, x: np.ndarray, round_bf16: bool = True):
    """Logits [T] of one series and the cached activations.  params: list of (W, b) fp32."""
    r = bf16 if round_bf16 else (lambda v: np.asarray(v, np.float64))
    acts = [r(x)]
    zs = []
    for li, (W, b) in enumerate(params):
        z = conv1d(acts[-1], r(W), np.asarray(b, np.float64))
        zs.append(z)
        if li < len(params) - 1:
            acts.append(r(np.maximum(z, 0.0)))
    return zs[-1][0], (acts, zs)


def softmax(z: np.ndarray) -> np.ndarray:
    e = np.exp(z - z.max())
    return e / e.sum()


def target(T: int, cps) -> np.ndarray | None:
    cps = [int(c) for c in cps if 0 <= c < T]
    if not cps:
        return None
    y = np.zeros(T)
    y[cps] = 1.0 / len(cps)
    return y


def loss_and_grads(params, xs, cps_list, round_bf16: bool = True):
    """Mean cross-entropy over the series with a target, and fp64 gradients w.r.t. (W, b)."""
    grads = [(np.zeros_like(np.asarray(W, np.float64)), np.zeros_like(np.asarray(b, np.float64)))
             for W, b in params]
    r = bf16 if round_bf16 else (lambda v: np.asarray(v, np.float64))
    Wr = [r(W) for W, _ in params]
    n_valid = sum(1 for x, c in zip(xs, cps_list) if target(x.shape[1], c) is not None)
    total = 0.0
    for x, cps in zip(xs, cps_list):
        T = x.shape[1]
        y = target(T, cps)
        if y is None:
            continue
        z, (acts, zs) = forward(params, x, round_bf16)
        p = softmax(z)
        total += -float(np.sum(y * np.log(np.maximum(p, 1e-300))))
        g = ((p - y) / n_valid)[None, :]  # dL/dz4, [1, T]
        for li in range(len(params) - 1, -1, -1):
            a = acts[li]
            Cin = a.shape[0]
            ap = np.zeros((Cin, T + 4))
            ap[:, 2:T + 2] = a
            gW, gb = grads[li]
            for d in range(WIDTH):
                gW[:, :, d] += g @ ap[:, d:d + T].T
            gb += g.sum(axis=1)
            if li > 0:
                # dL/da[i, t] = sum_{o, d} W[o, i, d] g[o, t - d + 2]
                gp = np.zeros((g.shape[0], T + 4))
                gp[:, 2:T + 2] = g
                da = np.zeros((Cin, T))
                for d in range(WIDTH):
                    da += Wr[li][:, :, d].T @ gp[:, 4 - d:4 - d + T]
                g = da * (a > 0)
    return total / max(n_valid, 1), grads


def adam_step(params, grads, m_state, v_state, step: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update with bias correction (Kingma & Ba, Algorithm 1); returns new params."""
    out = []
    for li, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((W, gW), (b, gb))):
            key = (li, j)
            m = b1 * m_state.get(key, 0.0) + (1 - b1) * g
            v = b2 * v_state.get(key, 0.0) + (1 - b2) * g * g
            m_state[key], v_state[key] = m, v
            mh = m / (1 - b1 ** step)
            vh = v / (1 - b2 ** step)
            new.append(np.asarray(p, np.float64) - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out


def init_params(rng: np.random.Generator):
    """He-uniform initial weights (fp32), zero biases."""
    params = []
    for cin, cout in LAYERS:
        bound = np.sqrt(6.0 / (cin * WIDTH))
        params.append((rng.uniform(-bound, bound, size=(cout, cin, WIDTH)).astype(np.float32),
                       np.zeros(cout, np.float32)))
    return params


# ----------------------------------------------------------------------------- proposals

def propose(z: np.ndarray, n_win: int = 3, half: int = 16):
    """Top n_win windows of +-half steps from the logits: repeatedly take the largest remaining
    logit (smallest step on ties) and suppress logits within +-half of it.  Returns the window
    centres and the softmax mass inside the union of the windows."""
    T = z.shape[0]
    p = softmax(np.asarray(z, np.float64))
    alive = np.ones(T, bool)
    centres = []
    covered = np.zeros(T, bool)
    for _ in range(n_win):
        if not alive.any():
            break
        zz = np.where(alive, z, -np.inf)
        c = int(np.argmax(zz))
        centres.append(c)
        lo, hi = max(0, c - half), min(T, c + half + 1)
        alive[lo:hi] = False
        covered[lo:hi] = True
    return centres, float(p[covered].sum())
