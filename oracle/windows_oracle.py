"""Window-only learned segmentation — TEST INFRASTRUCTURE ONLY.

The learned proposal narrows the exact scan to the splits inside the network's windows; the
full scan is its fallback for low confidence and for a series whose windows hold no
significant split.  This module restates that procedure plainly, for the GPU's window-only
option to be compared with: only ``tests/`` may import it.  The windows and the confidence
fallback are inputs (they come from the network, whose parity is tested on its own).

Per series (splits k in [lo + min_seg, hi - min_seg], k the first step of the right part):
  - a series whose confidence is below the threshold takes the full binary segmentation;
  - otherwise segment [lo, hi) is scanned only at its window splits, |k - c| <= half for a
    window centre c >= 0; the best is the largest exact D, the smallest k on ties (Sec. II-C-1
    definition of D; every index a candidate, Sec. IV-B-1 step (4));
  - a segment without window splits is not split; the top level without any, or whose best
    window split is not significant (p > alpha), falls back to the full binary segmentation;
  - a significant split is a change point and both sides are segmented the same way.
"""
from __future__ import annotations

import numpy as np

from . import ks_segment, pvalue


def split_d(x2d: np.ndarray, lo: int, hi: int, k: int):
    """Exact D of split k of segment [lo, hi) as (num, den): D = max_x |F_L(x) - F_R(x)|
    = max_x |c_L(x) n_R - c_R(x) n_L| / (n_L n_R), c the counts of samples <= x."""
    left = np.sort(x2d[lo:k].ravel())
    right = np.sort(x2d[k:hi].ravel())
    vals = np.unique(x2d[lo:hi].ravel())
    cl = np.searchsorted(left, vals, side="right").astype(np.int64)
    cr = np.searchsorted(right, vals, side="right").astype(np.int64)
    nl, nr = int(left.size), int(right.size)
    return int(np.max(np.abs(cl * nr - cr * nl))), nl * nr


def splits_d(x2d: np.ndarray, lo: int, hi: int, ks):
    """split_d for several splits of one segment at once, from cumulative counts:
    c_L(k, x) = samples of steps lo .. k - 1 with value <= x, C(x) = c_L(hi, x); then
    num = m max_x |H c_L - a C| with a = k - lo, H = hi - lo, and den = (m a)(m (H - a))
    (the same quantity: c_L n_R - c_R n_L = m (H c_L - a C))."""
    seg = x2d[lo:hi]
    H, m = seg.shape
    vals, rank = np.unique(seg, return_inverse=True)
    cnt = np.zeros((H, vals.size), np.int64)
    np.add.at(cnt, (np.repeat(np.arange(H), m), rank.ravel()), 1)
    cum = np.cumsum(np.cumsum(cnt, axis=1), axis=0)  # [t, r]: steps lo .. lo + t, values <= vals[r]
    C = cum[-1]
    out = []
    for k in ks:
        a = k - lo
        g = int(np.max(np.abs(H * cum[a - 1] - a * C)))
        out.append((m * g, (m * a) * (m * (H - a))))
    return out


def _full(x2d, alpha, min_seg, max_cp):
    T, m = x2d.shape
    _, cnt, idx, num, den, p = ks_segment(x2d.ravel(), np.array([0, T * m]), np.array([T], np.int32), alpha,
                                          min_seg, max_cp)
    n = min(int(cnt[0]), max_cp)
    return int(cnt[0]), [(int(idx[0, j]), int(num[0, j]), int(den[0, j]), float(p[0, j])) for j in range(n)]


class _Fallback(Exception):
    pass


def segment_series(x2d: np.ndarray, alpha: float, min_seg: int, max_cp: int, centres, half: int,
                   low_conf: bool):
    """(count, [(k, num, den, p)] ascending, fallback) for one [T, m] series."""
    if low_conf:
        c, cps = _full(x2d, alpha, min_seg, max_cp)
        return c, cps, 1
    T, m = x2d.shape
    cps = []

    def rec(lo, hi, top):
        A, B = lo + min_seg, hi - min_seg
        if B < A:
            return
        ks = [k for k in range(A, B + 1) if any(c >= 0 and abs(k - c) <= half for c in centres)]
        if not ks:
            if top:
                raise _Fallback
            return
        bk, bn, bd = -1, 0, 1
        for k, (n, d) in zip(ks, splits_d(x2d, lo, hi, ks)):
            if bk < 0 or n * bd > bn * d:
                bk, bn, bd = k, n, d
        p = pvalue(bn, bd, m * (hi - lo))
        if p <= alpha:
            cps.append((bk, bn, bd, p))
            rec(lo, bk, False)
            rec(bk, hi, False)
        elif top:
            raise _Fallback

    try:
        rec(0, T, True)
    except _Fallback:
        c, full = _full(x2d, alpha, min_seg, max_cp)
        return c, full, 1
    cps.sort()
    return len(cps), cps[:max_cp], 0
