"""Pins of the window-only segmentation oracle (oracle/windows_oracle.py) on the CPU.

- split_d against the C oracle's best split: over every split of a segment the largest
  split_d is the C oracle's D (a different implementation of the definition); the
  cumulative-count form splits_d equals split_d split by split;
- windows that cover every split reduce the procedure to the full binary segmentation, which
  the C oracle computes on its own;
- a low-confidence series takes the full segmentation and is flagged;
- a series whose windows hold no significant split falls back to the full segmentation, and
  one whose windows miss its change reports what the windows hold.
"""
import numpy as np

import oracle
import synth
from oracle import windows_oracle as W


def test_split_d_matches_c_oracle_best():
    rng = np.random.default_rng(3)
    for _ in range(12):
        T, m = int(rng.integers(4, 30)), int(rng.integers(1, 6))
        x = rng.integers(0, int(rng.integers(2, 40)), size=(T, m)).astype(np.uint32)
        x[int(rng.integers(1, T)):] += int(rng.integers(0, 5))
        lo = int(rng.integers(0, T - 2))
        hi = int(rng.integers(lo + 2, T + 1))
        k, num, den = oracle.scan_segment(x, lo, hi)
        best = None
        for kk in range(lo + 1, hi):
            n, d = W.split_d(x, lo, hi, kk)
            if best is None or n * best[2] > best[1] * d:
                best = (kk, n, d)
        assert best[1] * den == num * best[2]
        assert best[0] == k


def test_splits_d_equals_split_d():
    rng = np.random.default_rng(4)
    for _ in range(10):
        T, m = int(rng.integers(4, 40)), int(rng.integers(1, 9))
        x = rng.integers(0, int(rng.integers(2, 300)), size=(T, m)).astype(np.uint32)
        lo = int(rng.integers(0, T - 2))
        hi = int(rng.integers(lo + 2, T + 1))
        ks = list(range(lo + 1, hi))
        for k, (n, d) in zip(ks, W.splits_d(x, lo, hi, ks)):
            n2, d2 = W.split_d(x, lo, hi, k)
            assert (n, d) == (n2, d2)


def test_covering_windows_reduce_to_full_segmentation():
    b = synth.generate(1, 0, 1)
    x = b.series(0)
    T = x.shape[0]
    c_full, full = W._full(x, 1e-6, 1, 16)
    c, cps, fb = W.segment_series(x, 1e-6, 1, 16, [T // 2], T, False)
    assert fb == 0 and c == c_full and cps == full


def test_low_confidence_and_empty_windows_fall_back():
    b = synth.generate(1, 0, 1)
    x = b.series(0)
    c_full, full = W._full(x, 1e-6, 1, 16)
    assert c_full >= 1
    assert W.segment_series(x, 1e-6, 1, 16, [5], 2, True) == (c_full, full, 1)
    # no window at all
    assert W.segment_series(x, 1e-6, 1, 16, [-1, -1], 16, False) == (c_full, full, 1)
    # a series without a change: its windows hold nothing significant -> the full scan (none)
    rng = np.random.default_rng(5)
    y = (32 + rng.poisson(2, size=(64, 32))).astype(np.uint32)
    assert W._full(y, 1e-6, 1, 16) == (0, [])
    assert W.segment_series(y, 1e-6, 1, 16, [20, 40], 8, False) == (0, [], 1)
    # a window away from the change can still hold a significant split: the procedure then
    # reports it (the full scan's answer differs; the agreement rate counts such series)
    c, cps, fb = W.segment_series(x, 1e-6, 1, 16, [1], 2, False)
    assert fb == 0 and cps[0][0] <= 3
