"""Pins for the CPU oracle: it is checked against things other than itself.

- D and the split: exact-rational brute force straight from the textbook definition
  D = max_x |F(x) - G(x)| (paper Sec. II-C-1) over every split (Sec. IV-B-1 step (4)),
  exhaustively on tiny inputs with heavy ties; scipy's two-sample KS statistic; closed forms;
  invariants (order reversal, strictly increasing value maps, permutation within a step).
- p-value: scipy.special.kolmogorov (an independent implementation of the Kolmogorov
  survival function), a 50-digit mpmath evaluation, textbook quantiles, Eq. 1 consistency,
  and a loose permutation-test sanity check.
- Binary segmentation: a brute-force recursion built on the rational brute force and
  scipy's Kolmogorov function.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.special
import scipy.stats

import oracle
import synth


# ----------------------------------------------------------------------------- brute force

def brute_D(L, R) -> Fraction:
    """D = max over pooled x of |F_L(x) - F_R(x)| in exact rationals (Sec. II-C-1)."""
    best = Fraction(0)
    for x in sorted(set(L) | set(R)):
        fl = Fraction(sum(1 for v in L if v <= x), len(L))
        fr = Fraction(sum(1 for v in R if v <= x), len(R))
        best = max(best, abs(fl - fr))
    return best


def brute_scan(x2d, lo, hi, min_seg=1):
    best = None
    for k in range(lo + min_seg, hi - min_seg + 1):
        D = brute_D(list(x2d[lo:k].ravel()), list(x2d[k:hi].ravel()))
        if best is None or D > best[1]:
            best = (k, D)
    return best


def check_against_brute(x2d, lo=0, hi=None, min_seg=1):
    T, m = x2d.shape
    hi = T if hi is None else hi
    k, num, den = oracle.scan_segment(x2d, lo, hi, min_seg)
    bk, bD = brute_scan(x2d, lo, hi, min_seg)
    assert k == bk, (x2d.tolist(), lo, hi, k, bk)
    assert den == m * (k - lo) * m * (hi - k)
    assert Fraction(num, den) == bD
    assert 0 <= num <= den


def test_exhaustive_m1_T4_values_0_3():
    for vals in itertools.product(range(4), repeat=4):
        check_against_brute(np.array(vals, np.uint32).reshape(4, 1))


def test_exhaustive_m2_T3_values_0_2():
    for vals in itertools.product(range(3), repeat=6):
        check_against_brute(np.array(vals, np.uint32).reshape(3, 2))


def test_random_tiny_with_segments_and_min_seg(rng):
    for _ in range(300):
        T = int(rng.integers(2, 9))
        m = int(rng.integers(1, 5))
        x = rng.integers(0, 6, size=(T, m)).astype(np.uint32)
        lo = int(rng.integers(0, T - 1))
        hi = int(rng.integers(lo + 2, T + 1))
        min_seg = int(rng.integers(1, (hi - lo) // 2 + 1))
        check_against_brute(x, lo, hi, min_seg)


def test_scipy_ks_2samp_statistic(rng):
    """scipy's two-sample statistic is an independent implementation of the same D."""
    for _ in range(200):
        T = int(rng.integers(2, 30))
        m = int(rng.integers(1, 20))
        x = rng.integers(0, int(rng.integers(2, 200)), size=(T, m)).astype(np.uint32)
        k, num, den = oracle.scan_segment(x, 0, T)
        d = scipy.stats.ks_2samp(x[:k].ravel(), x[k:].ravel(), method="asymp").statistic
        assert abs(num / den - d) < 1e-12
        # and no other split has a larger scipy statistic
        for kk in range(1, T):
            dk = scipy.stats.ks_2samp(x[:kk].ravel(), x[kk:].ravel(), method="asymp").statistic
            assert dk <= d + 1e-12


# ----------------------------------------------------------------------------- closed forms

def test_disjoint_supports_give_D_one():
    rng = np.random.default_rng(7)
    for _ in range(50):
        T = int(rng.integers(2, 40))
        m = int(rng.integers(1, 16))
        k0 = int(rng.integers(1, T))
        x = np.empty((T, m), np.uint32)
        x[:k0] = rng.integers(1, 100, size=(k0, m))
        x[k0:] = rng.integers(100, 200, size=(T - k0, m))
        k, num, den = oracle.scan_segment(x, 0, T)
        # D = 1 exactly; an earlier split can also separate the supports (ties go left)
        assert num == den and k <= k0 and x[:k].max() < x[k:].min()


def test_all_equal_gives_D_zero_p_one():
    for T, m in [(2, 1), (5, 3), (64, 32)]:
        x = np.full((T, m), 77, np.uint32)
        k, num, den = oracle.scan_segment(x, 0, T)
        assert num == 0 and k == 1 and den == m * (T - 1) * m
        assert oracle.pvalue(num, den, T * m) == 1.0


def test_shifted_uniform_two_steps():
    """Step 0 = {1..m}, step 1 = {1+s..m+s}: D = min(s, m)/m, i.e. num = min(s,m) m, den = m^2."""
    for m in range(1, 12):
        for s in range(0, m + 3):
            x = np.stack([np.arange(1, m + 1), np.arange(1 + s, m + 1 + s)]).astype(np.uint32)
            k, num, den = oracle.scan_segment(x, 0, 2)
            assert (k, num, den) == (1, min(s, m) * m, m * m)


def test_nested_uniform_prefix_construction():
    """L = {1..a}, R = {1..b}, a < b: D = max_x (x/a - x/b) = 1 - a/b at x = a.  Two steps of
    equal size force the split: step 0 holds each of 1..a b times, step 1 each of 1..b a times
    (the same ECDFs as L and R), so T = 2 leaves only k = 1."""
    for a in range(1, 8):
        for b in range(a + 1, 10):
            D_direct = brute_D(list(range(1, a + 1)), list(range(1, b + 1)))
            assert D_direct == 1 - Fraction(a, b)
            x = np.array([np.repeat(np.arange(1, a + 1), b), np.repeat(np.arange(1, b + 1), a)], np.uint32)
            k, num, den = oracle.scan_segment(x, 0, 2)
            assert k == 1 and Fraction(num, den) == 1 - Fraction(a, b)
            assert den == (a * b) * (a * b)  # n_L n_R


# ----------------------------------------------------------------------------- invariants

def _random_series(rng, T, m, vmax):
    return rng.integers(0, vmax, size=(T, m)).astype(np.uint32)


def test_reversal_symmetry(rng):
    for _ in range(100):
        T, m = int(rng.integers(2, 30)), int(rng.integers(1, 10))
        x = _random_series(rng, T, m, int(rng.integers(2, 50)))
        k, num, den = oracle.scan_segment(x, 0, T)
        k2, num2, den2 = oracle.scan_segment(x[::-1].copy(), 0, T)
        assert Fraction(num, den) == Fraction(num2, den2)
        assert (num, den) == (num2, den2) or k2 != T - k  # same split => identical pair
        if k2 == T - k:
            assert (num, den) == (num2, den2)


def test_strictly_increasing_maps(rng):
    for _ in range(100):
        T, m = int(rng.integers(2, 30)), int(rng.integers(1, 10))
        x = _random_series(rng, T, m, 1000)
        ref = oracle.scan_segment(x, 0, T)
        assert oracle.scan_segment((2 * x + 7).astype(np.uint32), 0, T) == ref
        assert oracle.scan_segment((x.astype(np.uint64) ** 2).astype(np.uint32), 0, T) == ref


def test_permutation_within_steps(rng):
    for _ in range(100):
        T, m = int(rng.integers(2, 30)), int(rng.integers(2, 10))
        x = _random_series(rng, T, m, 20)
        ref = oracle.scan_segment(x, 0, T)
        y = np.array([rng.permutation(row) for row in x], np.uint32)
        assert oracle.scan_segment(y, 0, T) == ref


def test_sort_matches_numpy_stable_argsort(rng):
    for _ in range(20):
        T, m = int(rng.integers(2, 50)), int(rng.integers(1, 30))
        x = _random_series(rng, T, m, 40)
        sv, st = oracle.sort_series(x)
        order = np.argsort(x.ravel(), kind="stable")
        assert np.array_equal(sv, x.ravel()[order])
        assert np.array_equal(st, (order // m).astype(np.int32))


# ----------------------------------------------------------------------------- p-value

def test_q_matches_scipy_kolmogorov():
    lams = np.concatenate([np.linspace(0.05, 6.0, 4001), [1.18 - 1e-12, 1.18, 1.18 + 1e-12],
                           np.linspace(6.0, 18.5, 200)])
    for l in lams:
        q = oracle.kolmogorov_q(l)
        ref = float(scipy.special.kolmogorov(l))
        if ref < 1e-290:
            continue
        assert abs(q - ref) <= 1e-13 * ref + 1e-300, (l, q, ref)


def test_q_matches_50_digit_series():
    import mpmath
    mpmath.mp.dps = 50
    for l in [0.1, 0.3, 0.5, 0.8, 1.0, 1.1, 1.179999, 1.18, 1.2, 1.5, 2.0, 3.0, 5.0, 10.0, 13.0]:
        L = mpmath.mpf(l)
        ref = 2 * mpmath.nsum(lambda j: (-1) ** (j - 1) * mpmath.exp(-2 * j * j * L * L), [1, mpmath.inf])
        q = oracle.kolmogorov_q(l)
        assert abs(q - float(ref)) <= 2e-15 * float(ref) + 1e-300, (l, q, ref)


def test_textbook_quantiles():
    assert abs(oracle.kolmogorov_q(1.2238) - 0.10) < 1e-4
    assert abs(oracle.kolmogorov_q(1.3581) - 0.05) < 1e-4
    assert abs(oracle.kolmogorov_q(1.6276) - 0.01) < 1e-4


def test_q_limits():
    assert oracle.kolmogorov_q(0.0) == 1.0
    assert oracle.kolmogorov_q(-1.0) == 1.0
    assert oracle.kolmogorov_q(math.sqrt(345.0) * 1.0000001) == 0.0
    assert oracle.kolmogorov_q(18.0) > 0.0
    assert oracle.pvalue(0, 100, 20) == 1.0


def test_eq1_critical_value_consistency():
    """Eq. 1 (minus sign restored) inverts the first series term 2 exp(-2 lambda^2) = alpha."""
    for alpha in [0.1, 0.05, 0.01, 1e-3, 1e-6]:
        lam_a = math.sqrt(-0.5 * math.log(alpha / 2))
        # next-term size, plus rounding of lambda amplified by |d ln Q / d ln lambda| = 4 lambda^2
        assert abs(oracle.kolmogorov_q(lam_a) - alpha) <= 2.5 * math.exp(-8 * lam_a ** 2) + 4 * lam_a ** 2 * 4e-16 * alpha
        for n, m in [(10, 20), (128, 384), (1000, 1000)]:
            d = oracle.critical_value(alpha, n, m)
            assert abs(d * math.sqrt(n * m / (n + m)) - lam_a) < 1e-12


def test_lambda_definition():
    # lambda = sqrt(nL nR / N) D with D = num/den
    for nL, nR, num in [(32, 32, 100), (1280, 64000, 2 ** 30), (7, 9, 63)]:
        den = nL * nR
        N = nL + nR
        assert abs(oracle.lam(num, den, N) - math.sqrt(nL * nR / N) * num / den) < 1e-12 * oracle.lam(num, den, N)


def test_permutation_pvalue_sanity():
    """Loose: the asymptotic p and the exact permutation p of D agree in order of magnitude."""
    rng = np.random.default_rng(3)
    for _ in range(6):
        m = 4
        x = np.concatenate([rng.integers(0, 10, size=(2, m)), rng.integers(3, 13, size=(2, m))]).astype(np.uint32)
        pooled = list(x.ravel())
        D_obs = brute_D(pooled[:2 * m], pooled[2 * m:])
        n = len(pooled)
        ge = tot = 0
        for left in itertools.combinations(range(n), 2 * m):
            s = set(left)
            L = [pooled[i] for i in left]
            R = [pooled[i] for i in range(n) if i not in s]
            tot += 1
            ge += brute_D(L, R) >= D_obs
        p_perm = ge / tot
        nL = nR = 2 * m
        p_asym = oracle.pvalue(int(D_obs * nL * nR), nL * nR, nL + nR)
        assert p_asym >= 0.2 * p_perm and p_asym <= 5 * p_perm + 0.05


# ----------------------------------------------------------------------------- segmentation

def brute_segment(x2d, alpha, min_seg=1):
    T, m = x2d.shape
    out = []

    def rec(lo, hi):
        if hi - lo < 2 * min_seg:
            return
        k, D = brute_scan(x2d, lo, hi, min_seg)
        nL, nR = m * (k - lo), m * (hi - k)
        lam = math.sqrt(nL * nR / (nL + nR)) * float(D)
        p = float(scipy.special.kolmogorov(lam)) if lam > 0 else 1.0
        if abs(p - alpha) < 1e-9 * alpha:
            raise RuntimeError("borderline")
        if p <= alpha:
            rec(lo, k)
            out.append((k, D))
            rec(k, hi)

    rec(0, T)
    return out


def test_segmentation_against_brute_force(rng):
    checked = 0
    for _ in range(80):
        T = int(rng.integers(2, 14))
        m = int(rng.integers(1, 6))
        levels = np.sort(rng.integers(0, 40, size=3))
        cps = np.sort(rng.choice(np.arange(1, T), size=min(2, T - 1), replace=False))
        lvl = np.searchsorted(cps, np.arange(T), side="right")
        x = (levels[lvl][:, None] + rng.integers(0, 6, size=(T, m))).astype(np.uint32)
        alpha = float(rng.choice([0.5, 0.2, 0.05]))
        min_seg = int(rng.integers(1, 3))
        try:
            ref = brute_segment(x, alpha, min_seg)
        except RuntimeError:
            continue
        b = synth.from_arrays([x])
        rc, cnt, idx, num, den, p = oracle.ks_segment(b.samples, b.offsets, b.steps, alpha, min_seg, max_cp=16)
        assert rc == oracle.OK
        assert cnt[0] == len(ref)
        for c, (k, D) in enumerate(ref):
            assert idx[0, c] == k and Fraction(int(num[0, c]), int(den[0, c])) == D
        checked += 1
    assert checked > 60


def test_segmentation_capacity_reports_true_count():
    x = np.repeat(np.arange(0, 800, 100, dtype=np.uint32), 4).reshape(8, 4) * 0
    x = np.array([[10 * (t + 1)] * 16 for t in range(12)], np.uint32)  # 11 perfect steps
    b = synth.from_arrays([x])
    rc, cnt, idx, num, den, p = oracle.ks_segment(b.samples, b.offsets, b.steps, 0.05, 1, max_cp=4)
    rc_full, cnt_full, idx_full, *_ = oracle.ks_segment(b.samples, b.offsets, b.steps, 0.05, 1, max_cp=16)
    assert rc == oracle.ECAPACITY and cnt[0] == cnt_full[0] > 4
    assert np.array_equal(idx[0], idx_full[0, :4])


def test_single_series_64x32_recovers_truth():
    b = synth.generate(1, 0, 1)
    k, num, den, p = oracle.ks_scan(b.samples, b.offsets, b.steps)
    assert k[0] == 40 and p[0] == 0.0 and num[0] <= den[0] and num[0] / den[0] > 0.98


def test_three_level_truth_recovery_is_high():
    """Sanity statistic only: the exact segmentation finds the generator's change points."""
    b = synth.generate(2, 1, 8)
    rc, cnt, idx, *_ = oracle.ks_segment(b.samples, b.offsets, b.steps, 1e-6, nthreads=8)
    hits = sum(np.array_equal(idx[s, :cnt[s]], b.cps[s, :3]) for s in range(8))
    assert hits >= 7


def test_reduced_variant_equals_raw_for_m1(rng):
    """Eq. 2 with m = 1 is a strictly increasing map of each value, so KS gives the same split."""
    for _ in range(30):
        T = int(rng.integers(2, 40))
        x = rng.integers(0, 30, size=(T, 1)).astype(np.uint32)
        b = synth.from_arrays([x])
        r_raw = oracle.ks_scan(b.samples, b.offsets, b.steps)
        r_red = oracle.ks_scan(b.samples, b.offsets, b.steps, reduced=True)
        for a, c in zip(r_raw, r_red):
            assert np.array_equal(a, c)


def test_reduce_series_values():
    x = np.array([[3, 4, 5], [3, 3, 3], [10, 3, 7]], np.uint32)
    S = oracle.reduce_series(x)
    # min r = 3: sqrt(0+1+4), sqrt(0), sqrt(49+0+16)
    assert np.allclose(S, [math.sqrt(5), 0.0, math.sqrt(65)], rtol=0, atol=1e-15)


def test_reduce_series_pythagorean_closed_forms(rng):
    """Eq. 2 on steps whose offsets from the series minimum form Pythagorean quadruples and
    quintuples: the root is an exact integer, whatever the order of the FP64 sum (every partial
    sum is an integer below 2^53).  Reordering a step's samples and scaling every offset by an
    integer c (S scales by c exactly here) change nothing else."""
    quads = [(1, 2, 2, 3), (2, 3, 6, 7), (1, 4, 8, 9), (4, 4, 7, 9), (2, 6, 9, 11), (6, 6, 7, 11),
             (1, 12, 12, 17), (8, 9, 12, 17), (12, 16, 21, 29), (1, 2, 4, 10, 11)]
    base = 1000
    for c in (1, 7, 4096):
        rows, want = [], []
        for q in quads:
            *parts, root = q
            row = [base] + [base + c * v for v in parts]
            row += [base] * (5 - len(row))
            rows.append(row)
            want.append(c * root)
        x = np.array(rows, np.uint32)
        S = oracle.reduce_series(x)
        assert [float(v) for v in S] == [float(w) for w in want]
        xp = np.array([rng.permutation(r) for r in rows], np.uint32)
        assert np.array_equal(oracle.reduce_series(xp), S)


def test_single_series_64x32_golden_fixture():
    """The stored fixture (written by tests/golden/make_golden.py from the oracle) still holds."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "single_series_64x32_oracle.json")))
    b = synth.generate(1, 0, 1)
    assert int(b.samples.astype(np.uint64).sum()) == g["samples_sum"]
    k, num, den, p = oracle.ks_scan(b.samples, b.offsets, b.steps)
    assert (int(k[0]), int(num[0]), int(den[0]), float(p[0])) == \
        (g["scan"]["k"], g["scan"]["num"], g["scan"]["den"], g["scan"]["p"])


# ------------------------------------------------------------------ latency statistics (Sec. IV-C)

def test_latency_stats_against_numpy(rng):
    series = [rng.integers(1, 5000, size=(int(rng.integers(2, 40)), int(rng.integers(1, 30))), dtype=np.uint32)
              for _ in range(30)]
    b = synth.from_arrays(series)
    mean, p50, p95, std = oracle.latency_stats(b.samples, b.offsets, b.steps)
    for s, x in enumerate(series):
        v = x.ravel().astype(np.float64)
        assert p50[s] == np.percentile(x.ravel(), 50, method="inverted_cdf")
        assert p95[s] == np.percentile(x.ravel(), 95, method="inverted_cdf")
        assert abs(mean[s] - v.mean()) <= 1e-15 * v.mean()
        assert abs(std[s] - v.std()) <= 1e-12 * max(v.std(), 1.0)


def test_latency_stats_closed_forms():
    big = np.full((4, 8), 2**32 - 1, np.uint32)            # naive FP64 sums of squares would not cancel
    two = np.array([[7] * 6, [19] * 6], np.uint32)          # half 7, half 19
    one = np.array([[5], [5]], np.uint32)
    b = synth.from_arrays([big, two, one])
    mean, p50, p95, std = oracle.latency_stats(b.samples, b.offsets, b.steps)
    assert mean[0] == float(2**32 - 1) and std[0] == 0.0 and p50[0] == p95[0] == 2**32 - 1
    assert mean[1] == 13.0 and std[1] == 6.0 and p50[1] == 7 and p95[1] == 19
    assert mean[2] == 5.0 and std[2] == 0.0 and p50[2] == p95[2] == 5
