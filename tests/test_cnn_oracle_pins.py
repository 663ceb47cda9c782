"""Pins for the learned-proposal oracle (oracle/cnn_oracle.py), independent of its own code.

- convolution: scipy.signal.correlate of each input/output channel pair;
- gradients: fp64 central finite differences of the loss (bf16 rounding off);
- Adam: hand-computed update of a 3-parameter case (Kingma & Ba, Algorithm 1);
- bf16 rounding: exact bit patterns for values at, below and above a rounding tie;
- summaries: quantile ranks against explicit sorting, and the fixed step-size channel.
"""
import math

import numpy as np
import scipy.signal

from oracle import cnn_oracle as C


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    for cin, cout, T in [(17, 32, 40), (32, 1, 9), (3, 2, 5)]:
        x = rng.normal(size=(cin, T))
        W = rng.normal(size=(cout, cin, 5))
        b = rng.normal(size=cout)
        y = C.conv1d(x, W, b)
        ref = np.zeros((cout, T))
        for o in range(cout):
            ref[o] = b[o]
            for i in range(cin):
                ref[o] += scipy.signal.correlate(x[i], W[o, i], mode="same")
        assert np.allclose(y, ref, rtol=1e-12, atol=1e-10)


def test_param_count_of_the_stated_structure():
    # 17->32->32->32->1, width 5: 17*32*5+32 + 2*(32*32*5+32) + 32*5+1
    assert C.n_params() == 2752 + 2 * 5152 + 161 == 13217


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = [(W.astype(np.float64), b.astype(np.float64) + rng.normal(size=b.shape) * 0.1)
              for W, b in C.init_params(rng)]
    T = 12
    xs = [rng.normal(size=(17, T)) for _ in range(3)]
    cps = [[3, 8], [], [5]]
    loss, grads = C.loss_and_grads(params, xs, cps, round_bf16=False)
    eps = 1e-6
    for li in range(4):
        for which in (0, 1):
            arr = params[li][which]
            flat_idx = rng.choice(arr.size, size=min(6, arr.size), replace=False)
            for fi in flat_idx:
                idx = np.unravel_index(fi, arr.shape)
                old = arr[idx]
                arr[idx] = old + eps
                lp, _ = C.loss_and_grads(params, xs, cps, round_bf16=False)
                arr[idx] = old - eps
                lm, _ = C.loss_and_grads(params, xs, cps, round_bf16=False)
                arr[idx] = old
                fd = (lp - lm) / (2 * eps)
                g = grads[li][which][idx]
                assert abs(fd - g) <= 1e-5 * max(1.0, abs(fd)), (li, which, idx, fd, g)


def test_adam_three_parameters_by_hand():
    p = [(np.array([1.0, -2.0]), np.array([0.5]))]
    g = [(np.array([0.1, -0.3]), np.array([2.0]))]
    m, v = {}, {}
    out = C.adam_step(p, g, m, v, step=1, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8)
    # step 1: m_hat = g, v_hat = g^2, update = lr * g / (|g| + eps) ~ lr * sign(g)
    expect_W = np.array([1.0 - 1e-3 * 0.1 / (0.1 + 1e-8), -2.0 + 1e-3 * 0.3 / (0.3 + 1e-8)])
    expect_b = np.array([0.5 - 1e-3 * 2.0 / (2.0 + 1e-8)])
    assert np.allclose(out[0][0], expect_W, rtol=0, atol=1e-15)
    assert np.allclose(out[0][1], expect_b, rtol=0, atol=1e-15)
    # step 2 with a new gradient: m = .9 m + .1 g, v = .999 v + .001 g^2, bias-corrected
    g2 = [(np.array([0.2, 0.0]), np.array([-1.0]))]
    out2 = C.adam_step(out, g2, m, v, step=2, lr=1e-3)
    m2 = 0.9 * 0.1 * 0.1 + 0.1 * 0.2
    v2 = 0.999 * 0.001 * 0.01 + 0.001 * 0.04
    upd = 1e-3 * (m2 / (1 - 0.81)) / (math.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    assert abs(out2[0][0][0] - (expect_W[0] - upd)) < 1e-15


def test_bf16_rounding_bit_patterns():
    one = np.float32(1.0)
    ulp = 2.0 ** -7  # bf16 spacing at 1
    assert C.bf16(np.array([1.0]))[0] == 1.0
    assert C.bf16(np.array([1.0 + ulp / 2]))[0] == 1.0          # tie -> even (1.0)
    assert C.bf16(np.array([1.0 + 1.5 * ulp]))[0] == 1.0 + 2 * ulp  # tie -> even (1+2ulp)
    assert C.bf16(np.array([1.0 + 0.6 * ulp]))[0] == 1.0 + ulp
    assert C.bf16(np.array([-3.0]))[0] == -3.0
    assert one == 1.0


def test_summaries_definition():
    rng = np.random.default_rng(2)
    T, m = 7, 12
    x = rng.integers(1, 500, size=(T, m)).astype(np.uint32)
    f = C.summaries(x)
    med = np.sort(x.ravel())[(T * m) // 2]
    for t in range(T):
        s = np.sort(x[t])
        for i in range(16):
            r = min(m - 1, int(math.floor((i + 0.5) * m / 16)))
            assert abs(f[i, t] - (math.log2(s[r]) - math.log2(med))) < 1e-12
        assert abs(f[16, t] - (math.log2(1024 + 32 * t) - 10)) < 1e-12


def test_propose_windows_and_mass():
    z = np.full(100, -5.0)
    z[[10, 11, 50, 90]] = [3.0, 2.9, 2.0, 1.0]
    centres, conf = C.propose(z, 3, 16)
    assert centres == [10, 50, 90]  # 11 is suppressed by the window around 10
    p = np.exp(z - z.max())
    p /= p.sum()
    covered = np.zeros(100, bool)
    for c in centres:
        covered[max(0, c - 16):c + 17] = True
    assert abs(conf - p[covered].sum()) < 1e-12
