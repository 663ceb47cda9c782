"""GPU parity of the learned-proposal kernels against the numpy oracle (oracle/cnn_oracle.py).

Features are BF16 on both sides (at most one BF16 step apart where FP32 and FP64 logarithms
round differently); logits and gradients are compared with a relative L2 tolerance of 1e-3 per
tensor, from the same BF16 weights and features.
"""
import numpy as np
import pytest

import paper_2511_05958_b300 as mt4g
import synth
from oracle import cnn_oracle as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    assert torch.cuda.is_available()
    e = mt4g.Engine(0)
    yield e
    e.close()


def bf16_bits_to_float(t):
    a = t.cpu().numpy().astype(np.int32) & 0xFFFF
    return (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def split_features(feat, steps):
    """GPU feature rows -> list of [17, T] arrays."""
    out, r = [], 0
    for T in steps:
        out.append(feat[r + 2:r + 2 + T, :17].T.copy())
        r += T + 4
    return out


def flat_to_layers(w):
    """Flat [d][i][o] weights -> oracle layers [(W[o][i][d], b)], dropping input channel 17."""
    layers, off = [], 0
    for cin_pad, cin, cout in [(18, 17, 32), (32, 32, 32), (32, 32, 32), (32, 32, 1)]:
        n = 5 * cin_pad * cout
        W = w[off:off + n].reshape(5, cin_pad, cout)[:, :cin, :].transpose(2, 1, 0).astype(np.float64)
        off += n
        b = w[off:off + cout].astype(np.float64)
        off += cout
        layers.append((W, b))
    assert off == mt4g.CNN_PARAMS
    return layers


def layers_to_flat(grads):
    parts = []
    for (gW, gb), cin_pad in zip(grads, [18, 32, 32, 32]):
        cout, cin, _ = gW.shape
        full = np.zeros((5, cin_pad, cout))
        full[:, :cin, :] = gW.transpose(2, 1, 0)
        parts += [full.ravel(), gb.ravel()]
    return np.concatenate(parts)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_summaries_match_oracle(eng):
    rng = np.random.default_rng(0)
    series = [synth.generate(2, 5, 2).series(1)]
    for m in (1, 8, 16, 32, 33, 64, 100, 128, 256):
        T = int(rng.integers(2, 80))
        series.append(rng.integers(1, 3000, size=(T, m)).astype(np.uint32))
    # m = 32, 64, 128 sort one step per thread: several groups of 32 steps per warp, a ragged
    # last group, and rows that start off a 16-byte boundary (after a series of 3 samples)
    series.append(rng.integers(0, 1 << 32, size=(3, 1), dtype=np.uint64).astype(np.uint32))
    for m, T in ((128, 300), (64, 161), (32, 97)):
        v = rng.integers(0, 1 << 32, size=(T, m), dtype=np.uint64).astype(np.uint32)
        v[::7] = rng.integers(0, 4, size=(len(v[::7]), m))  # ties and zeros (read as 1)
        series.append(v)
    series.append(np.zeros((5, 4), np.uint32))  # values read as 1
    b = synth.from_arrays(series)
    feat = eng.summaries(mt4g.to_device_samples(b.samples), b.offsets, b.steps)
    got = bf16_bits_to_float(feat)
    # pad rows are zero
    r = 0
    for T in b.steps:
        assert (got[r:r + 2] == 0).all() and (got[r + T + 2:r + T + 4] == 0).all()
        assert (got[r + 2:r + 2 + T, 17] == 0).all()
        r += T + 4
    # The kernel evaluates log2(q) - log2(med) in FP32: each logarithm is at most 32 (samples are
    # 32-bit), so the difference carries an absolute error of a few FP32 steps at 32 (2^-18 each)
    # before its BF16 rounding; where q is close to the median the difference is tiny and that
    # absolute error dominates.  Bound: one BF16 step relative, plus 2^-16 absolute.
    for x, g in zip(series, split_features(got, b.steps)):
        ref = C.bf16(C.summaries(x))
        ulp = np.abs(ref) * 2.0 ** -7 + 2.0 ** -16
        assert (np.abs(g - ref) <= ulp).all(), np.max(np.abs(g - ref) - ulp)
        assert np.mean(g == ref) > 0.99


def _batch(eng, S=6, seed=3):
    b = synth.generate(2, seed, S)
    feat = eng.summaries(mt4g.to_device_samples(b.samples), b.offsets, b.steps)
    return b, feat


def test_forward_matches_oracle(eng):
    b, feat = _batch(eng)
    eng.cnn_init(7)
    w = eng.cnn_get_params()
    logits = eng.cnn_forward(feat, b.steps).cpu().numpy()
    params = flat_to_layers(w)
    xs = split_features(bf16_bits_to_float(feat), b.steps)
    r = 0
    for x, T in zip(xs, b.steps):
        z, _ = C.forward(params, x, round_bf16=True)
        g = logits[r + 2:r + 2 + T]
        assert rel_l2(g, z) < 1e-3
        r += T + 4


def test_forward_ragged_tiles_match_oracle(eng):
    """Inference runs tiles of 116 logits: series shorter than, equal to and one longer than a
    tile, several tiles with a ragged last one, and enough tiles that each CTA takes a run of
    consecutive tiles across series.  Pad rows hold non-zero values, which the zero padding of
    the convolutions must ignore."""
    import torch
    rng = np.random.default_rng(12)
    steps = [2, 3, 5, 115, 116, 117, 231, 232, 233, 600] + [int(t) for t in rng.integers(100, 400, size=300)]
    rows = sum(T + 4 for T in steps)
    f = rng.uniform(-3, 3, size=(rows, 18)).astype(np.float32)
    bits = (f.view(np.uint32) >> 16).astype(np.uint16)  # BF16 truncations, exact in both
    bits[:, 17] = 0
    feat = torch.from_numpy(bits.view(np.int16)).cuda()
    eng.cnn_init(21)
    w = eng.cnn_get_params()
    for off, n in ((2880, 32), (2880 + 32 + 5120, 32), (2880 + 2 * 5152, 32)):
        w[off:off + n] = rng.normal(size=n) * 0.2
    w[-1] = 0.3
    eng.cnn_set_params(w)
    logits = eng.cnn_forward(feat, np.asarray(steps, np.int32)).cpu().numpy()
    params = flat_to_layers(eng.cnn_get_params())
    xs = split_features(bits_to_float(bits), steps)
    r = 0
    for x, T in zip(xs, steps):
        z, _ = C.forward(params, x, round_bf16=True)
        g = logits[r + 2:r + 2 + T].astype(np.float64)
        assert rel_l2(g, z) < 1e-3, T
        r += T + 4


def bits_to_float(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def test_gradients_match_oracle(eng):
    import torch
    rng = np.random.default_rng(4)
    b, feat = _batch(eng, S=8, seed=6)
    eng.cnn_init(11)
    w = eng.cnn_get_params()
    # give biases non-zero values so every path is exercised
    w[2880:2912] = rng.normal(size=32) * 0.1
    eng.cnn_set_params(w)
    max_cp = 4
    cps = [list(b.cps[s, :3]) for s in range(8)]
    cps[2] = []          # a series without a target is masked out
    cps[5] = [7]
    cnt = torch.tensor([len(c) for c in cps], dtype=torch.int32, device="cuda")
    idx = torch.tensor([c + [-1] * (max_cp - len(c)) for c in cps], dtype=torch.int32, device="cuda")
    grad, loss = eng.cnn_grads(feat, 512, 8, cnt, idx)
    grad = grad.cpu().numpy().astype(np.float64)
    params = flat_to_layers(w)
    xs = split_features(bf16_bits_to_float(feat), b.steps)
    ref_loss, ref_grads = C.loss_and_grads(params, xs, cps, round_bf16=True)
    assert abs(float(loss.item()) - ref_loss) <= 1e-3 * abs(ref_loss)
    ref = layers_to_flat(ref_grads)
    off = 0
    errs = []
    for cin_pad, cout in [(18, 32), (32, 32), (32, 32), (32, 1)]:
        n = 5 * cin_pad * cout
        errs.append(rel_l2(grad[off:off + n], ref[off:off + n]))
        off += n
        if cout > 1:
            errs.append(rel_l2(grad[off:off + cout], ref[off:off + cout]))
        else:
            # the output bias gets sum_t (p_t - y_t) = 0 exactly: check it is zero to rounding
            assert abs(grad[off]) < 1e-5 and abs(ref[off]) < 1e-12
        off += cout
    assert max(errs) < 1e-3, errs
    # the zero input channel gets no gradient
    assert (grad[:2880].reshape(5, 18, 32)[:, 17, :] == 0).all()


def test_adam_step_and_checkpoint_roundtrip(eng, tmp_path):
    import torch
    b, feat = _batch(eng, S=4, seed=8)
    eng.cnn_init(5)
    w0 = eng.cnn_get_params().astype(np.float64)
    cnt = torch.tensor([3, 3, 3, 3], dtype=torch.int32, device="cuda")
    idx = torch.tensor(b.cps[:, :3], dtype=torch.int32, device="cuda").contiguous()
    g, _ = eng.cnn_grads(feat, 512, 4, cnt, idx)
    g = g.cpu().numpy().astype(np.float64)
    eng.cnn_train_step(feat, 512, 4, cnt, idx, lr=1e-3)
    w1 = eng.cnn_get_params().astype(np.float64)
    m, v = {}, {}
    exp = C.adam_step([(w0, np.zeros(1))], [(g, np.zeros(1))], m, v, step=1)[0][0]
    assert np.allclose(w1, exp, rtol=1e-5, atol=1e-7)
    path = str(tmp_path / "w.bin")
    eng.cnn_save(path)
    eng.cnn_init(99)
    eng.cnn_load(path)
    assert np.array_equal(eng.cnn_get_params().astype(np.float64), w1)
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    with pytest.raises(mt4g.Mt4gError) as e:
        eng.cnn_load(path)
    assert e.value.code == mt4g.EINVAL


def test_propose_matches_oracle_windows(eng):
    b, feat = _batch(eng, S=16, seed=9)
    eng.cnn_init(3)
    d = mt4g.to_device_samples(b.samples)
    win, conf = eng.propose(d, b.offsets, b.steps, 3, 16)
    logits = eng.cnn_forward(feat, b.steps).cpu().numpy()
    win = win.cpu().numpy()
    conf = conf.cpu().numpy()
    r = 0
    for s, T in enumerate(b.steps):
        z = logits[r + 2:r + 2 + T].astype(np.float64)
        centres, c = C.propose(z, 3, 16)
        assert list(win[s]) == centres
        assert abs(conf[s] - c) < 1e-4
        r += T + 4


def test_training_reduces_loss(eng):
    """A few hundred steps on one batch overfit it: the loss must drop."""
    import torch
    b, feat = _batch(eng, S=32, seed=12)
    eng.cnn_init(1)
    cnt = torch.full((32,), 3, dtype=torch.int32, device="cuda")
    idx = torch.tensor(b.cps[:, :3], dtype=torch.int32, device="cuda").contiguous()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    _, l0 = eng.cnn_grads(feat, 512, 32, cnt, idx)
    for _ in range(300):
        eng.cnn_train_step(feat, 512, 32, cnt, idx, lr=3e-3, loss=loss)
    _, l1 = eng.cnn_grads(feat, 512, 32, cnt, idx)
    assert float(l1.item()) < 0.5 * float(l0.item())


# ------------------------------------------------------------------ exact learned segmentation

def _segment(eng, b, mode, alpha=1e-6, min_seg=1, max_cp=16):
    r = eng.ks_segment(mt4g.to_device_samples(b.samples), b.offsets, b.steps, alpha, min_seg, max_cp, mode=mode)
    return r.rc, [t.cpu().numpy() for t in r[1:7]]


def _assert_same(full, learned):
    rc_f, (cf, idf, nf, df, pf, fbf) = full
    rc_l, (cl, idl, nl, dl, pl, fbl) = learned
    assert rc_f == rc_l
    assert np.array_equal(cf, cl)
    assert np.array_equal(idf, idl)
    assert np.array_equal(nf, nl)
    assert np.array_equal(df, dl)
    assert np.array_equal(pf, pl)  # identical splits give identical FP64 p-values
    assert (fbf == 0).all()


@pytest.mark.parametrize("seed", [0, 1])
def test_learned_mode_equals_full_on_three_level_series(eng, seed):
    import oracle
    b = synth.generate(2, 20 + seed, 256)
    eng.cnn_init(100 + seed)  # untrained: windows are often wrong, certification must catch it
    eng.set_option(mt4g.OPT_CONF_MIN_PPM, 0)  # every series takes the learned path
    eng.set_option(mt4g.OPT_SCAN_KPT, 1)  # slices: the probes run (the run sweep would take these)
    try:
        full = _segment(eng, b, mt4g.MODE_FULL)
        learned = _segment(eng, b, mt4g.MODE_LEARNED)
        stats = eng.learned_stats()
    finally:
        eng.set_option(mt4g.OPT_CONF_MIN_PPM, 900000)
        eng.set_option(mt4g.OPT_SCAN_KPT, 0)
    _assert_same(full, learned)
    assert (learned[1][5] == 0).all()  # no fallback at threshold 0
    assert stats["probe_groups"] > 256 and stats["certified"] + stats["refined"] == stats["probe_groups"]
    # and the oracle agrees on a sample
    sample = np.arange(0, 256, 16)
    sb = synth.from_arrays([b.series(s) for s in sample])
    orc, ocnt, oidx, onum, oden, op = oracle.ks_segment(sb.samples, sb.offsets, sb.steps, 1e-6, 1, 16, nthreads=8)
    assert np.array_equal(learned[1][0][sample], ocnt) and np.array_equal(learned[1][1][sample], oidx)
    assert np.array_equal(learned[1][2][sample], onum) and np.array_equal(learned[1][3][sample], oden)
    assert (np.abs(learned[1][4][sample] - op) <= 1e-12 * np.abs(op)).all()


@pytest.mark.parametrize("mixed", [False, True])
def test_learned_queue_launch_gate(eng, mixed):
    """A learned call launches the plain and the learned queue instantiation; the sort's count of
    series the sweep does not take decides which one works.  All swept (three-level series, at
    most 1536 distinct values): the plain kernel, every series falls back to the full scan.
    Mixed (plus series with thousands of distinct values): the learned kernel.  Either way the
    answers are the oracle's and the plain call's."""
    import oracle
    rng = np.random.default_rng(77)
    b0 = synth.generate(2, 41, 48)
    series = [b0.series(s) for s in range(48)]
    if mixed:
        for _ in range(8):  # thousands of distinct values: the run sweep does not take them
            T = int(rng.integers(40, 120))
            lev = rng.integers(1000, 40000, size=(T, 1))
            lev[T // 2:] += 5000
            series.append((lev + rng.integers(0, 60000, size=(T, 64))).astype(np.uint32))
    b = synth.from_arrays(series)
    eng.cnn_init(5)
    full = _segment(eng, b, mt4g.MODE_FULL)
    learned = _segment(eng, b, mt4g.MODE_LEARNED)
    unswept = eng.last_sweep()["unswept_series"]
    assert (unswept > 0) == mixed
    if not mixed:
        assert (learned[1][5] == 1).all()  # every series swept: the full scan, by the plain kernel
    rc_f, (cf, idf, nf, df, pf, _) = full
    rc_l, (cl, idl, nl, dl, pl, _) = learned
    assert rc_f == rc_l
    for a, c in ((cf, cl), (idf, idl), (nf, nl), (df, dl), (pf, pl)):
        assert np.array_equal(a, c)
    _, ocnt, oidx, onum, oden, op = oracle.ks_segment(b.samples, b.offsets, b.steps, 1e-6, 1, 16, nthreads=8)
    assert np.array_equal(cl, ocnt) and np.array_equal(idl, oidx)
    assert np.array_equal(nl, onum) and np.array_equal(dl, oden)
    assert (np.abs(pl - op) <= 1e-12 * np.abs(op)).all()


def test_learned_mode_fallback_threshold(eng):
    b = synth.generate(2, 31, 64)
    eng.cnn_init(7)
    full = _segment(eng, b, mt4g.MODE_FULL)
    eng.set_option(mt4g.OPT_CONF_MIN_PPM, 1000001)  # nobody is confident enough
    try:
        rc, res = _segment(eng, b, mt4g.MODE_LEARNED)
    finally:
        eng.set_option(mt4g.OPT_CONF_MIN_PPM, 900000)
    assert (res[5] == 1).all()
    _assert_same(full, (rc, res[:5] + [np.zeros_like(res[5])]))


def test_learned_mode_random_shapes_and_min_seg(eng):
    rng = np.random.default_rng(17)
    series = []
    for _ in range(120):
        T = int(rng.integers(2, 400))
        m = int(rng.integers(1, 200))
        x = rng.integers(0, int(rng.integers(2, 400)), size=(T, m))
        for _c in range(int(rng.integers(0, 4))):
            x[int(rng.integers(0, T)):] += int(rng.integers(0, 100))
        series.append(x.astype(np.uint32))
    b = synth.from_arrays(series)
    eng.cnn_init(5)
    eng.set_option(mt4g.OPT_CONF_MIN_PPM, 0)
    try:
        for tile in (1, 0):  # probes on slices; then the default, where the run sweep takes most
            eng.set_option(mt4g.OPT_SCAN_KPT, tile)
            for alpha, min_seg in [(1e-6, 1), (1e-2, 3), (0.3, 1)]:
                full = _segment(eng, b, mt4g.MODE_FULL, alpha, min_seg)
                rc, res = _segment(eng, b, mt4g.MODE_LEARNED, alpha, min_seg)
                if tile == 0:
                    assert res[5].any()  # series the sweep takes are scanned in full
                _assert_same(full, (rc, res[:5] + [np.zeros_like(res[5])]))
    finally:
        eng.set_option(mt4g.OPT_CONF_MIN_PPM, 900000)
        eng.set_option(mt4g.OPT_SCAN_KPT, 0)


def test_learned_mode_uneven_sample(eng):
    b3 = synth.generate(3, 2, 400)
    keep = [s for s in range(400) if b3.m[s] <= 256 and float(b3.steps[s]) ** 2 * float(b3.m[s]) < 4e8][:120]
    b = synth.from_arrays([b3.series(s) for s in keep])
    eng.cnn_init(9)
    eng.set_option(mt4g.OPT_CONF_MIN_PPM, 0)
    try:
        for tile in (1, mt4g.SCAN_SWEEP):
            eng.set_option(mt4g.OPT_SCAN_KPT, tile)
            full = _segment(eng, b, mt4g.MODE_FULL)
            rc, res = _segment(eng, b, mt4g.MODE_LEARNED)
            _assert_same(full, (rc, res[:5] + [np.zeros_like(res[5])]))
    finally:
        eng.set_option(mt4g.OPT_CONF_MIN_PPM, 900000)
        eng.set_option(mt4g.OPT_SCAN_KPT, 0)


def test_learned_mode_needs_weights():
    import torch
    e = mt4g.Engine(0)
    b = synth.generate(1, 0, 1)
    with pytest.raises(mt4g.Mt4gError) as err:
        e.ks_segment(mt4g.to_device_samples(b.samples), b.offsets, b.steps, 1e-6, mode=mt4g.MODE_LEARNED)
    assert err.value.code == mt4g.EINVAL
    e.close()
    torch.cuda.synchronize()


def test_trained_network_gains_over_untrained():
    """What training buys: on held-out series of the training distribution, the trained weights
    put the true change points inside their windows and are confident, so the learned path
    evaluates fewer (split, value) pairs than with untrained weights.  Answers are identical
    either way (certification is exact)."""
    import os
    weights = os.path.join(os.path.dirname(mt4g.__file__), "weights", "cnn_c2.bin")
    b = synth.generate(2, 4, 512)
    d = mt4g.to_device_samples(b.samples)
    e = mt4g.Engine(0)
    e.set_option(mt4g.OPT_SCAN_KPT, 1)  # slices everywhere: the probes run (no run sweep)
    try:
        full = e.ks_segment(d, b.offsets, b.steps, 1e-6, 1, 16, mode=mt4g.MODE_FULL)
        full = [t.cpu().numpy() for t in full[1:6]]
        assert e.wait() == mt4g.OK
        evals_full = e.last_work()
        e.set_option(mt4g.OPT_CONF_MIN_PPM, 0)  # both networks take the learned path everywhere
        out = {}
        for name in ("trained", "untrained"):
            if name == "trained":
                e.cnn_load(weights)
            else:
                e.cnn_init(2024)
            win, conf = e.propose(d, b.offsets, b.steps, 3, 16)
            win = win.cpu().numpy()
            covered = np.mean([all(any(abs(int(c) - int(w)) <= 16 for w in win[s] if w >= 0)
                                   for c in b.cps[s, :b.ncp[s]]) for s in range(512)])
            r = e.ks_segment(d, b.offsets, b.steps, 1e-6, 1, 16, mode=mt4g.MODE_LEARNED)
            res = [t.cpu().numpy() for t in r[1:6]]
            assert e.wait() == mt4g.OK
            for a, c in zip(full, res):
                assert np.array_equal(a, c)
            out[name] = {"covered": covered, "conf": float(conf.float().mean().item()),
                         "evals": e.last_work(), "stats": e.learned_stats()}
    finally:
        e.close()
    tr, un = out["trained"], out["untrained"]
    msg = (out, evals_full)
    assert tr["covered"] >= 0.95 and un["covered"] < 0.5, msg
    assert tr["conf"] >= 0.9 > un["conf"], msg
    assert tr["evals"] < un["evals"] < evals_full * 1.5, msg


def test_training_checkpoint_and_resume(tmp_path):
    """train.py writes the weights and Adam state every N steps and continues from them."""
    import json
    import os
    from paper_2511_05958_b300 import train
    out = str(tmp_path / "w.bin")
    common = ["--series", "256", "--chunk", "128", "--batch", "32", "--eval-series", "64", "--out", out]
    train.main(common + ["--steps", "20", "--checkpoint-every", "10"])
    assert os.path.exists(out + ".ckpt") and json.load(open(out + ".ckpt.json"))["step"] == 20
    e = mt4g.Engine(0)
    e.cnn_load(out + ".ckpt")
    w20 = e.cnn_get_params()
    e.close()
    train.main(common + ["--steps", "30", "--checkpoint-every", "10", "--resume"])
    log = json.load(open(os.path.splitext(out)[0] + ".train.json"))
    assert log["resumed_at_step"] == 20 and log["loss_curve"][-1]["step"] == 30
    e = mt4g.Engine(0)
    e.cnn_load(out)
    w30 = e.cnn_get_params()
    e.close()
    assert np.isfinite(w30).all() and not np.array_equal(w20, w30)
    assert json.load(open(out + ".ckpt.json"))["step"] == 30


@pytest.mark.parametrize("trained", [True, False])
def test_window_only_scan_matches_its_oracle(eng, trained):
    """MT4G_OPT_LEARNED_WINDOWS: swept series scanned only at their window splits, against the
    plain restatement of that procedure (oracle/windows_oracle.py) given the same windows and
    confidences: change points and D bit-exact, p within 1e-12, the same fallback flags.
    Untrained weights give poor windows: more fallbacks and answers that differ from the full
    scan, which the procedure must still reproduce exactly."""
    import os
    from oracle import windows_oracle as W
    b = synth.generate(2, 21, 40)
    d = mt4g.to_device_samples(b.samples)
    if trained:
        eng.cnn_load(os.path.join(os.path.dirname(mt4g.__file__), "weights", "cnn_c2.bin"))
    else:
        eng.cnn_init(5)
    win, conf = eng.propose(d, b.offsets, b.steps, 3, 16)
    win, conf = win.cpu().numpy(), conf.cpu().numpy()
    eng.set_option(mt4g.OPT_LEARNED_WINDOWS, 1)
    try:
        r = eng.ks_segment(d, b.offsets, b.steps, 1e-6, 1, 16, mode=mt4g.MODE_LEARNED)
    finally:
        eng.set_option(mt4g.OPT_LEARNED_WINDOWS, 0)
    cnt, idx, num, den, p, fb = [t.cpu().numpy() for t in r[1:7]]
    for s in range(len(b.steps)):
        low = bool(conf[s] < np.float32(0.9))  # the threshold as the library holds it (FP32)
        c, cps, f = W.segment_series(b.series(s), 1e-6, 1, 16, [int(c) for c in win[s]], 16, low)
        assert (int(cnt[s]), int(fb[s])) == (c, f), s
        for j, (k, n, dd, pp) in enumerate(cps):
            assert (int(idx[s, j]), int(num[s, j]), int(den[s, j])) == (k, n, dd), (s, j)
            assert abs(p[s, j] - pp) <= 1e-12 * max(pp, 1e-300), (s, j)


def test_window_only_ragged_shapes_and_min_seg(eng):
    """Window-only scans on series whose rows are not 8-byte aligned (m not a multiple of 4: the
    scalar load path), several T, and min_seg = 3, against oracle/windows_oracle.py."""
    from oracle import windows_oracle as W
    rng = np.random.default_rng(31)
    series = []
    for T, m in ((40, 6), (97, 12), (130, 40), (64, 5), (200, 24), (33, 7)):
        lv = rng.choice([30, 80, 200], size=3)
        cp = sorted(rng.choice(np.arange(5, T - 5), size=2, replace=False))
        x = np.empty((T, m), np.uint32)
        for a, bnd, l in zip([0, cp[0], cp[1]], [cp[0], cp[1], T], lv):
            x[a:bnd] = rng.poisson(l, size=(bnd - a, m))
        series.append(x)
    b = synth.from_arrays(series)
    d = mt4g.to_device_samples(b.samples)
    eng.cnn_init(9)
    win, conf = eng.propose(d, b.offsets, b.steps, 3, 6)
    win, conf = win.cpu().numpy(), conf.cpu().numpy()
    eng.set_option(mt4g.OPT_LEARNED_WINDOWS, 1)
    eng.set_option(mt4g.OPT_HALF_WIDTH, 6)
    eng.set_option(mt4g.OPT_CONF_MIN_PPM, 0)  # every series takes its windows
    try:
        r = eng.ks_segment(d, b.offsets, b.steps, 1e-6, 3, 16, mode=mt4g.MODE_LEARNED)
    finally:
        eng.set_option(mt4g.OPT_LEARNED_WINDOWS, 0)
        eng.set_option(mt4g.OPT_HALF_WIDTH, 16)
        eng.set_option(mt4g.OPT_CONF_MIN_PPM, 900000)
    cnt, idx, num, den, p, fb = [t.cpu().numpy() for t in r[1:7]]
    for s_, x in enumerate(series):
        c, cps, f = W.segment_series(x, 1e-6, 3, 16, [int(c_) for c_ in win[s_]], 6, False)
        assert (int(cnt[s_]), int(fb[s_])) == (c, f), s_
        for j, (k, n, dd, pp) in enumerate(cps):
            assert (int(idx[s_, j]), int(num[s_, j]), int(den[s_, j])) == (k, n, dd), (s_, j)
            assert abs(p[s_, j] - pp) <= 1e-12 * max(pp, 1e-300), (s_, j)

