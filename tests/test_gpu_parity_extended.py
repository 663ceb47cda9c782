"""GPU parity against the oracle on the cases the batch tests only sample or compare among GPU paths.

- The critical value of Eq. 1 beside every reported change point, for the sample sizes of the
  split that created it (the parent segment comes from replaying the binary segmentation with the
  oracle's own segment scan).
- The run sweep at its cap: series with 1535, 1536 and 1537 distinct values, and series whose
  upper segments are too wide for it.
- Full-shape series of the heavy (T, m) buckets of the uneven workload (T up to 4096, m = 256),
  which the batch test leaves to structural checks.

k, num and den bit-identical; p within 1e-12 relative; critical values within 1e-15 relative.
"""
import numpy as np
import pytest

import oracle
import paper_2511_05958_b300 as mt4g
import synth

pytestmark = pytest.mark.gpu

P_RTOL = 1e-12


@pytest.fixture(scope="module")
def eng():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    e = mt4g.Engine(0)
    yield e
    e.close()


def _close(a, b, rtol):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return bool((np.abs(a - b) <= rtol * np.abs(b)).all())


def _check_segment(eng, b, alpha, min_seg=1, max_cp=16, mode=mt4g.MODE_FULL, nthreads=8):
    r = eng.ks_segment(mt4g.to_device_samples(b.samples), b.offsets, b.steps, alpha, min_seg, max_cp, mode=mode)
    cnt, idx, num, den, p = (t.cpu().numpy() for t in r[1:6])
    orc, ocnt, oidx, onum, oden, op = oracle.ks_segment(b.samples, b.offsets, b.steps, alpha, min_seg, max_cp,
                                                        reduced=mode == mt4g.MODE_REDUCED, nthreads=nthreads)
    assert (r.rc == mt4g.ECAPACITY) == (orc == oracle.ECAPACITY)
    assert np.array_equal(cnt, ocnt), np.nonzero(cnt != ocnt)
    assert np.array_equal(idx, oidx)
    assert np.array_equal(num, onum)
    assert np.array_equal(den, oden)
    assert _close(p, op, P_RTOL)
    return r


def _check_scan(eng, b, nthreads=8):
    k, num, den, p = (t.cpu().numpy() for t in eng.ks_scan(mt4g.to_device_samples(b.samples), b.offsets, b.steps))
    ok, onum, oden, op = oracle.ks_scan(b.samples, b.offsets, b.steps, nthreads=nthreads)
    assert np.array_equal(k, ok) and np.array_equal(num, onum) and np.array_equal(den, oden)
    assert _close(p, op, P_RTOL)


# ------------------------------------------------------------------ Eq. 1 beside each change point

def _replay_parents(x, alpha, min_seg, reduced=False):
    """Binary segmentation replayed with the oracle's segment scan: {k: (lo, hi)} for every accepted
    split (Sec. II-C segmentation criterion, split by split with the test of Sec. IV-B-1 (4))."""
    if reduced:
        S_t = oracle.reduce_series(x)
        ranks = np.searchsorted(np.unique(S_t), S_t).astype(np.uint32)  # order and ties of S
        x = ranks.reshape(-1, 1)
    T, m = x.shape
    out = {}
    stack = [(0, T)]
    while stack:
        lo, hi = stack.pop()
        if hi - lo < 2 * min_seg:
            continue
        k, num, den = oracle.scan_segment(x, lo, hi, min_seg)
        if oracle.pvalue(num, den, m * (hi - lo)) <= alpha:
            out[k] = (lo, hi)
            stack += [(lo, k), (k, hi)]
    return out, m


@pytest.mark.parametrize("mode", [mt4g.MODE_FULL, mt4g.MODE_REDUCED])
def test_critical_values_match_eq1_oracle(eng, mode):
    rng = np.random.default_rng(61)
    series = [synth.generate(2, 8, 12).series(s) for s in range(12)]
    for _ in range(40):
        T = int(rng.integers(2, 200))
        m = int(rng.integers(1, 12))
        x = rng.integers(0, int(rng.integers(2, 400)), size=(T, m))
        for c in np.sort(rng.choice(np.arange(1, T), size=min(T - 1, int(rng.integers(0, 4))), replace=False)):
            x[c:] += int(rng.integers(0, 80))
        series.append(x.astype(np.uint32))
    b = synth.from_arrays(series)
    for alpha, min_seg in ((1e-6, 1), (1e-2, 3)):
        r = _check_segment(eng, b, alpha, min_seg, 16, mode)
        cnt, idx, crit = r.count.cpu().numpy(), r.idx.cpu().numpy(), r.crit.cpu().numpy()
        for s in range(b.S):
            parents, m = _replay_parents(b.series(s), alpha, min_seg, reduced=mode == mt4g.MODE_REDUCED)
            assert sorted(parents) == idx[s, :cnt[s]].tolist()
            for j in range(min(int(cnt[s]), 16)):
                k = int(idx[s, j])
                lo, hi = parents[k]
                want = oracle.critical_value(alpha, m * (k - lo), m * (hi - k))
                assert abs(crit[s, j] - want) <= 1e-15 * want, (s, k, crit[s, j], want)
            assert (crit[s, int(cnt[s]):] == 0.0).all()


def test_critical_value_host_input_and_eq1_consistency(eng):
    """The host-input call returns the same critical values, and every reported change point
    (accepted at p <= alpha) has D at or above its critical value: Q(lambda) <= alpha bounds the
    series' first term, 2 exp(-2 lambda^2) <= alpha + 2 exp(-8 lambda^2), whose inversion is Eq. 1."""
    import torch
    b = synth.generate(2, 9, 20)
    d = mt4g.to_device_samples(b.samples)
    r = eng.ks_segment(d, b.offsets, b.steps, 1e-6, 1, 16)
    host = torch.from_numpy(b.samples.view(np.int32)).pin_memory()
    h = eng.ks_segment_host(host, b.offsets, b.steps, 1e-6, 1, 16, chunk_samples=3 * 65536 + 1)
    assert torch.equal(r.crit, h.crit)
    cnt, num, den, crit = (t.cpu().numpy() for t in (r.count, r.dnum, r.dden, r.crit))
    assert cnt.sum() > 0
    for s in range(b.S):
        for j in range(cnt[s]):
            assert num[s, j] / den[s, j] >= crit[s, j] * (1 - 1e-9), (s, j)
            assert 0.0 < crit[s, j] < 1.0


# ------------------------------------------------------------------ run sweep at its cap

def test_run_sweep_cap_series_match_oracle(eng):
    """1535, 1536 and 1537 distinct values (the sweep's cap and one beyond it, sent back to the queue
    as slices), many distinct values with a wide span, and a series whose upper segments are too wide
    for the sweep: every answer equals the oracle's, with the run sweep and with 32-split slices."""
    rng = np.random.default_rng(29)
    series = []
    for U in (1535, 1536, 1537):
        h = U // 2  # steps 0..59 take values [0, h), steps 60..99 [h, U); every value occurs
        lo_part = np.concatenate([np.arange(h), rng.integers(0, h, size=60 * 40 - h)])
        hi_part = np.concatenate([np.arange(h, U), rng.integers(h, U, size=40 * 40 - (U - h))])
        rng.shuffle(lo_part)
        rng.shuffle(hi_part)
        series.append(np.concatenate([lo_part, hi_part]).astype(np.uint32).reshape(100, 40))
    x = rng.integers(0, 100000, size=(300, 16)).astype(np.uint32)
    x[120:] += 30000
    series.append(x)
    x = rng.integers(0, 30, size=(900, 64)).astype(np.uint32)  # m H^2 = 5.2e7 at the top: sweep
    x[300:] += 2
    x[650:] += 9
    series.append(x)
    x = rng.integers(0, 200, size=(1200, 1600)).astype(np.uint32)  # m H^2 >= 2^31 at the top: slices
    x[500:] += 3
    series.append(x)
    series.append(synth.generate(2, 77, 3).series(1))
    b = synth.from_arrays(series)
    d = mt4g.to_device_samples(b.samples)
    oseg = oracle.ks_segment(b.samples, b.offsets, b.steps, 1e-6, 1, 16, nthreads=8)[1:]
    oscan = oracle.ks_scan(b.samples, b.offsets, b.steps, nthreads=8)
    try:
        for kpt in (mt4g.SCAN_SWEEP, 1):
            eng.set_option(mt4g.OPT_SCAN_KPT, kpt)
            r = eng.ks_segment(d, b.offsets, b.steps, 1e-6, 1, 16)
            got = [t.cpu().numpy() for t in r[1:6]]
            for a, c in zip(got[:4], oseg[:4]):
                assert np.array_equal(a, c), kpt
            assert _close(got[4], oseg[4], P_RTOL)
            sc = [t.cpu().numpy() for t in eng.ks_scan(d, b.offsets, b.steps)]
            for a, c in zip(sc[:3], oscan[:3]):
                assert np.array_equal(a, c), kpt
            assert _close(sc[3], oscan[3], P_RTOL)
    finally:
        eng.set_option(mt4g.OPT_SCAN_KPT, 0)


# ------------------------------------------------------------------ heavy uneven series, full shape

def test_uneven_heavy_buckets_full_shape(eng):
    """One full-shape series of the uneven workload per heavy bucket: T near 4096, 2048-3583 and
    1024-2047 with m = 256, and T near 4096 and 2048-3583 with m = 64 (the shapes that dominate its
    scan cost, 4-pass radix sorts and more than 1536 distinct values), against the oracle."""
    S = 16384
    T, m, _, _ = synth.params(3, 2, S)
    buckets = [(3584, 4097, 256), (2048, 3584, 256), (1024, 2048, 256), (3584, 4097, 64), (2048, 3584, 64)]
    pick = []
    for t0, t1, mm in buckets:
        cand = np.nonzero((T >= t0) & (T < t1) & (m == mm))[0]
        assert len(cand) > 0, (t0, t1, mm)
        pick.append(int(cand[0]))
    b = synth.from_arrays([synth.generate(3, 2, 1, series_begin=s).series(0) for s in pick])
    assert int(b.offsets[-1]) > 2_000_000
    _check_segment(eng, b, 1e-6, 1, 16, nthreads=8)


# ------------------------------------------------------------------ run sweep with bound skipping

def test_sweep_bound_skipping_matches_oracle(eng):
    """MT4G_OPT_SWEEP_SKIP: splits an exact bound excludes are not evaluated, yet every answer
    equals the oracle's (heavy ties, ragged shapes, three-level series, reduced mode, a small batch
    whose segments are cut into parts), and fewer (split, value) pairs are evaluated."""
    rng = np.random.default_rng(71)
    b1 = synth.tiny_random(rng, 400, T_range=(2, 40), m_range=(1, 6), vmax=6)
    series = []
    for _ in range(50):
        T = int(rng.integers(2, 900))
        m = int(rng.integers(1, 9))
        x = rng.integers(0, int(rng.integers(2, 3000)), size=(T, m))
        for c in np.sort(rng.choice(np.arange(1, T), size=min(T - 1, 3), replace=False)):
            x[c:] += int(rng.integers(0, 200))
        series.append(x.astype(np.uint32))
    b2 = synth.from_arrays(series)
    b3 = synth.generate(2, 12, 40)
    try:
        for b, alpha in ((b1, 0.05), (b2, 1e-4), (b3, 1e-6)):
            eng.set_option(mt4g.OPT_SWEEP_SKIP, 0)
            _check_segment(eng, b, alpha)
            full = eng.last_work()
            eng.set_option(mt4g.OPT_SWEEP_SKIP, 1)
            _check_segment(eng, b, alpha)
            _check_scan(eng, b)
            _check_segment(eng, b, alpha, mode=mt4g.MODE_REDUCED)
            _check_segment(eng, b, alpha, min_seg=3)
        assert eng.last_sweep()["swept_segments"] > 0
        eng.set_option(mt4g.OPT_SWEEP_SKIP, 0)
        _check_segment(eng, b3, 1e-6)
        full = eng.last_work()
        eng.set_option(mt4g.OPT_SWEEP_SKIP, 1)
        _check_segment(eng, b3, 1e-6)
        assert eng.last_work() < 0.8 * full
    finally:
        eng.set_option(mt4g.OPT_SWEEP_SKIP, 0)


def test_sweep_bound_skipping_learned_mode(eng):
    """The learned call with bound skipping in the sweep answers as the full scan and the oracle."""
    import os
    b = synth.generate(2, 13, 24)
    eng.cnn_load(os.path.join(os.path.dirname(__file__), "..", "paper_2511_05958_b300", "weights", "cnn_c2.bin"))
    try:
        eng.set_option(mt4g.OPT_SWEEP_SKIP, 1)
        _check_segment(eng, b, 1e-6, mode=mt4g.MODE_LEARNED)
    finally:
        eng.set_option(mt4g.OPT_SWEEP_SKIP, 0)


def test_many_distinct_values_match_oracle(eng):
    """Series with 1.6k to 9.7k distinct values (beyond the run sweep's 1536: scanned in slices
    whatever tile is asked for), three value levels each, a series with more than 11552 values
    and one with m not a multiple of 4: every answer equals the oracle's, with the default plan and
    with the run sweep forced (its series go back to the queue as slices)."""
    rng = np.random.default_rng(83)
    series = []
    for U in (1700, 2600, 5000, 9000, 11000):
        m = int(rng.choice([4, 8, 12]))
        T = min(4000, max(120, -(-5 * U // m)))  # about five samples per value
        cps = np.sort(rng.choice(np.arange(T // 5, 4 * T // 5), size=2, replace=False))
        level = np.searchsorted(cps, np.arange(T), side="right")  # 0, 1, 2: three value ranges
        x = rng.integers(0, U // 3, size=(T, m)) + (level * (U // 3))[:, None]
        series.append(x.astype(np.uint32))
    x = rng.integers(0, 40000, size=(200, 100)).astype(np.uint32)  # beyond 11552 distinct values
    x[90:] += 20000
    series.append(x)
    x = rng.integers(0, 3000, size=(300, 10)).astype(np.uint32)  # m = 10: no 8-byte rows
    x[150:] += 900
    series.append(x)
    b = synth.from_arrays(series)
    U_all = [len(np.unique(b.series(s))) for s in range(b.S)]
    assert min(U_all[:5]) > 1536 and U_all[5] > 11552
    d = mt4g.to_device_samples(b.samples)
    oseg = oracle.ks_segment(b.samples, b.offsets, b.steps, 1e-6, 1, 16, nthreads=8)[1:]
    oscan = oracle.ks_scan(b.samples, b.offsets, b.steps, nthreads=8)
    try:
        for kpt in (0, mt4g.SCAN_SWEEP):
            eng.set_option(mt4g.OPT_SCAN_KPT, kpt)
            r = eng.ks_segment(d, b.offsets, b.steps, 1e-6, 1, 16)
            got = [t.cpu().numpy() for t in r[1:6]]
            for a, c in zip(got[:4], oseg[:4]):
                assert np.array_equal(a, c), kpt
            assert _close(got[4], oseg[4], P_RTOL)
            sc = [t.cpu().numpy() for t in eng.ks_scan(d, b.offsets, b.steps)]
            for a, c in zip(sc[:3], oscan[:3]):
                assert np.array_equal(a, c), kpt
            assert _close(sc[3], oscan[3], P_RTOL)
    finally:
        eng.set_option(mt4g.OPT_SCAN_KPT, 0)


def test_samples_pointer_off_a_16_byte_boundary(eng):
    """The counting sort writes each sample's table offset and then its run index with 8-byte
    accesses where the run-index array lines up with the samples' 16-byte boundary; a samples
    pointer one element past an allocation's start takes the 2-byte path instead.  Both give the
    oracle's segmentation."""
    import torch
    b = synth.generate(2, 12, 24)
    n = int(b.offsets[-1])
    buf = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    buf[1:] = torch.from_numpy(b.samples.view(np.int32)).cuda()
    _, ocnt, oidx, onum, oden, op = oracle.ks_segment(b.samples, b.offsets, b.steps, 1e-6, 1, 16, nthreads=8)
    for view in (buf[1:], torch.from_numpy(b.samples.view(np.int32)).cuda()):
        r = eng.ks_segment(view, b.offsets, b.steps, 1e-6, 1, 16)
        got = [t.cpu().numpy() for t in r[1:6]]
        for a, c in zip([ocnt, oidx, onum, oden], got[:4]):
            assert np.array_equal(a, c)
        assert (np.abs(got[4] - op) <= 1e-12 * np.abs(op)).all()
        assert eng.last_sweep()["counted_samples"] == n  # the counting path took every series

