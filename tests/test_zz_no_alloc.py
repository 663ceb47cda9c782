"""The allocation-free scan entry point (mt4g_ks_scan_noalloc) against mt4g_ks_scan and the oracle.

Callers that cannot allocate device memory (code inside a pool or arena someone else owns, a
process that forbids allocation after start-up) use the no-allocation variant; its results must be
those of the ordinary entry point and of the oracle: identical k and exact D, p within 1e-12
relative.  Two calls in a row check that the second is not disturbed by what the first left in the
shared static array.  This file is collected last so that a stop at the first failure has already
run every other test.
"""
import numpy as np
import pytest

import oracle
import paper_2511_05958_b300 as mt4g
import synth

pytestmark = pytest.mark.gpu


def _batches():
    rng = np.random.default_rng(77)
    a = synth.generate(1, 0, 1)
    series = [a.series(0)]
    for _ in range(60):
        T = int(rng.integers(2, 300))
        m = int(rng.integers(1, 20))
        x = rng.integers(0, int(rng.integers(2, 3000)), size=(T, m))
        x[int(rng.integers(0, T)):] += int(rng.integers(0, 100))
        series.append(x.astype(np.uint32))
    b1 = synth.from_arrays(series)
    b2 = synth.generate(2, 9, 6)  # 6 x 65536 samples: near the sample limit
    return [b1, b2]


def _noalloc(b):
    import torch
    d = mt4g.to_device_samples(b.samples)
    S = b.S
    out = mt4g.ScanResult(torch.full((S,), -7, dtype=torch.int32, device="cuda"),
                          torch.full((S,), -7, dtype=torch.int64, device="cuda"),
                          torch.full((S,), -7, dtype=torch.int64, device="cuda"),
                          torch.full((S,), -7.0, dtype=torch.float64, device="cuda"))
    rc = mt4g.ks_scan_noalloc(d, b.offsets, b.steps, out)
    assert rc == mt4g.OK, rc
    return [t.cpu().numpy() for t in out]


def test_noalloc_matches_ks_scan_twice_in_a_row():
    import torch
    assert torch.cuda.is_available()
    eng = mt4g.Engine(0)
    for b in _batches():
        ref = [t.cpu().numpy() for t in eng.ks_scan(mt4g.to_device_samples(b.samples), b.offsets, b.steps)]
        ok, onum, oden, op = oracle.ks_scan(b.samples, b.offsets, b.steps, nthreads=8)
        assert np.array_equal(ref[0], ok) and np.array_equal(ref[1], onum) and np.array_equal(ref[2], oden)
        assert (np.abs(ref[3] - op) <= 1e-12 * np.abs(op)).all()
        for _ in range(2):
            k, num, den, p = _noalloc(b)
            assert np.array_equal(k, ref[0]) and np.array_equal(num, ref[1]) and np.array_equal(den, ref[2])
            assert (np.abs(p - ref[3]) <= 1e-12 * np.abs(ref[3])).all()
    eng.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    """Beyond its stated limits the entry point returns MT4G_EINVAL before any GPU work; the
    binding rejects buffers too small for the tables it is given."""
    import torch
    S = mt4g.NOALLOC_MAX_SERIES + 1
    too_many = mt4g.NOALLOC_MAX_SAMPLES + 2
    d = torch.zeros(max(too_many, 2 * S), dtype=torch.int32, device="cuda")

    def outs(n):
        return mt4g.ScanResult(torch.zeros(n, dtype=torch.int32, device="cuda"),
                               torch.zeros(n, dtype=torch.int64, device="cuda"),
                               torch.zeros(n, dtype=torch.int64, device="cuda"),
                               torch.zeros(n, dtype=torch.float64, device="cuda"))
    assert mt4g.ks_scan_noalloc(d, np.array([0, too_many], np.int64), np.array([2], np.int32), outs(1)) == mt4g.EINVAL
    offs = np.arange(S + 1, dtype=np.int64) * 2
    assert mt4g.ks_scan_noalloc(d, offs, np.full(S, 2, np.int32), outs(S)) == mt4g.EINVAL
    with pytest.raises(mt4g.Mt4gError):
        mt4g.ks_scan_noalloc(d[:8], np.array([0, 16], np.int64), np.array([2], np.int32), outs(1))
    with pytest.raises(mt4g.Mt4gError):
        mt4g.ks_scan_noalloc(d, np.array([0, 16, 32], np.int64), np.array([2, 2], np.int32), outs(1))
