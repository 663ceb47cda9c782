"""Batching machinery on the GPU: CUDA-graph replay, the scan-tile autotuner, host input.

None of them changes any result: graph replays, tuned tiles and chunked host input must give the
oracle's answers (k, num, den bit-identical, p within 1e-12 relative) and those of direct calls.
"""
import numpy as np
import pytest

import oracle
import paper_2511_05958_b300 as mt4g
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture()
def eng():
    import torch
    assert torch.cuda.is_available()
    e = mt4g.Engine(0)
    yield e
    e.close()


def _seg(eng, d, b, mode=mt4g.MODE_FULL, out=None):
    r = eng.ks_segment(d, b.offsets, b.steps, 1e-6, 1, 16, mode=mode, out=out)
    return r, [t.cpu().numpy().copy() for t in r[1:6]]


def _same(x, y):
    for a, c in zip(x, y):
        assert np.array_equal(a, c)


def _oracle_same(b, got, alpha=1e-6, min_seg=1, max_cp=16):
    """got = [count, idx, dnum, dden, p] of a segmentation against the oracle's."""
    _, ocnt, oidx, onum, oden, op = oracle.ks_segment(b.samples, b.offsets, b.steps, alpha, min_seg, max_cp,
                                                      nthreads=8)
    _same([ocnt, oidx, onum, oden], got[:4])
    assert (np.abs(got[4] - op) <= 1e-12 * np.abs(op)).all()


def test_graph_replay_matches_direct_calls(eng):
    b = synth.generate(2, 41, 64)
    d = mt4g.to_device_samples(b.samples)
    _, ref = _seg(eng, d, b)
    eng.set_option(mt4g.OPT_GRAPH, 1)
    r1, g1 = _seg(eng, d, b)          # captured
    _same(ref, g1)
    r2, g2 = _seg(eng, d, b, out=r1)  # replayed (same pointers and tables)
    _same(ref, g2)
    _oracle_same(b, g2)
    # new data behind the same pointer: the replay reads it
    b2 = synth.generate(2, 42, 64)
    d.copy_(mt4g.to_device_samples(b2.samples))
    _, g3 = _seg(eng, d, b2, out=r1)
    eng.set_option(mt4g.OPT_GRAPH, 0)
    _, ref3 = _seg(eng, d, b2)
    _same(ref3, g3)
    _oracle_same(b2, g3)
    # a different shape is captured again
    eng.set_option(mt4g.OPT_GRAPH, 1)
    b3 = synth.generate(3, 2, 40)
    d3 = mt4g.to_device_samples(b3.samples)
    _, g4 = _seg(eng, d3, b3)
    eng.set_option(mt4g.OPT_GRAPH, 0)
    _, ref4 = _seg(eng, d3, b3)
    _same(ref4, g4)
    _oracle_same(b3, g4)


def test_graph_replay_scan_and_learned(eng):
    b = synth.generate(2, 43, 48)
    d = mt4g.to_device_samples(b.samples)
    ref_scan = [t.cpu().numpy() for t in eng.ks_scan(d, b.offsets, b.steps)]
    eng.cnn_init(4)
    eng.set_option(mt4g.OPT_CONF_MIN_PPM, 0)
    _, ref_l = _seg(eng, d, b, mode=mt4g.MODE_LEARNED)
    eng.set_option(mt4g.OPT_GRAPH, 1)
    out = eng.ks_scan(d, b.offsets, b.steps)
    for _ in range(2):
        out = eng.ks_scan(d, b.offsets, b.steps, out=out)
        for a, c in zip(ref_scan, out):
            assert np.array_equal(a, c.cpu().numpy())
    r, g1 = _seg(eng, d, b, mode=mt4g.MODE_LEARNED)
    _, g2 = _seg(eng, d, b, mode=mt4g.MODE_LEARNED, out=r)
    _same(ref_l, g1)
    _same(ref_l, g2)
    eng.set_option(mt4g.OPT_GRAPH, 0)
    eng.set_option(mt4g.OPT_CONF_MIN_PPM, 900000)


def test_graph_after_proposal_workspace_growth(eng):
    """A learned call that grows the proposal workspace after a graph was captured drops the
    graph (it points into the old workspace) but keeps its stream, events and pinned staging:
    the next graph call recaptures on them, and closing the engine frees each once."""
    small, big = synth.generate(2, 44, 8), synth.generate(2, 45, 64)
    ds, db = mt4g.to_device_samples(small.samples), mt4g.to_device_samples(big.samples)
    eng.cnn_init(4)
    eng.set_option(mt4g.OPT_GRAPH, 1)
    _, g1 = _seg(eng, ds, small)
    eng.set_option(mt4g.OPT_GRAPH, 0)
    _, l1 = _seg(eng, db, big, mode=mt4g.MODE_LEARNED)  # first proposal workspace, sized for 64 series
    eng.set_option(mt4g.OPT_GRAPH, 1)
    r, g2 = _seg(eng, ds, small)
    _, g3 = _seg(eng, ds, small, out=r)
    eng.set_option(mt4g.OPT_GRAPH, 0)
    _same(g1, g2)
    _same(g1, g3)
    _oracle_same(small, g1)
    _oracle_same(big, l1)


def test_autotune_keeps_results_and_roundtrips(eng, tmp_path):
    b = synth.generate(3, 2, 300)
    keep = [s for s in range(300) if float(b.steps[s]) ** 2 * float(b.m[s]) < 3e8][:120]
    bb = synth.from_arrays([b.series(s) for s in keep])
    d = mt4g.to_device_samples(bb.samples)
    _, ref = _seg(eng, d, bb)
    eng.autotune(d, bb.offsets, bb.steps)
    tiles = {eng.autotune_get(int(T), int(m)) for T, m in zip(bb.steps, bb.m)}
    assert tiles <= {1, 2, 4, mt4g.SCAN_SWEEP}
    _, tuned = _seg(eng, d, bb)
    _same(ref, tuned)
    _oracle_same(bb, tuned)
    path = str(tmp_path / "tune.txt")
    eng.autotune_save(path)
    e2 = mt4g.Engine(0)
    e2.autotune_load(path)
    for T, m in zip(bb.steps, bb.m):
        assert e2.autotune_get(int(T), int(m)) == eng.autotune_get(int(T), int(m))
    e2.close()


def test_host_input_chunks_match_device_input(eng):
    """mt4g_ks_segment_host: chunked copies overlapped with segmentation give the device-input
    answers, for chunk sizes from one series per chunk to one chunk, in full and learned mode;
    the capacity status of a middle chunk reaches mt4g_wait()."""
    import torch
    b = synth.generate(2, 44, 40)
    d = mt4g.to_device_samples(b.samples)
    host = torch.from_numpy(b.samples.view(np.int32)).pin_memory()
    eng.cnn_init(8)
    eng.set_option(mt4g.OPT_CONF_MIN_PPM, 0)
    try:
        for mode in (mt4g.MODE_FULL, mt4g.MODE_LEARNED):
            _, ref = _seg(eng, d, b, mode=mode)
            for chunk in (1, 3 * 65536 + 1, 10**9):
                r = eng.ks_segment_host(host, b.offsets, b.steps, 1e-6, 1, 16, mode=mode, chunk_samples=chunk)
                _same(ref, [t.cpu().numpy() for t in r[1:6]])
            _oracle_same(b, [t.cpu().numpy() for t in r[1:6]])
        # numpy input, ragged series, a capacity overflow in one chunk only
        rng = np.random.default_rng(5)
        series = [rng.integers(0, 50, size=(int(rng.integers(2, 60)), int(rng.integers(1, 9))), dtype=np.uint32)
                  for _ in range(30)]
        series[17] = np.repeat(np.arange(40, dtype=np.uint32)[:, None] * 1000, 64, axis=1)  # 39 change points
        bb = synth.from_arrays(series)
        full = eng.ks_segment(mt4g.to_device_samples(bb.samples), bb.offsets, bb.steps, 1e-6, 1, 8)
        assert full.rc == mt4g.ECAPACITY
        hr = eng.ks_segment_host(bb.samples, bb.offsets, bb.steps, 1e-6, 1, 8, chunk_samples=200)
        assert hr.rc == mt4g.ECAPACITY
        for a, c in zip(full[1:6], hr[1:6]):
            assert np.array_equal(a.cpu().numpy(), c.cpu().numpy())
        _oracle_same(bb, [t.cpu().numpy() for t in hr[1:6]], max_cp=8)
    finally:
        eng.set_option(mt4g.OPT_CONF_MIN_PPM, 900000)


def test_host_input_rejects_bad_batches_before_any_work(eng):
    """Arguments a chunk would reject are rejected up front: nothing is enqueued."""
    b = synth.generate(2, 45, 6)
    steps = b.steps.copy()
    steps[5] = 7  # the last series' sample count is no multiple of 7
    with pytest.raises(mt4g.Mt4gError) as e:
        eng.ks_segment_host(b.samples, b.offsets, steps, 1e-6, 1, 16, chunk_samples=1)
    assert e.value.code == mt4g.EINVAL and "series 5" in str(e.value)
    with pytest.raises(mt4g.Mt4gError) as e:
        eng.ks_segment_host(b.samples, b.offsets, b.steps, 1.5, 1, 16)
    assert e.value.code == mt4g.EINVAL


def test_consistency_checks_pass_and_change_nothing(eng):
    """MT4G_OPT_CHECKS: the sort-output check passes on every workload shape (equal-value runs,
    uneven series, the reduced path, host input) and leaves every answer unchanged."""
    import torch
    eng.cnn_init(8)
    for cfg, seed, S in ((1, 51, 40), (2, 52, 40), (3, 53, 24)):
        b = synth.generate(cfg, seed, S)
        d = mt4g.to_device_samples(b.samples)
        for mode in (mt4g.MODE_FULL, mt4g.MODE_REDUCED, mt4g.MODE_LEARNED):
            eng.set_option(mt4g.OPT_CHECKS, 0)
            r0, ref = _seg(eng, d, b, mode=mode)
            sc0 = eng.ks_scan(d, b.offsets, b.steps) if mode == mt4g.MODE_FULL else None
            eng.set_option(mt4g.OPT_CHECKS, 1)
            r1, got = _seg(eng, d, b, mode=mode)
            assert r1.rc == r0.rc and eng.wait() == r0.rc
            _same(ref, got)
            if sc0 is not None:
                sc1 = eng.ks_scan(d, b.offsets, b.steps)
                _same([t.cpu().numpy() for t in sc0], [t.cpu().numpy() for t in sc1])
        host = torch.from_numpy(b.samples.view(np.int32)).pin_memory()
        r2 = eng.ks_segment_host(host, b.offsets, b.steps, 1e-6, 1, 16, chunk_samples=3 * 65536 + 1)
        eng.set_option(mt4g.OPT_CHECKS, 0)
        _, ref2 = _seg(eng, d, b)
        _same(ref2, [t.cpu().numpy() for t in r2[1:6]])


def test_sweep_counters(eng):
    """mt4g_last_sweep: a plain call on series the run sweep takes ranks every sample and sweeps
    segments; with the sweep off (32-split slices) both counters are zero and answers agree."""
    b = synth.generate(2, 61, 24)
    d = mt4g.to_device_samples(b.samples)
    _, ref = _seg(eng, d, b)
    c = eng.last_sweep()
    n = int(b.offsets[-1])
    assert c["ranked_samples"] == n and c["swept_segments"] >= 24
    assert c["counted_samples"] == n and c["unswept_series"] == 0  # narrow spans: counted, all swept
    eng.set_option(mt4g.OPT_SCAN_KPT, 1)
    try:
        _, sl = _seg(eng, d, b)
        c1 = eng.last_sweep()
    finally:
        eng.set_option(mt4g.OPT_SCAN_KPT, 0)
    assert c1 == {"swept_segments": 0, "ranked_samples": 0, "counted_samples": 0, "unswept_series": 0}
    _same(ref, sl)
    # a wide value span: radix-sorted, still ranked and swept
    x = np.random.default_rng(3).integers(0, 1 << 30, size=(64, 8)).astype(np.uint32)
    x[:, :] = (x % 900) * 1000003 % (1 << 31)  # 900 distinct values spread over 2^31
    x[40:] += 5
    bw = synth.from_arrays([x])
    dw = mt4g.to_device_samples(bw.samples)
    _, w0 = _seg(eng, dw, bw)
    cw = eng.last_sweep()
    assert cw["ranked_samples"] == 512 and cw["counted_samples"] == 0 and cw["unswept_series"] == 0
    eng.set_option(mt4g.OPT_SCAN_KPT, 1)
    try:
        _, w1 = _seg(eng, dw, bw)
    finally:
        eng.set_option(mt4g.OPT_SCAN_KPT, 0)
    _same(w0, w1)
