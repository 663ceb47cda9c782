"""Multi-rank host logic on CPU (gloo, world size 2): cost-balanced series shards, per-rank work,
gathering to rank 0 and the max-over-ranks timing reduction.  The per-rank compute here is the CPU
oracle (the GPU engine is the same call on each rank's own GPU); the gathered answers must equal a
single-process run over the whole batch."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2511_05958_b300 import multi
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = synth.generate(3, 2, 24)
        keep = [s for s in range(24) if float(b.steps[s]) ** 2 * b.m[s] < 2e7]
        bb = synth.from_arrays([b.series(s) for s in keep])
        shards, load = multi.shard_by_cost(bb.steps, bb.m, world)
        idx = shards[rank]
        sub, off, st = multi.sub_batch(bb.samples, bb.offsets, bb.steps, idx)
        rc, cnt, cp, num, den, p = oracle.ks_segment(sub, off, st, 1e-6, 1, 16)
        full = multi.gather_rows({"cnt": cnt, "idx": cp, "num": num, "den": den}, idx, bb.S)
        t = multi.max_over_ranks(1.0 + rank)
        if rank == 0:
            rc0, c0, i0, n0, d0, p0 = oracle.ks_segment(bb.samples, bb.offsets, bb.steps, 1e-6, 1, 16)
            ok = (np.array_equal(full["cnt"], c0) and np.array_equal(full["idx"], i0)
                  and np.array_equal(full["num"], n0) and np.array_equal(full["den"], d0))
            covered = sorted(np.concatenate(shards).tolist()) == list(range(bb.S))
            q.put({"ok": bool(ok), "covered": covered, "tmax": t, "load": load.tolist(), "S": bb.S})
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_gather_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res["ok"] and res["covered"] and res["tmax"] == 2.0
    lo, hi = sorted(res["load"])
    assert hi <= 2.0 * lo + 1  # cost-balanced shards


def test_shards_cover_every_series_once():
    from paper_2511_05958_b300 import multi
    rng = np.random.default_rng(3)
    T = rng.integers(32, 4097, 500)
    m = rng.choice([8, 16, 64, 256], 500)
    for world in (1, 2, 3, 8):
        shards, load = multi.shard_by_cost(T, m, world)
        allidx = np.sort(np.concatenate(shards))
        assert np.array_equal(allidx, np.arange(500))
        assert max(load) <= min(load) + (T.astype(float) ** 2 * m).max() + 1e-6
