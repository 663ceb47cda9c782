"""Train the change-point proposal network on the GPU with the library's own kernels.

    python -m paper_2511_05958_b300.train [--series 2000000] [--steps 20000] [--batch 512]
                                          [--lr 1e-3] [--seed 3] [--out weights/cnn_c2.bin]
                                          [--checkpoint-every N] [--resume]

Training set: `series` series of the T=512, m=128, three-change-point workload (lognormal levels
35/300/800/1100 cycles, 0.5% outliers; generator seed 3), drawn on the GPU in chunks.  Each chunk
is labelled by the exact full binary segmentation (alpha 1e-6, the change points are the
targets) and summarised (17 features per step); the raw samples are then dropped, so the set
costs about 18.6 KB per series on the device.  Training: `steps` Adam steps (lr, beta 0.9/0.999,
eps 1e-8) on batches of `batch` series drawn uniformly with replacement.  The weights file and a
JSON log (loss curve, label statistics, timings, and the proposal quality on a held-out batch)
are written beside each other.  With --checkpoint-every N the weights and Adam state (the
library's checksummed format) are also written every N steps to OUT.ckpt, with the step in
OUT.ckpt.json; --resume continues from there.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

T_STEPS, M_SAMPLES, MAX_CP, ALPHA = 512, 128, 8, 1e-6


def build_training_set(eng, n_series, chunk, seed, dev):
    import torch

    import paper_2511_05958_b300 as mt4g
    import synth

    rows = T_STEPS + 4
    feats = torch.empty((n_series, rows, mt4g.FEAT_CHANNELS), dtype=torch.int16, device=dev)
    cnt = torch.empty(n_series, dtype=torch.int32, device=dev)
    idx = torch.empty((n_series, MAX_CP), dtype=torch.int32, device=dev)
    truth_hits = 0
    for b0 in range(0, n_series, chunk):
        n = min(chunk, n_series - b0)
        samples, meta = synth.generate_gpu(2, seed, n, series_begin=b0, device=dev)
        r = eng.ks_segment(samples, meta.offsets, meta.steps, ALPHA, 1, MAX_CP, mode=mt4g.MODE_FULL)
        cnt[b0:b0 + n] = r.count
        idx[b0:b0 + n] = r.idx
        eng.summaries(samples, meta.offsets, meta.steps, out=feats[b0:b0 + n].view(-1, mt4g.FEAT_CHANNELS))
        c = r.count.cpu().numpy()
        i = r.idx.cpu().numpy()
        truth_hits += int(np.sum((c == meta.ncp) & np.all(i == meta.cps[:, :MAX_CP], axis=1)))
        del samples, r
    return feats, cnt, idx, truth_hits


def evaluate(eng, seed, n, dev, n_win=3, half=16):
    """Proposal quality on held-out series of the benchmark distribution (host generator)."""
    import torch

    import paper_2511_05958_b300 as mt4g
    import synth

    b = synth.generate(2, seed, n)
    d = mt4g.to_device_samples(b.samples, dev)
    win, conf = eng.propose(d, b.offsets, b.steps, n_win, half)
    win = win.cpu().numpy()
    conf = conf.cpu().numpy()
    covered = 0
    for s in range(n):
        cps = b.cps[s, :b.ncp[s]]
        covered += all(any(abs(int(c) - int(w)) <= half for w in win[s] if w >= 0) for c in cps)
    torch.cuda.synchronize()
    return {"series": n, "conf_ge_0.9": float(np.mean(conf >= 0.9)), "median_conf": float(np.median(conf)),
            "all_true_cps_in_windows": covered / n}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--series", type=int, default=2_000_000)
    ap.add_argument("--chunk", type=int, default=16384)
    ap.add_argument("--steps", type=int, default=20_000)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--init-seed", type=int, default=12345)
    ap.add_argument("--out", default=os.path.join(HERE, "weights", "cnn_c2.bin"))
    ap.add_argument("--checkpoint-every", type=int, default=0,
                    help="every N steps write weights + Adam state to OUT.ckpt (0: only the final file)")
    ap.add_argument("--eval-series", type=int, default=2048, help="held-out series for the proposal quality")
    ap.add_argument("--resume", action="store_true",
                    help="continue from OUT.ckpt (weights, Adam moments and step) instead of a fresh init")
    args = ap.parse_args(argv)

    import torch

    import paper_2511_05958_b300 as mt4g

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    eng = mt4g.Engine(0)
    log = {"args": vars(args), "n_params_trained": 13217}
    t0 = time.time()
    feats, cnt, idx, hits = build_training_set(eng, args.series, args.chunk, args.seed, dev)
    torch.cuda.synchronize()
    log["data_seconds"] = time.time() - t0
    c = cnt.cpu().numpy()
    log["labels"] = {"mean_cps": float(c.mean()), "frac_3_cps": float(np.mean(c == 3)),
                     "frac_0_cps": float(np.mean(c == 0)), "exact_truth_recovery": hits / args.series}

    ckpt = args.out + ".ckpt"
    first_step = 1
    if args.resume and os.path.exists(ckpt):
        # the checkpoint carries the weights, the Adam moments and the Adam step; its sidecar the
        # loop step.  Batches after a resume are drawn from a generator reseeded with that step.
        eng.cnn_load(ckpt)
        with open(ckpt + ".json") as f:
            first_step = int(json.load(f)["step"]) + 1
        log["resumed_at_step"] = first_step - 1
    else:
        eng.cnn_init(args.init_seed)
    g = torch.Generator(device=dev)
    g.manual_seed(args.seed + (first_step - 1))
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    curve = []
    t1 = time.time()
    acc, nacc = 0.0, 0
    for step in range(first_step, args.steps + 1):
        sel = torch.randint(0, args.series, (args.batch,), device=dev, generator=g)
        bf = feats.index_select(0, sel).view(-1, mt4g.FEAT_CHANNELS)
        eng.cnn_train_step(bf, T_STEPS, args.batch, cnt.index_select(0, sel), idx.index_select(0, sel).contiguous(),
                           lr=args.lr, loss=loss)
        if step % 100 == 0:
            acc += float(loss.item())
            nacc += 1
        if step % 1000 == 0 or step == args.steps:
            curve.append({"step": step, "loss": acc / max(nacc, 1)})
            print(f"step {step}: loss {acc / max(nacc, 1):.4f}", flush=True)
            acc, nacc = 0.0, 0
        if args.checkpoint_every and step % args.checkpoint_every == 0:
            os.makedirs(os.path.dirname(os.path.abspath(ckpt)), exist_ok=True)
            eng.cnn_save(ckpt)
            with open(ckpt + ".json", "w") as f:
                json.dump({"step": step}, f)
    torch.cuda.synchronize()
    log["train_seconds"] = time.time() - t1
    log["loss_curve"] = curve
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    eng.cnn_save(args.out)
    log["held_out"] = evaluate(eng, 4, args.eval_series, dev)
    with open(os.path.splitext(args.out)[0] + ".train.json", "w") as f:
        json.dump(log, f, indent=1)
        f.write("\n")
    print(json.dumps(log["held_out"]), flush=True)
    eng.close()


if __name__ == "__main__":
    main()
