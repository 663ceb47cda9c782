"""Benchmark of the B300 KS change-point engine.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload learned|plain|uneven]

Workloads (synthetic series from the seeded generator, resident in HBM before timing):
  learned (default): 65536 series, T=512 steps, m=128 uint32 samples per step, three change points
      per series (lognormal levels 35/300/800/1100 cycles, 0.5% U{2000..10000} outliers), seed 4;
      17.2 GB per batch.  One step = one learned+exact binary segmentation (alpha 1e-6): per-series
      radix sort + run table, per-step summaries, the proposal CNN, windows; series the run sweep
      takes (at most 1536 distinct values) are scanned in full by it, the others by exact window
      and grid scans with certification, refinement or full-scan fallback; FP64 p-values.  The
      plain full exact segmentation of the same batch is timed alongside; every series' answers
      of the two paths are compared (agreement) and the fallback rate is reported.  So is the
      learned path with the sweep off (32-split slices: window and grid probes for every series).
  plain: 1024 series of the same distribution (seed 1), plain full exact segmentation.
  uneven: 16384 series, T ~ U{32..4096}, m in {8,16,64,256}, 0-4 change points with level ratios
      log-uniform in [1.01, 30], 1% Pareto(1.5) tails (seed 2); plain full segmentation, one
      persistent-kernel launch over the whole batch with scan tiles per (log2 T, log2 m) bucket
      from the autotuner (mt4g_autotune, run on the batch before timing), each step one CUDA-graph
      replay (MT4G_OPT_GRAPH); the stage times come from extra direct calls with the same tiles.
Every batch is larger than the 126 MB L2, so consecutive steps do not hit in L2.

Prints one JSON line (rank 0).  Under torchrun each rank processes its own batch of the same shape
(series are independent; no collective on the data path): weak scaling, value = all series
processed / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALPHA = 1e-6
MAX_CP = 16
METRIC = "KS change-point series/s & samples/s; learned+exact vs plain at equal answers"
WEIGHTS = os.path.join(ROOT, "paper_2511_05958_b300", "weights", "cnn_c2.bin")
WORKLOADS = {
    # name: (generator config, seed, series, learned, description)
    "learned": (2, 4, 65536, True, "learned+exact segmentation, 65536 series x T=512 x m=128 uint32 "
                                   "(3 change points, lognormal levels, 0.5% outliers)"),
    "plain": (2, 1, 1024, False, "plain full segmentation, 1024 series x T=512 x m=128 uint32"),
    "uneven": (3, 2, 16384, False, "plain full segmentation, 16384 uneven series, T 32..4096, m 8..256"),
}
LAUNCHES = {False: 4, True: 9}  # our kernels per call (plain / learned: two gated queue launches)
RECIPES = {2: "synth recipe 2 (T=512, m=128, levels 35/300/800/1100, 0.5% outliers)",
           3: "synth recipe 3 (T 32..4096, m 8..256, 0-4 level ratios 1.01..30, Pareto tails)"}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, per series, from the ncu
# captures summarised under profiles/ (4096 series of recipe 2); keyed by (workload, stage) and
# scaled by the number of series.  The sort: profiles/sort_series_kernel_4096x512x128.md (the
# plain workload runs the same kernel on the same distribution).  Only kernels captured as they
# are now appear here; the others report null.
# The queue: profiles/queue_kernel_sweep_4096x512x128.md (4096 series; learned calls on this
# distribution run the same plain instantiation as plain calls).
NCU_TRAFFIC_PER_SERIES = {("plain", "sort"): 1668.576e6 / 4096, ("learned", "sort"): 1668.576e6 / 4096,
                          ("learned", "queue"): 2358.536e6 / 4096, ("plain", "queue"): 2358.536e6 / 4096}
STAGES = ["upload", "sort", "proposals", "queue", "collect"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="learned", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kpt", type=int, default=0, help="force the scan tile (1, 2, 4, or 8 for the run sweep); 0 = automatic")
    ap.add_argument("--series", type=int, default=None,
                    help="override the batch size (only for small profiler captures; not a bench value)")
    return ap.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload_config(name, world, S):
    cfg, seed, _, learned, desc = WORKLOADS[name]
    return {"workload": desc, "series_per_gpu": S, "global_series": S * world, "alpha": ALPHA, "min_seg": 1,
            "max_cp": MAX_CP, "generator": f"{RECIPES[cfg]}, seed {seed}", "learned": learned,
            "l2": "inputs larger than L2", "parallelism": f"replicas x{world} (series sharded, no collective)"}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling the SM clock and throttle reasons while a timed region runs.

    Any NVML client attached to the GPU (this sampler, an idle nvidia-smi, or one NVML handle in
    the process) slows the segmentation by about 2.3% on B300, whatever it queries and however
    often, so every device-timed arm that a ratio compares runs with a sampler of its own."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc = index, None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle timing

def oracle_sample(args, baseline=False):
    """A bounded, deterministic sample of the workload for the oracle: every k-th series.  The
    reference arm times it once per step (a few seconds each); the CPU baseline beside the GPU
    line times a larger one once (about 10-20 s on 16 host cores)."""
    cfg, seed, S, _, _ = WORKLOADS[args.workload]
    import synth
    n = ({"learned": 4096, "plain": 1024, "uneven": 1024} if baseline else
         {"learned": 1024, "plain": 96, "uneven": 256})[args.workload]
    stride = max(1, S // n)
    idx = np.arange(0, S, stride)[:n]
    if cfg == 3:  # keep the sample's CPU time bounded: the oracle is O(T N) per segment
        T, m, _, _ = synth.params(cfg, seed, S)
        cost = T.astype(np.float64) ** 2 * m
        idx = idx[cost[idx] < 2e8]
    parts = [synth.generate(cfg, seed, 1, series_begin=int(s)).series(0) for s in idx]
    return synth.from_arrays(parts), f"{len(idx)} of {S} series (every {stride}th" + \
        (", cost-capped)" if cfg == 3 else ")")


def run_oracle(sb, nthreads):
    import oracle
    t0 = time.perf_counter()
    oracle.ks_segment(sb.samples, sb.offsets, sb.steps, ALPHA, 1, MAX_CP, nthreads=nthreads)
    return time.perf_counter() - t0


def run_reference(args, rank, world):
    """The oracle timed on the host cores, on a bounded sample of the same workload."""
    if rank != 0:
        return
    sb, desc = oracle_sample(args)
    cores = os.cpu_count() or 1
    times = [run_oracle(sb, cores) for _ in range(args.steps)]
    t = float(np.mean(times))
    v = sb.S / t
    S = WORKLOADS[args.workload][2]
    line = {"metric": METRIC, "value": v, "unit": "series/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 samples / int64 D / f64 p", "data": "synthetic",
            "config": workload_config(args.workload, 1, S),
            "samples_per_s": float(v * sb.offsets[-1] / sb.S),
            "cpu_baseline": {"value": v, "unit": "series/s", "cores": cores, "kind": "oracle",
                             "sample": desc + " per step"},
            "e2e": {"value": v, "unit": "series/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- B300 arm

def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import paper_2511_05958_b300 as mt4g
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    cfg, seed, S, learned, _ = WORKLOADS[args.workload]
    if args.series:
        S = args.series
    b = synth.generate(cfg, seed + 1000 * rank, S)
    host = torch.from_numpy(b.samples.view(np.int32)).pin_memory()
    d_samples = host.to(dev)
    Ntot = int(b.offsets[-1])
    eng = mt4g.Engine(local)
    eng.set_option(mt4g.OPT_STAGE_TIMING, 1)
    eng.set_option(mt4g.OPT_SCAN_KPT, args.kpt)
    if learned:
        eng.cnn_load(WEIGHTS)
    mode = mt4g.MODE_LEARNED if learned else mt4g.MODE_FULL
    stream = torch.cuda.current_stream(dev)
    graph = args.workload == "uneven"
    tune_s = None
    if graph and not args.kpt:  # the uneven workload: autotuned tiles per shape bucket, graph replay per step
        t0 = time.perf_counter()
        eng.autotune(d_samples, b.offsets, b.steps, stream=stream)
        tune_s = time.perf_counter() - t0

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(t):
        if world > 1:
            import torch.distributed as dist
            tt = torch.tensor([t], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        return t

    def timed(m, steps, warm, clocks=None):
        out = None
        for _ in range(max(warm, 3)):
            out = eng.ks_segment(d_samples, b.offsets, b.steps, ALPHA, 1, MAX_CP, mode=m, stream=stream, out=out,
                                 sync=False)
        assert eng.wait() in (mt4g.OK, mt4g.ECAPACITY), eng.last_error()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            out = eng.ks_segment(d_samples, b.offsets, b.steps, ALPHA, 1, MAX_CP, mode=m, stream=stream, out=out,
                                 sync=False)
        e1.record(stream)
        barrier()
        clk = clocks.stop() if clocks else None
        status = eng.wait()
        if graph:  # graph replays record no stage times: time direct calls with the same tiles
            eng.set_option(mt4g.OPT_GRAPH, 0)
            for _ in range(min(steps, 3) + 1):
                eng.ks_segment(d_samples, b.offsets, b.steps, ALPHA, 1, MAX_CP, mode=m, stream=stream, out=out,
                               sync=False)
            eng.wait()
            eng.set_option(mt4g.OPT_GRAPH, 1)
            stages = eng.stage_times(min(steps, 3))
        else:
            stages = eng.stage_times(min(steps, 64))
        return max_over_ranks(e0.elapsed_time(e1) / 1e3), out, status, stages, eng.last_work(), clk

    clocks = ClockSampler(local)
    if graph:
        eng.set_option(mt4g.OPT_GRAPH, 1)
    t_main, out_main, status, stages, evals, clk = timed(mode, args.steps, args.warmup, clocks)
    if graph:
        eng.set_option(mt4g.OPT_GRAPH, 0)
    stats = eng.learned_stats() if learned else None
    sweep = eng.last_sweep()
    ranked, counted = sweep["ranked_samples"], sweep["counted_samples"]
    value = S * world * args.steps / t_main
    line = {"metric": METRIC, "value": value, "unit": "series/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_main / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 samples / int32-int64 exact D / f64 p"
            + (" / bf16-fp32 proposal CNN" if learned else ""), "data": "synthetic",
            "config": workload_config(args.workload, world, S), "samples_per_s": value * Ntot / S,
            "status": int(status), "gpu_launches": LAUNCHES[learned] * args.steps,
            "swept_segments": sweep["swept_segments"], "ranked_samples": ranked, "counted_samples": counted,
            "unswept_series": sweep["unswept_series"]}
    if graph:
        tiles = {}
        for T_, m_ in zip(b.steps, b.m):
            key = f"T2^{int(T_).bit_length() - 1},m2^{int(m_).bit_length() - 1}"
            tiles[key] = eng.autotune_get(int(T_), int(m_))
        line["cuda_graph"] = True
        line["autotune"] = {"seconds": tune_s, "tiles": dict(sorted(tiles.items())),
                            "tile_codes": "1/2/4 = groups of 32 splits per work item, 8 = run sweep",
                            "forced_tile": args.kpt or None}
        # the learned path on the same batch (the network trained on the three-level recipe; its
        # window and grid probes serve the series scanned in slices), direct calls with the same
        # tiles, answers compared with the plain call's on the device
        eng.cnn_load(WEIGHTS)
        res_p = [x.clone() for x in out_main[1:6]]
        graph = False
        t_l, out_l, _, stages_l, evals_l, clk_l = timed(mt4g.MODE_LEARNED, args.steps, 1, ClockSampler(local))
        st_l = eng.learned_stats()
        same_l = torch.ones(S, dtype=torch.bool, device=dev)
        for a_, c_ in zip(res_p, out_l[1:6]):
            same_l &= (a_ == c_).reshape(S, -1).all(dim=1)
        line["learned"] = {"value": S * world * args.steps / t_l, "ms_per_step": t_l / args.steps * 1e3,
                           "speedup_vs_plain": t_main / t_l, "agreement": float(same_l.float().mean().item()),
                           "fallback_rate": float(out_l[6].float().mean().item()), "evals": evals_l,
                           "evals_plain": evals, "certified_segments": st_l["certified"],
                           "refined_segments": st_l["refined"], "clocks": clk_l,
                           "stage_ms": dict(zip(STAGES, np.asarray(stages_l).mean(axis=0).tolist()))}
    if learned:
        res_l = [x.clone() for x in out_main[1:6]]
        fb = out_main[6].clone()
        t_plain, out_plain, _, stages_p, evals_p, clk_p = timed(mt4g.MODE_FULL, args.steps, 1, ClockSampler(local))
        same = torch.ones(S, dtype=torch.bool, device=dev)
        for a, c in zip(res_l, out_plain[1:6]):
            same &= (a == c).reshape(S, -1).all(dim=1)
        plain_value = S * world * args.steps / t_plain
        eng.set_option(mt4g.OPT_SCAN_KPT, 1)  # the probe path on slices, for comparison
        try:
            t_sl, out_sl, _, stages_sl, evals_sl, clk_sl = timed(mode, args.steps, 1, ClockSampler(local))
            stats_sl = eng.learned_stats()
            same_sl = torch.ones(S, dtype=torch.bool, device=dev)
            for a, c in zip(res_l, out_sl[1:6]):
                same_sl &= (a == c).reshape(S, -1).all(dim=1)
        finally:
            eng.set_option(mt4g.OPT_SCAN_KPT, 0)
        line["learned_slices"] = {
            "value": S * world * args.steps / t_sl, "ms_per_step": t_sl / args.steps * 1e3,
            "agreement": float(same_sl.float().mean().item()), "evals": evals_sl,
            "certified_segments": stats_sl["certified"], "refined_segments": stats_sl["refined"],
            "clocks": clk_sl, "stage_ms": dict(zip(STAGES, np.asarray(stages_sl).mean(axis=0).tolist()))}
        # window-only scans of the swept series (no certification): agreement with the full
        # scan measured per series, low-confidence and non-significant series fall back
        eng.set_option(mt4g.OPT_LEARNED_WINDOWS, 1)
        try:
            t_w, out_w, _, stages_w, evals_w, clk_w = timed(mode, args.steps, 1, ClockSampler(local))
        finally:
            eng.set_option(mt4g.OPT_LEARNED_WINDOWS, 0)
        same_w = torch.ones(S, dtype=torch.bool, device=dev)
        for a_, c_ in zip(out_plain[1:6], out_w[1:6]):
            same_w &= (a_ == c_).reshape(S, -1).all(dim=1)
        line["learned_windows"] = {
            "value": S * world * args.steps / t_w, "ms_per_step": t_w / args.steps * 1e3,
            "speedup_vs_plain": t_plain / t_w, "agreement": float(same_w.float().mean().item()),
            "fallback_rate": float(out_w[6].float().mean().item()), "evals": evals_w, "clocks": clk_w,
            "stage_ms": dict(zip(STAGES, np.asarray(stages_w).mean(axis=0).tolist()))}
        line.update({"plain_value": plain_value, "plain_ms_per_step": t_plain / args.steps * 1e3,
                     "speedup_vs_plain": value / plain_value, "agreement": float(same.float().mean().item()),
                     "fallback_rate": float(fb.float().mean().item()),
                     "certified_segments": stats["certified"], "refined_segments": stats["refined"],
                     "evals_learned": evals, "evals_plain": evals_p, "plain_clocks": clk_p,
                     "plain_stage_ms": dict(zip(STAGES, np.asarray(stages_p).mean(axis=0).tolist()))})

    # ---------------- end to end through host buffers (pinned), copies in the timed region
    h2d = b.samples.nbytes + b.offsets.nbytes + b.steps.nbytes
    e_steps = max(1, min(args.steps, 5))
    # the call's chunk size (a public argument): a short trial of 2, 4, 8 and 16 chunks before the
    # timed region picks it.  Each chunk overlaps its copy with the previous chunk's segmentation
    # and ends on its heaviest series' critical path, so the best count depends on the batch.
    trials = {}
    for nch in (2, 4, 8, 16):
        cs = (Ntot + nch - 1) // nch
        eng.ks_segment_host(host, b.offsets, b.steps, ALPHA, 1, MAX_CP, mode=mode, stream=stream,
                            chunk_samples=cs)
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        eng.ks_segment_host(host, b.offsets, b.steps, ALPHA, 1, MAX_CP, mode=mode, stream=stream,
                            chunk_samples=cs, sync=False)
        g1.record(stream)
        barrier()
        trials[nch] = max_over_ranks(g0.elapsed_time(g1))
    e_chunks = min(trials, key=trials.get)
    e_cs = (Ntot + e_chunks - 1) // e_chunks
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    outs_h = None
    for _ in range(e_steps):
        # the public host-input call: chunked host-to-device copies overlapped with segmentation
        r = eng.ks_segment_host(host, b.offsets, b.steps, ALPHA, 1, MAX_CP, mode=mode, stream=stream,
                                chunk_samples=e_cs, sync=False)
        if outs_h is None:
            outs_h = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in r[1:]]
        for h_, x in zip(outs_h, r[1:]):
            h_.copy_(x, non_blocking=True)
    f1.record(stream)
    barrier()
    te = max_over_ranks(f0.elapsed_time(f1) / 1e3)
    d2h = sum(x.numel() * x.element_size() for x in outs_h)  # every result tensor read back per step
    line["e2e"] = {"value": S * world * e_steps / te, "unit": "series/s", "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h), "steps": e_steps, "chunks": e_chunks,
                   "chunk_trial_ms": {str(k): round(v, 2) for k, v in trials.items()}}

    # ---------------- rooflines: every stage's kernel against its bound; the dominant one is `roofline`
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    ms = dict(zip(STAGES, np.asarray(stages).mean(axis=0).tolist()))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or 2032.0
    nominal_int = sms * 128 * sm_mhz * 1e6 / 1e12
    int_peak = mt4g.int32_peak(local)
    rooflines = {
        "queue": {"kernel": "queue_kernel (exact scans, p-values, segmentation)", "bound": "alu",
                  "achieved": 4.0 * evals / (ms["queue"] / 1e3) / 1e12, "peak": int_peak, "unit": "Tops/s",
                  "traffic": None,
                  "algorithmic_units": f"{evals:.4g} (split, distinct value) evaluations x 4 int ops",
                  "peak_source": "measured: mt4g_int32_peak (the scan's 4-op step mix on every SM, this run)",
                  "nominal_peak": nominal_int,
                  "nominal_source": f"{sms} SMs x 128 INT32 lanes x {sm_mhz:.0f} MHz (median SM clock under load)"},
        "sort": {"kernel": "sort_series_kernel (radix or counting sort + run table + run indices)", "bound": "hbm",
                 "achieved": (10.0 * (Ntot - counted) + 6.0 * ranked) / (ms["sort"] / 1e3) / 1e9,
                 "peak": hbm_peak, "unit": "GB/s", "traffic": None,
                 "algorithmic_units": f"{Ntot - counted} radix-sorted samples x 10 B (4 B read + 6 B sorted "
                                      f"value/label written) + {ranked} ranked samples x 6 B (4 B read, 2 B run "
                                      f"index written; {counted} of them by counting, without labels)",
                 "peak_source": f"{hbm_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
    }
    if learned and ranked > 0 and sweep["unswept_series"] == 0:
        # every series was swept: the proposal kernels returned at once (nothing to measure)
        line["proposals_skipped"] = True
    elif learned:
        rooflines["proposals"] = {"kernel": "summaries + CNN + windows", "bound": "hbm",
                                  "achieved": 4.0 * Ntot / (ms["proposals"] / 1e3) / 1e9, "peak": hbm_peak,
                                  "unit": "GB/s", "traffic": None,
                                  "algorithmic_units": f"{Ntot} samples x 4 B read",
                                  "peak_source": f"{hbm_src} HBM copy bandwidth"}
    for k, r in rooflines.items():
        r["frac"] = r["achieved"] / r["peak"]
        per = NCU_TRAFFIC_PER_SERIES.get((args.workload, k))
        r["traffic"] = per * S if per is not None else None
    dominant = max(rooflines, key=lambda k: ms[k])
    roof = dict(rooflines[dominant])
    line["rooflines"] = {k: {kk: v[kk] for kk in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic")}
                         for k, v in rooflines.items()}
    roof["stage_ms"] = ms
    line["roofline"] = roof
    line["clocks"] = clk
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sb, desc = oracle_sample(args, baseline=True)
        cores = os.cpu_count() or 1
        t = run_oracle(sb, cores)
        line["cpu_baseline"] = {"value": sb.S / t, "unit": "series/s", "cores": cores, "kind": "oracle",
                                "sample": f"{desc}, one segmentation pass, {t:.1f} s"}
        # the same oracle on one host thread, on the first 64 series of that sample
        import synth
        one = synth.from_arrays([sb.series(s) for s in range(min(64, sb.S))])
        t1 = run_oracle(one, 1)
        line["cpu_baseline"]["single_thread"] = {"value": one.S / t1, "unit": "series/s", "cores": 1,
                                                 "sample": f"first {one.S} series of the sample, {t1:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    eng.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
