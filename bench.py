"""Benchmark of the B300 KS change-point engine.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload plain]

One step = one full pass of the hot path over one batch of synthetic series that is already
resident in HBM: per-series radix sort + run table, the all-splits exact scan, the FP64
p-value and binary segmentation (alpha = 1e-6) through the device work queue.
Workload "plain": 1024 series, T=512 steps, m=128 uint32 samples per step, three change points
per series (lognormal levels 35/300/800/1100 cycles, 0.5% U{2000..10000} outliers), 268 MB of
input per batch, larger than the 126 MB L2, so consecutive steps do not hit in L2.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own batch of the same shape
(series are independent, no collective on the data path): weak scaling, value = all series
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
WORKLOADS = {
    # name: (generator config, seed, series)
    "plain": (2, 1, 1024),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="plain", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kpt", type=int, default=0, help="force the scan tile (1, 2, 4); 0 = automatic")
    ap.add_argument("--series", type=int, default=None,
                    help="override the batch size (only for small profiler captures; not a bench value)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(name, world):
    cfg, seed, S = WORKLOADS[name]
    return {"workload": "plain binary segmentation, 1024 series x T=512 x m=128 uint32 (c2 generator)",
            "series_per_gpu": S, "T": 512, "m": 128, "alpha": ALPHA, "min_seg": 1, "max_cp": MAX_CP,
            "global_series": S * world, "l2": "inputs (268 MB per batch) larger than L2",
            "parallelism": f"replicas x{world} (series sharded, no collective)"}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

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
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names[1:], f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The oracle timed on the host cores, on a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle
    import synth
    cfg, seed, S = WORKLOADS[args.workload]
    sample_n = 64
    stride = S // sample_n
    idx = np.arange(0, S, stride)[:sample_n]
    b = synth.generate(cfg, seed, S)
    sb = synth.from_arrays([b.series(int(s)) for s in idx])
    cores = os.cpu_count() or 1
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.ks_segment(sb.samples[:sb.offsets[1]], sb.offsets[:2], sb.steps[:1], ALPHA, 1, MAX_CP, nthreads=1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.ks_segment(sb.samples, sb.offsets, sb.steps, ALPHA, 1, MAX_CP, nthreads=cores)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    v = len(idx) / t
    line = {"metric": "KS change-point series/s (plain full exact segmentation)", "value": v, "unit": "series/s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 samples / int64 D / f64 p", "data": "synthetic",
            "config": workload_config(args.workload, 1),
            "samples_per_s": v * 512 * 128,
            "cpu_baseline": {"value": v, "unit": "series/s", "cores": cores, "kind": "oracle",
                             "sample": f"{len(idx)} of {S} series (every {stride}th) per step"},
            "e2e": {"value": v, "unit": "series/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args):
    import oracle
    import synth
    cfg, seed, S = WORKLOADS[args.workload]
    sample_n = 96
    stride = S // sample_n
    idx = np.arange(0, S, stride)[:sample_n]
    b = synth.generate(cfg, seed, S)
    sb = synth.from_arrays([b.series(int(s)) for s in idx])
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.ks_segment(sb.samples, sb.offsets, sb.steps, ALPHA, 1, MAX_CP, nthreads=cores)
    t = time.perf_counter() - t0
    return {"value": len(idx) / t, "unit": "series/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(idx)} of {S} series (every {stride}th), one segmentation pass, {t:.1f} s"}


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
    cfg, seed, S = WORKLOADS[args.workload]
    if args.series:
        S = args.series
    b = synth.generate(cfg, seed + 1000 * rank, S)
    host = torch.from_numpy(b.samples.view(np.int32)).pin_memory()
    d_samples = host.to(dev)
    eng = mt4g.Engine(local)
    eng.set_option(mt4g.OPT_STAGE_TIMING, 1)
    eng.set_option(mt4g.OPT_SCAN_KPT, args.kpt)
    stream = torch.cuda.current_stream(dev)
    out = None

    def step():
        nonlocal out
        out = eng.ks_segment(d_samples, b.offsets, b.steps, ALPHA, 1, MAX_CP, stream=stream, out=out, sync=False)

    for _ in range(max(args.warmup, 3)):
        step()
    assert eng.wait() in (mt4g.OK, mt4g.ECAPACITY)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---------------- device-resident timing
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    status = eng.wait()
    # per-stage durations of the timed calls (events the library recorded on `stream`)
    stage_ms = eng.stage_times(min(args.steps, 64))
    evals = eng.last_work()
    t = ms_total / 1e3
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    series_total = S * world * args.steps
    value = series_total / t
    ms_step = t / args.steps * 1e3

    # ---------------- end to end through host buffers (pinned), copies in the timed region
    res_host = None
    d2h_bytes = S * 4 + S * MAX_CP * (4 + 8 + 8 + 8)
    h2d_bytes = b.samples.nbytes + b.offsets.nbytes + b.steps.nbytes
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        d_in = host.to(dev, non_blocking=True)
        r = eng.ks_segment(d_in, b.offsets, b.steps, ALPHA, 1, MAX_CP, stream=stream, sync=False)
        res_host = [x.to("cpu", non_blocking=True) for x in r[1:]]
    f1.record(stream)
    barrier()
    te = f0.elapsed_time(f1) / 1e3
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([te], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        te = float(tt.item())
    e2e_value = series_total / te

    # ---------------- roofline of the dominant kernel
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    st = np.asarray(stage_ms)  # [steps, stages] ms: upload, sort, queue, collect
    sort_ms = float(st[:, 1].mean())
    queue_ms = float(st[:, 2].mean())
    Ntot = int(b.offsets[-1])
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or 2032.0
    evals = float(evals)
    if queue_ms >= sort_ms:
        # INT32 ALU bound: 4 integer ops (2 multiply-adds, |.|, max) per (split k, distinct value)
        ops = 4.0 * evals
        achieved = ops / (queue_ms / 1e3) / 1e12
        peak = sms * 128 * sm_mhz * 1e6 / 1e12
        roof = {"kernel": "queue_kernel (all-splits scan + p-value + segmentation)", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": None, "algorithmic_units": f"{evals:.4g} (k, distinct value) evaluations x 4 int ops",
                "peak_source": f"{sms} SMs x 128 INT32 lanes x {sm_mhz:.0f} MHz median SM clock"}
    else:
        byts = 10.0 * Ntot
        achieved = byts / (sort_ms / 1e3) / 1e9
        roof = {"kernel": "sort_series_kernel (radix sort + run table)", "bound": "hbm", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                "algorithmic_units": f"{Ntot} samples x 10 B (4 B read + 6 B sorted value/label written)",
                "peak_source": f"{hbm_src} HBM copy bandwidth"}
    roof["stage_ms"] = {"upload": float(st[:, 0].mean()), "sort": sort_ms, "queue": queue_ms,
                        "collect": float(st[:, 3].mean())}

    line = {"metric": "KS change-point series/s (plain full exact segmentation)", "value": value,
            "unit": "series/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 samples / int32-int64 exact D / f64 p", "data": "synthetic",
            "config": workload_config(args.workload, world), "samples_per_s": value * 512 * 128,
            "status": int(status), "gpu_launches": 3 * args.steps,
            "e2e": {"value": e2e_value, "unit": "series/s", "h2d_bytes_per_step": int(h2d_bytes),
                    "d2h_bytes_per_step": int(d2h_bytes)},
            "roofline": roof, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    eng.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
