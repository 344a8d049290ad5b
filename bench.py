#!/usr/bin/env python
"""Benchmark of the two-stage k-means hot path on GB300.

One step = one whole kmeans2_fit (GPU sampling of S_s and the initial centers,
the fast stage on S_s, the slow stage on S_n) on synthetic data resident in
HBM.  Metric: distance evaluations per second, sum over stages of Q * N * k
(the cost model of Section 3), plus time-to-converge per fit.

  python bench.py [--gpus N --steps K --warmup W] [--config NAME] [--impl ours|reference]

Default workload ("aniso8"): n = 500,000,000 points, d = 8, k = 32, anisotropic
Gaussian mixture (eigenvalues log-uniform in [0.1, 2], Haar rotations, means
U[-10, 10]^8, Dirichlet(1) weights) with 2% uniform background noise, subset
fraction 1%, tol 1e-5, max_iter 50 per stage, seed 0.  X is 16 GB, far larger
than L2, so no flush is needed between steps.

Under torchrun (N > 1) every rank fits its own replica of the workload (seed +
rank): the fit has no cross-rank exchange in this build ("replicas only"), the
value is the total over ranks divided by the slowest rank's time ("weak").

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the only other place this file runs the oracle;
the other is the cpu_baseline leg).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CONFIGS = {
    # name: generator, n, d, k, subset fraction, tol, max_iter, seed
    "gauss2d": dict(gen="iso", n=20_000, d=2, k=4, f=0.1, tol=1e-6, max_iter=100, seed=0),
    "aniso8": dict(gen="aniso", n=500_000_000, d=8, k=32, f=0.01, tol=1e-5, max_iter=50, seed=0),
    "aniso8_small": dict(gen="aniso", n=20_000_000, d=8, k=32, f=0.01, tol=1e-5, max_iter=50,
                         seed=0),
    "vmf128": dict(gen="vmf", n=50_000_000, d=128, k=1024, f=0.02, tol=1e-6, max_iter=50, seed=0),
}
METRIC = "two-stage k-means distance evals/s (time-to-converge per fit beside it)"
UNIT = "distance evals/s"
SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _gen(cfg, device, seed):
    import torch
    from paper_1108_1351_gb300 import synth
    n, d, k = cfg["n"], cfg["d"], cfg["k"]
    if cfg["gen"] == "iso":
        return synth.iso_gaussian_mixture(n, d, k, seed, device=device)
    if cfg["gen"] == "aniso":
        return synth.aniso_gaussian_noise(n, d, k, seed, device=device, chunk=1 << 24)
    if cfg["gen"] == "vmf":
        return synth.vmf_mixture(n, d, k, seed, device=device, chunk=1 << 20)
    raise ValueError(cfg["gen"])


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self.th = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(X_host, cfg, budget_s: float = 12.0):
    """The oracle as it stands, timed on the host cores: Lloyd steps on the
    first rows of the same data until ~budget_s of CPU work."""
    import numpy as np
    import oracle
    oracle.build()
    k, d = cfg["k"], cfg["d"]
    nt = max(1, oracle.max_threads())
    rows = min(len(X_host), 2_000_000)
    Xs = np.ascontiguousarray(X_host[:rows])
    C = Xs[:k].astype(np.float64)
    evals, t = 0, 0.0
    steps = 0
    while t < budget_s and steps < 50:
        t0 = time.perf_counter()
        C, lab, J, sh, em = oracle.lloyd_step(Xs, C, nthreads=nt)
        t += time.perf_counter() - t0
        evals += rows * k
        steps += 1
    return {"value": evals / t, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{steps} FP64 Lloyd steps on the first {rows} rows of the workload "
                      f"(d={d}, k={k}), {t:.1f} s"}


def run_reference(args, cfg):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_1108_1351_gb300 import synth
    oracle.build()
    nt = max(1, oracle.max_threads())
    rows = 1_000_000 if cfg["n"] > 1_000_000 else cfg["n"]
    small = dict(cfg, n=rows)
    X = _gen(small, "cpu", cfg["seed"]).numpy()
    k = cfg["k"]
    C = X[:k].astype(np.float64)
    for _ in range(args.warmup):
        oracle.lloyd_step(X, C, nthreads=nt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        C, lab, J, sh, em = oracle.lloyd_step(X, C, nthreads=nt)
    t = time.perf_counter() - t0
    value = rows * k * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.config, "n": cfg["n"], "d": cfg["d"], "k": k,
                       "subset_fraction": cfg["f"], "tol": cfg["tol"], "max_iter": cfg["max_iter"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": f"one FP64 Lloyd step per timed step on {rows} rows of the "
                                       f"workload's distribution (d={cfg['d']}, k={k})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, cfg):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_1108_1351_gb300 as km

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    km.load()
    n, d, k = cfg["n"], cfg["d"], cfg["k"]
    X = _gen(cfg, dev, cfg["seed"] + rank)
    torch.cuda.synchronize()
    centers = torch.empty(k, d, dtype=torch.float64, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def one(profile=None):
        return km.fit(X, k, cfg["f"], cfg["seed"] + rank, cfg["tol"], cfg["max_iter"],
                      centers_out=centers, labels_out=labels, stream=stream, profile=profile,
                      precision=args.precision)

    for _ in range(args.warmup):
        one()
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    clocks.start()
    prof = km.Profile()
    results = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        results.append(one(prof))
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    evals = sum(r.distance_evals for r in results)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    ev = torch.tensor([float(evals)], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(ev, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    total_evals = float(ev.item())

    # end to end through the same C-ABI call with HOST buffers
    e2e = None
    if args.e2e_steps > 0:
        Xh = torch.empty((n, d), dtype=torch.float32, pin_memory=True)
        Xh.copy_(X)
        ch = torch.empty((k, d), dtype=torch.float64, pin_memory=True)
        lh = torch.empty((n,), dtype=torch.int32, pin_memory=True)
        del X
        torch.cuda.empty_cache()
        km.fit(Xh, k, cfg["f"], cfg["seed"] + rank, cfg["tol"], cfg["max_iter"], centers_out=ch,
               labels_out=lh, stream=stream, precision=args.precision)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_evals = 0
        for _ in range(args.e2e_steps):
            r = km.fit(Xh, k, cfg["f"], cfg["seed"] + rank, cfg["tol"], cfg["max_iter"],
                       centers_out=ch, labels_out=lh, stream=stream, precision=args.precision)
            e_evals += r.distance_evals
        torch.cuda.synchronize()
        te = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
        ee = torch.tensor([float(e_evals)], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
            dist.all_reduce(ee, op=dist.ReduceOp.SUM)
        e2e = {"value": float(ee.item()) / float(te.item()), "unit": UNIT,
               "h2d_bytes_per_step": n * d * 4, "d2h_bytes_per_step": n * 4 + k * d * 8,
               "steps": args.e2e_steps, "ms_per_step": 1e3 * float(te.item()) / args.e2e_steps}
        Xh_host = Xh.numpy()
    else:
        Xh_host = X[: min(n, 2_000_000)].cpu().numpy()

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0
    peaks, peak_src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    p32 = 2.0 * FP32_LANES_PER_SM * SM_COUNT_GB300 * sm_max * 1e6 / 1e12     # TFLOP/s
    achieved = prof.assign_flops / (prof.assign_ms * 1e-3) / 1e12 if prof.assign_ms > 0 else None
    roofline = {"bound": "alu", "kernel": f"assign_small<{d}>" if d <= 16 else "assign_large",
                "achieved": achieved, "peak": p32, "unit": "TFLOP/s",
                "frac": (achieved / p32) if achieved else None, "traffic": None,
                "peak_source": f"derived: {SM_COUNT_GB300} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                               f"x {sm_max:.0f} MHz ({peak_src} max clock)",
                "kernel_ms_avg": prof.assign_ms / max(1, prof.assign_launches),
                "kernel_launches": prof.assign_launches,
                "achieved_hbm_gbs": prof.assign_bytes / (prof.assign_ms * 1e-3) / 1e9
                if prof.assign_ms > 0 else None,
                "hbm_peak_gbs": peaks.get("hbm_gbs")}
    if clk and clk.get("sm_mhz"):
        roofline["frac_at_observed_clock"] = achieved / (p32 * clk["sm_mhz"] / sm_max) if achieved else None
    r0 = results[-1]
    line = {
        "metric": METRIC, "value": total_evals / (ms_max * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.config, "n": n, "d": d, "k": k, "subset_fraction": cfg["f"],
                   "tol": cfg["tol"], "max_iter": cfg["max_iter"], "seed": cfg["seed"],
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (X is %.1f GB)" % (n * d * 4 / 1e9)
                   if n * d * 4 > 2e8 else "inputs smaller than L2"},
        "time_to_converge_s": (ms_max / args.steps) / 1e3,
        "fit": {"J": r0.J, "iters_fast": r0.iters_fast, "iters_slow": r0.iters_slow,
                "converged_fast": r0.converged_fast, "converged_slow": r0.converged_slow,
                "rechecked_points": r0.rechecked_points, "distance_evals": r0.distance_evals,
                "subset_size": r0.subset_size, "empty_clusters": r0.empty_clusters},
        "gpu_launches": int(prof.kernel_launches),
        "roofline": roofline,
        "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(Xh_host, cfg, budget_s=args.cpu_budget)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="aniso8", choices=sorted(CONFIGS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16", "tf32x3"],
                    help="distance-kernel form (every form returns the same labels)")
    args = ap.parse_args()
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)
    return run_ours(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
