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

Under torchrun (N > 1) the ranks run ONE row-sharded fit (the shard-session API
over NCCL: each rank holds its own 5e8-row block of one data set, drawn from
the same mixture with its own sample stream, and the ranks all-reduce the
integer partials every iteration); the value is the global distance
evaluations divided by the slowest rank's time, per-GPU rows fixed ("weak").
``--parallelism replicas`` instead fits an independent replica per rank.

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
    "vmf128_small": dict(gen="vmf", n=2_000_000, d=128, k=1024, f=0.02, tol=1e-6, max_iter=50,
                         seed=0),
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


def _gen(cfg, device, seed, sample_seed=None):
    import torch
    from paper_1108_1351_gb300 import synth
    n, d, k = cfg["n"], cfg["d"], cfg["k"]
    if cfg["gen"] == "iso":
        return synth.iso_gaussian_mixture(n, d, k, seed, device=device)
    if cfg["gen"] == "aniso":
        return synth.aniso_gaussian_noise(n, d, k, seed, device=device, chunk=1 << 24,
                                          sample_seed=sample_seed)
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
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, max clock and the throttle reasons seen Active in
        nvidia-smi CSV rows of FIELDS (malformed rows skipped); None if no row
        parses."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
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


TF32_PER_BF16 = 1.1 / 2.25      # nominal dense TF32 : BF16 tensor rate on GB300


def fp32_peak(dev, stream):
    """Measured FP32 FMA throughput of this GPU (TFLOP/s, 2 flop per FMA): the
    probe library's scalar and packed (fma.rn.f32x2) FMA chains at full
    occupancy, best of three timed launches each, with the SM clock sampled
    while they run.  None if the probe library cannot be loaded."""
    import ctypes
    import torch
    path = os.path.join(ROOT, "paper_1108_1351_gb300", "libfp32peak.so")
    try:
        lib = ctypes.CDLL(path)
    except OSError:
        return None
    lib.fp32_fma_probe.restype = ctypes.c_int
    lib.fp32_fma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(ctypes.c_double)]
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    sp = ctypes.c_void_p(stream.cuda_stream)

    def run(packed, iters):
        ms, fmas = ctypes.c_float(), ctypes.c_double()
        rc = lib.fp32_fma_probe(packed, blocks, iters, ctypes.c_void_p(out.data_ptr()), sp,
                                ctypes.byref(ms), ctypes.byref(fmas))
        if rc != 0:
            raise RuntimeError(f"fp32_fma_probe failed ({rc})")
        return 2.0 * fmas.value / (ms.value * 1e-3) / 1e12, ms.value

    res = {}
    clk = ClockSampler(None)
    clk.start()
    for packed, name in ((0, "scalar"), (1, "packed_f32x2")):
        rate, ms = run(packed, 20_000)                        # warm-up and calibration
        iters = max(20_000, int(20_000 * 150.0 / max(ms, 1e-3)))   # ~150 ms per launch
        res[name] = max(run(packed, iters)[0] for _ in range(3))
    c = clk.stop()
    res["tflops"] = max(res["scalar"], res["packed_f32x2"])
    res["sm_mhz"] = c["sm_mhz"] if c else None
    res["sm_max_mhz"] = c["sm_max_mhz"] if c else None
    return res


def h2d_rate(Xh, dev, nbytes: int = 1 << 31):
    """GB/s of a host -> device copy of the first `nbytes` of the pinned host
    tensor Xh into a fresh device buffer (best of three, CUDA events on a
    private stream; untimed diagnostic beside the end-to-end number).  None
    if the copy cannot be made."""
    import torch
    try:
        flat = Xh.reshape(-1).view(torch.uint8)
        nbytes = min(nbytes, flat.numel())
        src = flat[:nbytes]
        dst = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        s = torch.cuda.Stream(dev)
        best = None
        with torch.cuda.stream(s):
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                dst.copy_(src, non_blocking=True)
                e1.record(s)
                e1.synchronize()
                gbs = nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
                best = gbs if best is None else max(best, gbs)
        del dst
        return best
    except Exception:
        return None


def select_loop_ceiling(dev, stream, peak):
    """The inner loop of the small-d distance kernel (d = 8, two points per
    thread, centers as interleaved pairs in shared memory) timed alone by the
    probe library: with the kernel's packed-key top-2, and with one minimum
    per center pair instead (loads and FMAs only).  TFLOP/s of each (2 flop
    per FMA, best of three launches) and as a fraction of `peak`; None if the
    probe library cannot be loaded."""
    import ctypes
    import torch
    path = os.path.join(ROOT, "paper_1108_1351_gb300", "libfp32peak.so")
    try:
        lib = ctypes.CDLL(path)
        fn = lib.fp32_select_probe
    except (OSError, AttributeError):
        return None
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)]
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 4
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    sp = ctypes.c_void_p(stream.cuda_stream)

    def run(mode, iters):
        ms, fmas = ctypes.c_float(), ctypes.c_double()
        rc = fn(mode, blocks, iters, ctypes.c_void_p(out.data_ptr()), sp, ctypes.byref(ms),
                ctypes.byref(fmas))
        if rc != 0:
            raise RuntimeError(f"fp32_select_probe failed ({rc})")
        return 2.0 * fmas.value / (ms.value * 1e-3) / 1e12, ms.value

    res = {"loop": "d = 8, 2 points per thread, 32 centers per chunk, no global memory"}
    for mode, name in ((0, "with_top2"), (1, "fma_only")):
        rate, ms = run(mode, 200)                              # warm-up and calibration
        iters = max(200, int(200 * 50.0 / max(ms, 1e-3)))     # ~50 ms per launch
        best = max(run(mode, iters)[0] for _ in range(3))
        res[name] = {"tflops": best, "frac": best / peak if peak else None}
    return res


def roofline_of(form: str, d: int, k: int, prof, clk, p32=None):
    """Roofline entry of the distance kernel the fit ran (the dominant kernel):
    algorithmic FLOP = 2 N k d per launch (the cross term only), achieved =
    their sum over the profiled launches / their summed CUDA-event time.  The
    CUDA-core forms are measured against the FP32 FMA peak of this GPU
    (fp32_peak, when given) with the unit-count figure beside it."""
    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    achieved = prof.assign_flops / (prof.assign_ms * 1e-3) / 1e12 if prof.assign_ms > 0 else None
    if form in ("bf16", "fp16"):
        kernel, bound = "assign_bf16", "tensor"
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
        peak_source = f"{src} bf16_tflops_sustained (kernel timed inside a long fit)"
        if form == "fp16":
            # the single-pass instantiation (its time includes the split-BF16
            # second pass over the rows it leaves undecided)
            nc = 256 if k >= 512 else (128 if k > 64 else 64)
            kernel = f"assign_bf16<{nc},1>"
            peak_source += "; dense FP16 and BF16 tensor rates are equal (nominal)"
    elif form == "tf32x3":
        kernel, bound = "assign_tc32", "tensor"
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))) * TF32_PER_BF16
        peak_source = f"{src} bf16_tflops_sustained x nominal TF32/BF16 ratio 1.1/2.25"
    else:
        kernel = f"assign_small<{d}>" if d <= 16 else "assign_large"
        bound = "alu"
        derived = 2.0 * FP32_LANES_PER_SM * SM_COUNT_GB300 * sm_max * 1e6 / 1e12
        if p32 and p32.get("tflops"):
            peak = p32["tflops"]
            peak_source = (f"measured: FP32 FMA probe on this GPU ({p32['scalar']:.1f} TFLOP/s "
                           f"scalar, {p32['packed_f32x2']:.1f} packed f32x2, SM clock "
                           f"{p32['sm_mhz']} MHz); derived {derived:.1f} = {SM_COUNT_GB300} SMs x "
                           f"{FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz")
        else:
            peak = derived
            peak_source = (f"derived: {SM_COUNT_GB300} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                           f"{sm_max:.0f} MHz ({src} max clock)")
    roof = {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic_of(kernel, prof, d), "peak_source": peak_source,
            "kernel_ms_avg": prof.assign_ms / max(1, prof.assign_launches),
            "kernel_launches": prof.assign_launches,
            "achieved_hbm_gbs": prof.assign_bytes / (prof.assign_ms * 1e-3) / 1e9
            if prof.assign_ms > 0 else None,
            "hbm_peak_gbs": peaks.get("hbm_gbs")}
    if achieved and bound == "alu" and clk and clk.get("sm_mhz"):
        roof["frac_at_observed_clock"] = achieved / (peak * clk["sm_mhz"] / sm_max)
    return roof


def traffic_of(kernel: str, prof, d: int):
    """DRAM bytes per launch of `kernel` from its committed ncu summary
    (profiles/<kernel>*.md lines 'traffic-per-point: <kernel> <bytes> <sha256 of
    the kernel source>'), scaled by the points of an average timed launch; None
    when there is no summary or the kernel source changed since the capture."""
    import glob
    import hashlib
    base = kernel.split("<")[0]
    src = {"assign_small": "assign_fp32.cu", "assign_large": "assign_fp32.cu",
           "assign_bf16": "assign_bf16.cu", "assign_tc32": "assign_tc32.cu"}.get(base)
    if not src or prof.assign_launches == 0:
        return None
    path = os.path.join(ROOT, "paper_1108_1351_gb300", "csrc", src)
    try:
        with open(path, "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(f) as fh:
            for ln in fh:
                parts = ln.strip().strip("`").split()
                if len(parts) == 4 and parts[0] == "traffic-per-point:" and parts[1] == kernel:
                    if parts[3] != sha:
                        return None
                    # assign_bytes counts 4 d bytes per point of every timed launch
                    points = prof.assign_bytes / (4.0 * d) / max(1, prof.assign_launches)
                    return float(parts[2]) * points
    return None


def reduce_over_ranks(ms: float, work: float, ws: int, device):
    """(max over ranks of the elapsed ms, sum over ranks of the work); the
    identity at one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def cpu_baseline(X_host, cfg, budget_s: float = 12.0, budget_1core_s: float = 4.0):
    """The oracle as it stands, timed on the host cores: Lloyd steps on the
    first rows of the same data until ~budget_s of CPU work on all cores, then
    ~budget_1core_s on one core (on proportionally fewer rows)."""
    import numpy as np
    import oracle
    oracle.build()
    k, d = cfg["k"], cfg["d"]
    nt = max(1, oracle.max_threads())

    def timed_steps(rows, threads, budget):
        Xs = np.ascontiguousarray(X_host[:rows])
        C = Xs[:k].astype(np.float64)
        evals, t, steps = 0, 0.0, 0
        while t < budget:
            t0 = time.perf_counter()
            C, lab, J, sh, em = oracle.lloyd_step(Xs, C, nthreads=threads)
            t += time.perf_counter() - t0
            evals += rows * k
            steps += 1
        return evals / t, steps, t

    rows = min(len(X_host), 2_000_000)
    v, steps, t = timed_steps(rows, nt, budget_s)
    rows1 = min(len(X_host), max(k, rows // nt))
    v1, steps1, t1 = timed_steps(rows1, 1, budget_1core_s)
    return {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{steps} FP64 Lloyd steps on the first {rows} rows of the workload "
                      f"(d={d}, k={k}), {t:.1f} s",
            "one_core": {"value": v1, "unit": UNIT, "cores": 1,
                         "sample": f"{steps1} FP64 Lloyd steps on the first {rows1} rows, "
                                   f"{t1:.1f} s"}}


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
    sharded = ws > 1 and args.parallelism == "sharded"
    if sharded:
        # rank r's rows [r n, (r + 1) n) of one data set: the same mixture,
        # its own sample stream (rank 0's block is the single-GPU workload)
        X = _gen(cfg, dev, cfg["seed"], sample_seed=cfg["seed"] + 7919 * rank)
    else:
        X = _gen(cfg, dev, cfg["seed"] + rank)
    torch.cuda.synchronize()
    centers = torch.empty(k, d, dtype=torch.float64, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def one(profile=None):
        if sharded and profile is None:
            return km.fit_data_parallel(X, rank * n, ws * n, k, cfg["f"], cfg["seed"], cfg["tol"],
                                        cfg["max_iter"], precision=args.precision,
                                        profile=launch_counter)
        # the profiled fits of a sharded run time the same kernel on one
        # rank's block (the launch a rank makes per iteration)
        return km.fit(X, k, cfg["f"], cfg["seed"] + (0 if sharded else rank), cfg["tol"],
                      cfg["max_iter"], centers_out=centers, labels_out=labels, stream=stream,
                      profile=profile, precision=args.precision)

    launch_counter = km.Profile()

    p32 = fp32_peak(dev, stream) if rank == 0 else None
    for _ in range(args.warmup):
        one()
    launch_counter.kernel_launches = 0             # sharded: count the timed fits only
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    clocks.start()
    results = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rng = torch.cuda.nvtx.range_start("timed")     # lets ncu select the timed launches
    e0.record(stream)
    for _ in range(args.steps):
        results.append(one())                      # the default path: graph-captured stage loops
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_end(rng)
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    timed_launches = int(launch_counter.kernel_launches)
    evals = sum(r.distance_evals for r in results)
    if sharded:
        # every rank reports the global count of one fit: count it once
        ms_max, total_evals = reduce_over_ranks(ms, evals / ws, ws, dev)
    else:
        ms_max, total_evals = reduce_over_ranks(ms, evals, ws, dev)

    # the distance kernel's own time for the roofline: separate profiled fits
    # (host-driven loop, CUDA events around every launch of the fused
    # distance kernel on the call's stream), after the timed region
    prof = km.Profile()
    prng = torch.cuda.nvtx.range_start("profiled")   # the launch list's ncu range
    for _ in range(args.profile_fits):
        one(prof)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_end(prng)

    # end to end through the same C-ABI call with HOST buffers
    e2e = None
    if args.e2e_steps > 0 and sharded:
        # each step: this rank's block host -> device, the sharded fit, its
        # labels device -> host (the same rows as the device-resident run)
        Xh = torch.empty((n, d), dtype=torch.float32, pin_memory=True)
        Xh.copy_(X)
        lh = torch.empty((n,), dtype=torch.int32, pin_memory=True)
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_evals = 0
        for _ in range(args.e2e_steps):
            X.copy_(Xh, non_blocking=True)
            r = one()
            lh.copy_(r.labels)
            e_evals += r.distance_evals
        torch.cuda.synchronize()
        te_ms, ee = reduce_over_ranks(1e3 * (time.perf_counter() - t0), e_evals / ws, ws, dev)
        e2e = {"value": ee / (te_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": n * d * 4, "d2h_bytes_per_step": n * 4,
               "per": "rank (each rank copies its own block)",
               "steps": args.e2e_steps, "ms_per_step": te_ms / args.e2e_steps}
        Xh_host = Xh[: min(n, 2_000_000)].numpy()
    elif args.e2e_steps > 0:
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
        te_ms, ee = reduce_over_ranks(1e3 * (time.perf_counter() - t0), e_evals, ws, dev)
        e2e = {"value": ee / (te_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": n * d * 4, "d2h_bytes_per_step": n * 4 + k * d * 8,
               "steps": args.e2e_steps, "ms_per_step": te_ms / args.e2e_steps,
               "h2d_gbs_measured": h2d_rate(Xh, dev)}
        Xh_host = Xh.numpy()
    else:
        Xh_host = X[: min(n, 2_000_000)].cpu().numpy()

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0
    r0 = results[-1]
    roofline = roofline_of(r0.precision_used, d, k, prof, clk, p32)
    roofline["measured"] = (f"{args.profile_fits} profiled fits after the timed region, CUDA "
                            f"events around each launch of the distance kernel")
    if roofline.get("kernel") == "assign_small<8>":
        # what the kernel's own inner loop reaches with nothing else around it
        roofline["loop_ceiling"] = select_loop_ceiling(dev, stream, roofline.get("peak"))
    line = {
        "metric": METRIC, "value": total_evals / (ms_max * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.config, "n": n, "d": d, "k": k, "subset_fraction": cfg["f"],
                   "tol": cfg["tol"], "max_iter": cfg["max_iter"], "seed": cfg["seed"],
                   "parallelism": ("sharded" if sharded else "replicas") if ws > 1 else "single",
                   "rows_per_gpu": n, "rows_total": n * ws if sharded else n,
                   "l2": "inputs larger than L2 (X is %.1f GB)" % (n * d * 4 / 1e9)
                   if n * d * 4 > 2e8 else "inputs smaller than L2"},
        "time_to_converge_s": (ms_max / args.steps) / 1e3,
        "time_to_converge_note": ("one whole fit to its stopping rule (tol %g, max_iter %d per "
                                  "stage); fit.converged_* say whether tol or max_iter ended "
                                  "each stage" % (cfg["tol"], cfg["max_iter"])),
        # each timed call's own wall time (host clock inside the library; rank 0)
        "time_to_converge_median_s": statistics.median(r.seconds for r in results) if results else None,
        "fit": {"J": r0.J, "iters_fast": r0.iters_fast, "iters_slow": r0.iters_slow,
                "converged_fast": r0.converged_fast, "converged_slow": r0.converged_slow,
                "rechecked_points": r0.rechecked_points, "distance_evals": r0.distance_evals,
                "subset_size": r0.subset_size, "empty_clusters": r0.empty_clusters},
        # kernels per fit (the profiled fits run the same kernels as the graph
        # body; a sharded fit counts its own session's launches) x steps
        "gpu_launches": (timed_launches if sharded else
                         int(prof.kernel_launches) // max(1, args.profile_fits) * args.steps),
        "fp32_peak_probe": p32,
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


SERVE = dict(rate=200.0, duration=60.0, seed=0, f=0.1, tol=1e-6, max_iter=100)


def _serve_trace(trace, srv, dev, *, drain_cap: float):
    """Replay the arrival trace against one server: a client thread submits each
    job at its arrival time as a lazy job (its points are generated on the
    device only when the server admits it, so waiting jobs hold no device
    memory); the main thread collects finished jobs.  Latency = completion -
    scheduled arrival, both on the server's clock.  Jobs still unfinished
    drain_cap seconds after the last arrival are reported as censored
    (latency >= their age)."""
    from paper_1108_1351_gb300 import synth

    outstanding = {}            # ticket -> (job spec, scheduled arrival)
    lock = threading.Lock()
    state = {"submitted": 0, "late": 0.0, "error": None}
    stop = threading.Event()
    start = srv.now() + 0.5

    def make_for(js):
        def make(X):
            X.copy_(synth.iso_gaussian_mixture(js.n, js.d, js.k, js.seed, lo=-20.0, hi=20.0,
                                               device=dev))
        return make

    def client():
        try:
            for js in trace:
                t_sched = start + js.t_arrival
                while not stop.is_set():
                    now = srv.now()
                    if now >= t_sched:
                        break
                    time.sleep(min(0.002, t_sched - now))
                if stop.is_set():
                    return
                state["late"] = max(state["late"], srv.now() - t_sched)
                with lock:      # recorded before the collector can see it finish
                    t = srv.submit_lazy(js.n, js.d, js.k, SERVE["f"], js.seed, SERVE["tol"],
                                        SERVE["max_iter"], make_for(js))
                    outstanding[t] = (js, t_sched)
                    state["submitted"] += 1
        except Exception as e:      # reported by the collector
            state["error"] = repr(e)

    th = threading.Thread(target=client, daemon=True)
    th.start()
    done = []
    last_arrival = start + (trace[-1].t_arrival if trace else 0.0)
    while True:
        sv = srv.wait_any(0.05)          # blocks in the library, without the GIL
        if sv is not None:
            with lock:
                js, t_sched = outstanding.pop(sv.ticket)
            done.append((js, t_sched, sv))
            continue
        if state["error"]:
            raise RuntimeError(state["error"])
        if not th.is_alive() and not outstanding and state["submitted"] == len(trace):
            break
        if srv.now() > last_arrival + drain_cap:
            break
        time.sleep(0.002)
    t_end = srv.now()
    stop.set()
    th.join(timeout=120)
    with lock:
        censored = [t_end - t_sched for (js, t_sched) in outstanding.values()]
    never = len(trace) - state["submitted"]
    return done, censored, never, start, t_end, state["late"]


def _latency_summary(done, censored, never, start, t_end):
    import numpy as np
    lat = [sv.t_done - t_sched for (js, t_sched, sv) in done if sv.status == 0]
    fails = sum(1 for (_, _, sv) in done if sv.status != 0)
    cens = list(censored) + [t_end - start] * never
    allv = np.asarray(lat + cens, dtype=np.float64)
    evals = sum(sv.result.distance_evals for (_, _, sv) in done if sv.status == 0)
    span = max((sv.t_done for (_, _, sv) in done), default=t_end) - start
    done_lat = np.asarray(lat, dtype=np.float64)
    failures = [{"n": js.n, "d": js.d, "k": js.k, "seed": js.seed, "status": sv.status}
                for (js, _, sv) in done if sv.status != 0][:20]
    return {"completed": len(lat), "failed": fails, "failures": failures, "censored": len(cens),
            "jobs_per_s": len(lat) / span if span > 0 else None,
            "completed_p50_s": float(np.percentile(done_lat, 50)) if done_lat.size else None,
            "completed_p99_s": float(np.percentile(done_lat, 99)) if done_lat.size else None,
            "p50_s": float(np.percentile(allv, 50)) if allv.size else None,
            "p99_s": float(np.percentile(allv, 99)) if allv.size else None,
            "mean_s": float(allv.mean()) if allv.size else None,
            "max_s": float(allv.max()) if allv.size else None,
            "distance_evals_per_s": evals / span if span > 0 else None,
            "span_s": span}


def run_serve(args):
    """Serving workload: Poisson arrivals of jobs of mixed n, d, k, served by the
    continuous-batching server (args.serve_slots slots, AUTO form) and, on the
    same trace and under the same admission policy, one job at a time in the
    plain FP32 form.  Two traces: an overload trace (args.rate jobs/s for
    args.duration s; unfinished jobs are reported as censored) and a
    sustainable trace at args.stable_frac of the one-at-a-time arm's measured
    capacity (its completions per second under overload, an unbiased FIFO
    sample of the job mix), drained completely so that p50 / p99 cover every
    job."""
    import torch
    import paper_1108_1351_gb300 as km
    from paper_1108_1351_gb300 import synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    km.load()
    free, total = torch.cuda.mem_get_info(dev)
    budget = int(free * 0.8)
    # warm-up: one small job of each dimension through a throwaway server
    with km.Server(hbm_budget=budget, max_slots=2) as srv:
        for d in (4, 16, 64, 128):
            X = synth.iso_gaussian_mixture(50_000, d, 32, 99, device=dev)
            srv.wait(srv.submit(X, 32, 0.1, 99, 1e-6, 20))
    # the served arm's stage loops: graphs with device-side while conditions
    # ("graph") or driven from the worker threads ("host"); the one-at-a-time
    # arm runs each job alone, as graphs
    arms = (("served", args.serve_slots, "auto", args.serve_loop == "graph"),
            ("one_at_a_time_fp32", 1, "fp32", True))

    def run_trace(trace, drain_cap):
        out = {}
        for name, slots, prec, graph in arms:
            with km.Server(hbm_budget=budget, max_slots=slots, precision=prec,
                           policy=args.policy, aging_s=args.aging, use_graph=graph) as srv:
                done, censored, never, start, t_end, late = _serve_trace(
                    trace, srv, dev, drain_cap=drain_cap)
                summ = _latency_summary(done, censored, never, start, t_end)
                st = srv.stats()
            summ.update({"slots": slots, "precision": prec, "policy": args.policy,
                         "stage_loops": "graph" if graph else "host",
                         "kernel_launches": st["kernel_launches"],
                         "hbm_peak_gb": st["hbm_peak"] / 1e9, "client_max_lag_s": late})
            out[name] = summ
        return out

    clocks = ClockSampler(None)
    clocks.start()
    over_trace = synth.arrival_trace(rate=args.rate, duration=args.duration,
                                     seed=SERVE["seed"] + rank)
    over = run_trace(over_trace, args.drain_cap)
    capacity = over["one_at_a_time_fp32"]["jobs_per_s"] or 1.0
    stable_rate = args.stable_frac * capacity
    stable_trace = synth.arrival_trace(rate=stable_rate, duration=args.stable_duration,
                                       seed=SERVE["seed"] + 1 + rank)
    stable = run_trace(stable_trace, args.stable_drain_cap)
    clk = clocks.stop()
    if rank != 0:
        return 0
    srv_s = stable["served"]
    one_s = stable["one_at_a_time_fp32"]
    line = {
        "metric": "serving: p50 latency over every job at a sustainable Poisson arrival rate "
                  "(p99, saturated jobs/s and distance evals/s beside)",
        "value": srv_s["p50_s"], "unit": "s", "n_gpus": ws, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * srv_s["span_s"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": "serve", "n": "log-U[1e4, 2e7]", "d": [4, 16, 64, 128],
                   "k": "log-U[4, 1024]", "subset_fraction": SERVE["f"], "tol": SERVE["tol"],
                   "max_iter": SERVE["max_iter"], "hbm_budget_gb": budget / 1e9,
                   "policy": args.policy,
                   "overload": {"rate_per_s": args.rate, "duration_s": args.duration,
                                "jobs": len(over_trace), "drain_cap_s": args.drain_cap},
                   "stable": {"rate_per_s": stable_rate, "duration_s": args.stable_duration,
                              "jobs": len(stable_trace),
                              "rate_rule": "%.2f x the one-at-a-time arm's completions per "
                                           "second under overload" % args.stable_frac}},
        "stable": {"served": srv_s, "one_at_a_time_fp32": one_s,
                   "p50_ratio_one_over_served": (one_s["p50_s"] / srv_s["p50_s"])
                   if srv_s["p50_s"] else None,
                   "p99_ratio_one_over_served": (one_s["p99_s"] / srv_s["p99_s"])
                   if srv_s["p99_s"] else None},
        "overload": over,
        "saturated_jobs_per_s": {"served": over["served"]["jobs_per_s"],
                                 "one_at_a_time_fp32": capacity},
        "gpu_launches": int(srv_s["kernel_launches"]), "roofline": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


SWEEP = dict(fractions=(0.01, 0.10, 0.15, 0.20, 0.30, 0.40),
             tols=(1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10), max_iter=500,
             seed=0)


def run_sweep(args):
    """Normal (single-stage) k-means vs the two-stage method (Section 6, Tables
    2-3, Fig. 13) on a synthetic stand-in: for each stopping tolerance, normal
    k-means is Lloyd on S_n from the same k initial data points the two-stage
    fit draws (kmeans2_fit with start_stage = 1), and the two-stage fit runs for
    each subset fraction; time-to-converge and final J side by side."""
    import torch
    import paper_1108_1351_gb300 as km
    from paper_1108_1351_gb300 import synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    km.load()
    n, d, k = args.sweep_n, args.sweep_d, args.sweep_k
    X = synth.aniso_gaussian_noise(n, d, k, SWEEP["seed"] + rank, device=dev, chunk=1 << 24)
    stream = torch.cuda.current_stream(dev)
    seed = SWEEP["seed"] + rank

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    rows = []
    for f in SWEEP["fractions"]:
        sub, pos = km.sample(n, k, f, seed)
        C0 = X[sub[pos]].double()          # the two-stage fit's own initial centers
        for tol in SWEEP["tols"]:
            normal, t_n = timed(lambda: km.fit(X, k, f, seed, tol, SWEEP["max_iter"],
                                               init_centers=C0, start_stage=1, stream=stream))
            two, t_2 = timed(lambda: km.fit(X, k, f, seed, tol, SWEEP["max_iter"], stream=stream))
            rows.append({"subset_fraction": f, "tol": tol,
                         "normal": {"s": t_n, "J": normal.J, "iters": normal.iters_slow},
                         "two_stage": {"s": t_2, "J": two.J, "iters_fast": two.iters_fast,
                                       "iters_slow": two.iters_slow},
                         "speedup": t_n / t_2 if t_2 > 0 else None,
                         "J_rel_diff": (two.J - normal.J) / normal.J if normal.J else None})
    if rank != 0:
        return 0
    best = max(r["speedup"] for r in rows)
    line = {"metric": "two-stage vs normal k-means: time-to-converge speedup (J beside)",
            "value": best, "unit": "x (best over the sweep)", "n_gpus": ws, "steps": 1,
            "warmup": 2, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep", "n": n, "d": d, "k": k,
                       "generator": "anisotropic Gaussian mixture + 2% noise",
                       "max_iter": SWEEP["max_iter"]},
            "sweep": rows, "roofline": None}
    print(json.dumps(line), flush=True)
    return 0


def run_sharded(args, cfg):
    """The data-parallel form on one GPU: the default workload split into
    --shards row blocks, each run as a rank (own sums, labels and near-tie
    list, replicated centers) with the integer partials all-reduced in rank
    order every iteration (kmeans2_fit_sharded); the unsharded fit beside it."""
    import torch
    import paper_1108_1351_gb300 as km

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    km.load()
    X = _gen(cfg, dev, cfg["seed"] + rank)
    stream = torch.cuda.current_stream(dev)
    fargs = (cfg["k"], cfg["f"], cfg["seed"] + rank, cfg["tol"], cfg["max_iter"])

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r = fn()
        torch.cuda.synchronize()
        return r, (time.perf_counter() - t0) / args.steps

    clk = ClockSampler(None)
    clk.start()
    r, t = timed(lambda: km.fit_sharded(X, *fargs, args.shards, stream=stream))
    r1, t1 = timed(lambda: km.fit(X, *fargs, stream=stream))
    clocks = clk.stop()
    same = (r.J == r1.J and (r.iters_fast, r.iters_slow) == (r1.iters_fast, r1.iters_slow)
            and bool(torch.equal(r.labels, r1.labels)) and bool(torch.equal(r.centers, r1.centers)))
    t_ms, evals = reduce_over_ranks(1e3 * t, r.distance_evals, ws, dev)
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": evals / (t_ms * 1e-3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "sharded", "n": cfg["n"], "d": cfg["d"], "k": cfg["k"],
                       "ranks_on_one_gpu": args.shards,
                       "exchange": "int64 partials summed in rank order per iteration"},
            "time_to_converge_s": t_ms / 1e3, "unsharded_time_to_converge_s": t1,
            "identical_to_unsharded": same,
            "fit": {"J": r.J, "iters_fast": r.iters_fast, "iters_slow": r.iters_slow},
            "roofline": None, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_streamed(args, cfg):
    """Host-resident X streamed through the GPU each slow-stage iteration
    (kmeans2_fit_streamed), on the default workload held in pinned host
    memory, with the resident fit on the same data beside it."""
    import torch
    import paper_1108_1351_gb300 as km

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    km.load()
    n, d, k = cfg["n"], cfg["d"], cfg["k"]
    Xd = _gen(cfg, dev, cfg["seed"] + rank)
    Xh = torch.empty((n, d), dtype=torch.float32, pin_memory=True)
    Xh.copy_(Xd)
    args_fit = (k, cfg["f"], cfg["seed"] + rank, cfg["tol"], cfg["max_iter"])
    resident = km.fit(Xd, *args_fit, precision="fp32")
    torch.cuda.synchronize()
    del Xd
    torch.cuda.empty_cache()
    def timed(chunk):
        for _ in range(args.warmup):
            km.fit_streamed(Xh, *args_fit, chunk)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r = km.fit_streamed(Xh, *args_fit, chunk)
        torch.cuda.synchronize()
        return r, (time.perf_counter() - t0) / args.steps

    clk = ClockSampler(None)
    clk.start()
    r, t = timed(args.chunk_points)         # staged chunks through two device buffers
    rc, tc = timed(-1)                      # page-locked X read in place over the link
    clocks = clk.stop()
    same = all(x.J == resident.J and (x.iters_fast, x.iters_slow) ==
               (resident.iters_fast, resident.iters_slow) for x in (r, rc))
    t_ms, evals = reduce_over_ranks(1e3 * t, r.distance_evals, ws, dev)
    if rank != 0:
        return 0
    passes = r.iters_slow + 1                 # the max-|x| pass and every slow iteration
    line = {"metric": METRIC, "value": evals / (t_ms * 1e-3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "streamed", "n": n, "d": d, "k": k,
                       "X_host_gb": n * d * 4 / 1e9, "host_memory": "pinned",
                       "mode": "staged chunks", "chunk_points": args.chunk_points},
            "time_to_converge_s": t_ms / 1e3,
            "link_gb_per_s": passes * n * d * 4 / (t_ms * 1e-3) / 1e9,
            "in_place": {"time_to_converge_s": tc,
                         "link_gb_per_s": passes * n * d * 4 / tc / 1e9},
            "resident_time_to_converge_s": resident.seconds,
            "identical_to_resident": bool(same),
            "fit": {"J": r.J, "iters_fast": r.iters_fast, "iters_slow": r.iters_slow},
            "roofline": None, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


BATCH = dict(count=4096, seed=0, f=0.1, tol=1e-6, max_iter=100)


def run_batched(args):
    """Batched workload: many independent instances (n log-uniform in [1e3,
    1e6], d in {2, 8, 32, 64}, k uniform in [2, 256], Gaussian mixtures with
    means U[-20, 20]^d) fitted by one kmeans2_fit_batched call, and the same
    instances fitted one kmeans2_fit call at a time (FP32 form) as the
    baseline; a sample of instances is checked bit for bit between the two."""
    import numpy as np
    import torch
    import paper_1108_1351_gb300 as km
    from paper_1108_1351_gb300 import synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    km.load()
    dims = tuple(int(v) for v in args.batch_dims.split(",")) if args.batch_dims else (2, 8, 32, 64)
    specs = synth.instance_specs(args.instances, seed=BATCH["seed"] + rank * args.instances,
                                 dims=dims)
    Xs = [synth.instance_data(s, device=dev) for s in specs]
    torch.cuda.synchronize()
    ks = [s.k for s in specs]
    seeds = [s.seed for s in specs]
    stream = torch.cuda.current_stream(dev)

    prof = km.Profile()

    def batched(profile=None):
        return km.fit_batched(Xs, ks, BATCH["f"], seeds, BATCH["tol"], BATCH["max_iter"],
                              stream=stream, profile=profile)[0]

    for _ in range(args.warmup):
        res = batched()
    clocks = ClockSampler(None)
    clocks.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = batched()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    evals = sum(r.distance_evals for r in res)
    # one more call in the profiled (host-driven) mode: the distance kernels'
    # own time for the roofline entry, and the number of kernels a call launches
    torch.cuda.synchronize()
    tp0 = time.perf_counter()
    prng = torch.cuda.nvtx.range_start("profiled")   # the launch list's ncu range
    batched(prof)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_end(prng)
    prof_call_ms = 1e3 * (time.perf_counter() - tp0)
    launches = int(prof.kernel_launches)
    peaks, src = _peaks()
    derived = 2.0 * FP32_LANES_PER_SM * SM_COUNT_GB300 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e-6
    probe = fp32_peak(dev, stream)
    p32 = probe["tflops"] if probe else derived
    ach = prof.assign_flops / (prof.assign_ms * 1e-3) / 1e12 if prof.assign_ms > 0 else None
    roofline = {"bound": "alu", "kernel": "batch_assign<DC> (all dimension classes)",
                "achieved": ach, "peak": p32, "unit": "TFLOP/s",
                "frac": ach / p32 if ach else None, "traffic": None,
                "peak_source": ("measured: FP32 FMA probe on this GPU (%.1f TFLOP/s); derived "
                                "%.1f" % (p32, derived)) if probe else
                               f"derived: {SM_COUNT_GB300} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                               f"x max clock ({src})",
                "kernel_ms_per_call": prof.assign_ms,
                "call_ms_profiled": prof_call_ms}
    # baseline: the same instances, one kmeans2_fit at a time (plain FP32 form)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    singles = [km.fit(X, k, BATCH["f"], sd, BATCH["tol"], BATCH["max_iter"], precision="fp32",
                      stream=stream) for X, k, sd in zip(Xs, ks, seeds)]
    torch.cuda.synchronize()
    ms_single = 1e3 * (time.perf_counter() - t0)
    rng = np.random.default_rng(1)
    sample = rng.choice(len(specs), size=min(64, len(specs)), replace=False)
    same = all(torch.equal(res[i].labels, singles[i].labels) and res[i].J == singles[i].J and
               (res[i].iters_fast, res[i].iters_slow) == (singles[i].iters_fast, singles[i].iters_slow)
               for i in sample)
    ms_max, total_evals = reduce_over_ranks(ms, evals, ws, dev)
    if rank != 0:
        return 0
    npts = sum(s.n for s in specs)
    line = {
        "metric": METRIC, "value": total_evals / (ms_max * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batched", "instances": len(specs), "points": npts,
                   "n": "log-U[1e3, 1e6]", "d": list(dims), "k": "U[2, 256]",
                   "subset_fraction": BATCH["f"], "tol": BATCH["tol"],
                   "max_iter": BATCH["max_iter"],
                   "l2": "inputs larger than L2 (%.1f GB)" % (sum(s.n * s.d for s in specs) * 4e-9)},
        "time_to_converge_s": ms_max / 1e3,
        "one_at_a_time_fp32": {"time_to_converge_s": ms_single / 1e3,
                               "value": sum(r.distance_evals for r in singles) / (ms_single * 1e-3),
                               "speedup_of_batched": ms_single / ms_max},
        "sampled_instances_identical": bool(same), "sampled": int(len(sample)),
        "tile_shapes": {str(dd): km.batched_tile_shape(dd) for dd in dims},
        "gpu_launches": launches, "roofline": roofline, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="aniso8",
                    choices=sorted(CONFIGS) + ["serve", "batched", "sweep", "streamed", "sharded"])
    ap.add_argument("--shards", type=int, default=4,
                    help="sharded: ranks simulated on this GPU")
    ap.add_argument("--chunk-points", type=int, default=1 << 26,
                    help="streamed: rows per streamed chunk")
    ap.add_argument("--sweep-n", type=int, default=10_000_000, help="sweep: points")
    ap.add_argument("--sweep-d", type=int, default=12, help="sweep: dimensions")
    ap.add_argument("--sweep-k", type=int, default=16, help="sweep: clusters")
    ap.add_argument("--instances", type=int, default=BATCH["count"],
                    help="batched: number of independent instances")
    ap.add_argument("--batch-dims", default="",
                    help="batched: comma-separated dimensions to draw from (default 2,8,32,64)")
    ap.add_argument("--duration", type=float, default=30.0,
                    help="serve: seconds of Poisson arrivals of the overload trace")
    ap.add_argument("--rate", type=float, default=SERVE["rate"],
                    help="serve: arrivals per second of the overload trace")
    ap.add_argument("--stable-frac", type=float, default=0.8,
                    help="serve: sustainable rate as a share of the one-at-a-time capacity")
    ap.add_argument("--stable-duration", type=float, default=60.0,
                    help="serve: seconds of arrivals of the sustainable trace")
    ap.add_argument("--stable-drain-cap", type=float, default=600.0,
                    help="serve: seconds after the last sustainable arrival before giving up")
    ap.add_argument("--policy", default="fifo", choices=["fifo", "shortest"],
                    help="serve: admission policy of both arms")
    ap.add_argument("--serve-slots", type=int, default=8, help="serve: jobs running at once")
    ap.add_argument("--serve-loop", default="host", choices=["graph", "host"],
                    help="serve: the served arm's stage loops (while-graphs or host-driven)")
    ap.add_argument("--aging", type=float, default=30.0,
                    help="serve: seconds after which a waiting job is admitted before smaller ones")
    ap.add_argument("--drain-cap", type=float, default=30.0,
                    help="serve: seconds after the last overload arrival before unfinished jobs "
                         "are censored")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--profile-fits", type=int, default=2,
                    help="profiled fits after the timed region (roofline kernel times)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--parallelism", default="sharded", choices=["sharded", "replicas"],
                    help="N > 1: one row-sharded fit over NCCL, or one replica per rank")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16", "fp16", "tf32x3"],
                    help="distance-kernel form (every form returns the same labels)")
    args = ap.parse_args()
    if args.config == "sharded":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the sharded workload compares "
                              "with the unsharded GPU fit in the same line"}))
            return 0
        return run_sharded(args, CONFIGS["aniso8"])
    if args.config == "streamed":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the streamed workload compares "
                              "with the resident GPU fit in the same line"}))
            return 0
        return run_streamed(args, CONFIGS["aniso8"])
    if args.config == "sweep":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the sweep compares two GPU "
                              "forms of the method with each other"}))
            return 0
        return run_sweep(args)
    if args.config == "batched":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload's "
                              "baseline is the one-at-a-time FP32 form in the same line"}))
            return 0
        return run_batched(args)
    if args.config == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serving workload has no "
                              "oracle arm; its baseline is the one-job-at-a-time FP32 form"}))
            return 0
        return run_serve(args)
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)
    return run_ours(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
