"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

Under torchrun every rank fits its own replica ("replicas only": the fit has
no cross-rank exchange), the reported time is the slowest rank's and the work
is the sum over ranks; only rank 0 prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms, work = bench.reduce_over_ranks(10.0 * (rank + 1), 100 * (rank + 1), ws, "cpu")
        out.put((rank, ms, work))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, ms, work in got:
        assert ms == 20.0          # slowest rank
        assert work == 300.0       # sum of the ranks' work


def test_reduce_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, 7, 1, "cpu") == (12.5, 7.0)


def test_reference_arm_rank_nonzero_exits_silently():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0", "--config", "gauss2d"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_rank0_prints_one_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--config", "gauss2d"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_baseline_reports_all_cores_and_one_core():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    X = np.random.default_rng(0).standard_normal((20_000, 4)).astype(np.float32)
    rec = bench.cpu_baseline(X, dict(k=8, d=4), budget_s=0.2, budget_1core_s=0.1)
    assert rec["kind"] == "oracle" and rec["value"] > 0 and rec["cores"] >= 1
    one = rec["one_core"]
    assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == rec["unit"]


# ---------------------------------------------------------------- data-parallel driver
# fit_data_parallel drives one shard per rank and turns each exchange the
# shard asks for into one all_reduce over the group.  On CPU the CUDA shard is
# replaced by a stand-in that speaks the same protocol (initial centers as an
# FP64 sum with -0.0 where a rank does not hold the row, max |x| as an int64
# max, per-iteration integer partials as an int64 sum) and assigns with the
# oracle.  The data lie on a 1/8 grid, so its integer sums (x * 8) are exact
# and the means equal the oracle's FP64 means bit for bit.

class OracleShard:
    SCALE = 8.0

    def __init__(self, X_local, row0, n_total, k, f, seed, tol, max_iter, **kw):
        import numpy as np
        import torch
        import oracle
        self.np, self.torch, self.oracle = np, torch, oracle
        self.X = np.asarray(X_local, dtype=np.float32)
        self.n_local, self.d = self.X.shape
        self.k, self.tol, self.max_iter = k, tol, max_iter
        sub, self.pos = oracle.sample(n_total, k, f, seed)
        self.a = int(np.searchsorted(sub, row0))
        b = int(np.searchsorted(sub, row0 + self.n_local))
        self.Xs = self.X[sub[self.a:b] - row0]
        self.buf = torch.zeros(2 * k * self.d + k, dtype=torch.int64)
        self.phase, self.stage, self.iters, self.maxabs = "start", 0, [0, 0], []
        self.labels = np.zeros(0, np.int32)

    def _stage_X(self):
        return self.Xs if self.stage == 0 else self.X

    def _begin(self):
        X = self._stage_X()
        self.buf[0] = int(self.np.abs(X).max() * self.SCALE) if len(X) else 0
        self.phase = "maxabs"
        return "max", self.buf[:1]

    def _pass(self):
        np, k, d = self.np, self.k, self.d
        X = self._stage_X()
        lab = self.oracle.assign(X, self.C)[0] if len(X) else np.zeros(0, np.int32)
        self.labels = lab
        S = np.zeros((k, d), np.int64)
        np.add.at(S, lab, np.rint(X * self.SCALE).astype(np.int64))
        N = np.bincount(lab, minlength=k).astype(np.int64)
        self.buf[:k * d] = self.torch.from_numpy(S.ravel())
        self.buf[k * d:k * d + k] = self.torch.from_numpy(N)
        self.phase = "iter"
        return "sum", self.buf[:k * d + k]

    def advance(self):
        np, k, d = self.np, self.k, self.d
        kd = k * d
        f64 = self.buf.view(self.torch.float64)
        if self.phase == "start":
            C = np.full((k, d), -0.0)
            p = self.pos - self.a
            own = (p >= 0) & (p < len(self.Xs))
            C[own] = self.Xs[p[own]]
            f64[:kd] = self.torch.from_numpy(C.ravel())
            self.phase = "init"
            return "sum", f64[:kd]
        if self.phase == "init":
            self.C = f64[:kd].numpy().reshape(k, d).copy()
            return self._begin()
        if self.phase == "maxabs":
            self.maxabs.append(int(self.buf[0]))
            return self._pass()
        if self.phase == "iter":
            tot = self.buf[:kd + k].numpy()
            S = tot[:kd].reshape(k, d).astype(np.float64) / self.SCALE
            N = tot[kd:]
            Cn = np.where(N[:, None] > 0, S / np.maximum(N, 1)[:, None], self.C)
            shift = float(np.sqrt(((Cn - self.C) ** 2).sum(axis=1).max()))
            self.C = Cn
            self.iters[self.stage] += 1
            if shift <= self.tol or self.iters[self.stage] >= self.max_iter:
                if self.stage == 0:
                    self.stage = 1
                    return self._begin()
                self.phase = "done"
                return None
            return self._pass()
        return None

    def result(self):
        return dict(labels=self.labels, centers=self.C, iters=tuple(self.iters),
                    maxabs=list(self.maxabs))

    def close(self):
        pass


def _grid_data():
    import numpy as np
    rng = np.random.default_rng(4)
    n, d, k = 3_001, 3, 5
    mu = rng.integers(-40, 40, size=(k, d))
    comp = rng.integers(0, k, size=n)
    X = np.round((mu[comp] + 2.0 * rng.standard_normal((n, d))) * 8) / 8
    return X.astype(np.float32), k


def _dp_rank(rank, ws, port, bounds, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1108_1351_gb300.binding import fit_data_parallel
    from tests.test_multirank_cpu import OracleShard, _grid_data
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        X, k = _grid_data()
        lo, hi = bounds[rank], bounds[rank + 1]
        r = fit_data_parallel(X[lo:hi], lo, len(X), k, 0.2, 7, 1e-9, 100,
                              shard_factory=OracleShard)
        out.put((rank, r["labels"].tolist(), r["centers"].tolist(), r["iters"], r["maxabs"]))
    finally:
        dist.destroy_process_group()


def test_data_parallel_driver_gloo_world2():
    import numpy as np
    import oracle
    oracle.build()
    X, k = _grid_data()
    bounds = (0, 1_234, len(X))
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_dp_rank, args=(r, 2, port, bounds, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    o = oracle.fit(X, k, 0.2, 7, 1e-9, 100)
    labels = np.concatenate([np.asarray(g[1], np.int32) for g in got])
    assert np.array_equal(labels, o["labels"])
    for _, _, centers, iters, maxabs in got:
        assert np.array_equal(np.asarray(centers), o["centers"])      # replicated, exact
        assert iters == (o["iters_fast"], o["iters_slow"])
        sub, _ = oracle.sample(len(X), k, 0.2, 7)
        assert maxabs == [int(np.abs(X[sub]).max() * 8), int(np.abs(X).max() * 8)]


def test_clock_summary_of_nvidia_smi_rows():
    sys.path.insert(0, ROOT)
    import bench
    rows = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "garbage line",                                                               # skipped
    ]
    s = bench.ClockSampler.summarize(rows)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    assert bench.ClockSampler.summarize(["x"]) is None
    hot = rows[:1] + ["0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active"]
    assert bench.ClockSampler.summarize(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_traffic_line_is_used_only_for_the_source_it_was_measured_on(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import hashlib
    import bench
    (tmp_path / "paper_1108_1351_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "paper_1108_1351_gb300" / "csrc" / "assign_bf16.cu"
    src.write_text("// kernel v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "x.md").write_text(f"`traffic-per-point: assign_bf16 520.0 {sha}`\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))

    class Prof:
        assign_launches = 4
        assign_bytes = 4 * (4.0 * 128 * 1000)      # four launches of 1000 points, d = 128

    assert bench.traffic_of("assign_bf16", Prof, 128) == 520.0 * 1000
    assert bench.traffic_of("assign_small<8>", Prof, 8) is None       # no line for it
    src.write_text("// kernel v2\n")                                   # source changed since
    assert bench.traffic_of("assign_bf16", Prof, 128) is None


def test_committed_traffic_lines_match_the_kernel_sources():
    """Every 'traffic-per-point:' line under profiles/ is keyed to the sha256 of
    the kernel source it was captured on, and the bench drops a line whose
    source has changed since.  The committed lines must therefore match the
    committed sources, or the bench's roofline would report no traffic."""
    import glob
    import hashlib
    src_of = {"assign_small": "assign_fp32.cu", "assign_large": "assign_fp32.cu",
              "assign_bf16": "assign_bf16.cu", "assign_tc32": "assign_tc32.cu"}
    found = 0
    for md in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(md) as fh:
            for line in fh:
                parts = line.strip().strip("`").split()
                if len(parts) != 4 or parts[0] != "traffic-per-point:":
                    continue
                found += 1
                src = src_of[parts[1].split("<")[0]]
                with open(os.path.join(ROOT, "paper_1108_1351_gb300", "csrc", src), "rb") as f:
                    sha = hashlib.sha256(f.read()).hexdigest()
                assert parts[3] == sha, (os.path.basename(md), parts[1])
                assert float(parts[2]) > 0
    assert found >= 2
