"""The data-parallel fit as two processes on one GPU (GPU).

Each process is one rank: it holds a block of rows of X, runs the real CUDA
shard session (kmeans2_shard_*) through fit_data_parallel, and every exchange
the session asks for (initial centers, max |x|, the per-iteration integer
partials) is one torch.distributed all_reduce over a gloo group, staged
through host memory.  No kernel waits on the other rank: each rank's stream is
synchronised at every exchange point before the host reduces.  Integer sums do
not depend on how the rows are split, so the labels, centers, J and iteration
counts equal kmeans2_fit on the whole X bit for bit."""
import multiprocessing as mp
import os
import socket
import sys
from datetime import timedelta

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data(spec):
    from paper_1108_1351_gb300 import synth
    n, d, k = spec["n"], spec["d"], spec["k"]
    return synth.aniso_gaussian_noise(n, d, k, spec["data_seed"])


def _rank(rank, ws, port, bounds, spec, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=timedelta(seconds=120))
    try:
        import paper_1108_1351_gb300 as km
        km.load()
        X = _data(spec)
        lo, hi = bounds[rank], bounds[rank + 1]
        Xr = X[lo:hi].contiguous().cuda()
        r = km.fit_data_parallel(Xr, lo, spec["n"], spec["k"], spec["f"], spec["seed"],
                                 spec["tol"], spec["max_iter"], precision=spec["precision"])
        out.put((rank, r.labels.cpu().numpy(), r.centers.cpu().numpy(), r.J,
                 (r.iters_fast, r.iters_slow), r.precision_used))
    except Exception as e:                      # reported by the parent
        out.put((rank, repr(e), None, None, None, None))
    finally:
        dist.destroy_process_group()


CASES = [
    # CUDA-core form, d = 8, uneven split
    dict(n=200_003, d=8, k=32, f=0.05, seed=5, tol=1e-6, max_iter=40, precision="fp32",
         data_seed=11, cut=77_777),
    # split-BF16 tensor-core form
    dict(n=60_001, d=64, k=520, f=0.1, seed=6, tol=1e-6, max_iter=20, precision="bf16",
         data_seed=12, cut=31_000),
]


@pytest.mark.parametrize("spec", CASES, ids=["fp32-d8", "bf16-d64"])
def test_two_process_shards_equal_single_fit(spec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1351_gb300 import build
    build.build()
    import paper_1108_1351_gb300 as km
    km.load()
    bounds = (0, spec["cut"], spec["n"])
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, bounds, spec, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get() for _ in range(2))
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    for g in got:
        assert g[2] is not None, g[1]
    X = _data(spec).cuda()
    ref = km.fit(X, spec["k"], spec["f"], spec["seed"], spec["tol"], spec["max_iter"],
                 precision=spec["precision"])
    labels = np.concatenate([g[1] for g in got])
    assert np.array_equal(labels, ref.labels.cpu().numpy())
    for _, _, centers, J, iters, used in got:
        assert np.array_equal(centers, ref.centers.cpu().numpy())     # every replica, exact
        assert J == ref.J
        assert iters == (ref.iters_fast, ref.iters_slow)
        assert used == ref.precision_used
