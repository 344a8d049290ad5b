"""Every kernel variant of the batched form gives the single-fit results (GPU).

The batched form picks, per dimension class, a tile shape by timing: the
point slots per lane of its distance kernel and the lanes that share a point
("p" or "pxg").  Which one wins depends on the GPU and the workload, so the
debug build (KMEANS2_DEBUG=1) accepts KMEANS2_DEBUG_BATCH_POINTS to force one
shape on every class that offers it.
A mixed batch (d from 3 to 64, d both a multiple of 4 and not, k from 1 to
256) runs under each forced shape in a child process; labels, centers, J and
iteration counts must equal kmeans2_fit on each job alone (release library,
this process)."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

JOBS = [(40_000, 3, 9), (30_001, 8, 33), (25_000, 20, 129), (20_003, 21, 37), (18_000, 32, 256),
        (15_001, 40, 128), (12_000, 64, 200), (9_000, 63, 1), (40_000, 17, 64), (7_000, 48, 130)]

CASE = r"""
import hashlib, json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import synth
km.load()
dev = torch.device("cuda", 0)
def digest(r):
    lab = torch.as_tensor(r.labels).cpu().numpy().astype(np.int32)
    cen = torch.as_tensor(r.centers).cpu().numpy().astype(np.float64)
    return [r.J, r.iters_fast, r.iters_slow, hashlib.sha256(lab.tobytes()).hexdigest(),
            hashlib.sha256(cen.tobytes()).hexdigest()]
Xs = [synth.aniso_gaussian_noise(n, d, max(2, k // 2), 100 + j, device=dev)
      for j, (n, d, k) in enumerate(JOBS)]
ks = [k for _, _, k in JOBS]
out = {"lib": km.LIB_PATH}
if BATCHED:
    res, rc = km.fit_batched(Xs, ks, 0.1, list(range(len(JOBS))), 1e-6, 25)
    out["rc"] = rc
    out["fits"] = [digest(r) for r in res]
else:
    out["fits"] = [digest(km.fit(X, k, 0.1, j, 1e-6, 25, precision="fp32"))
                   for j, (X, k) in enumerate(zip(Xs, ks))]
print(json.dumps(out))
"""


def _run(batched: bool, points=None):
    env = dict(os.environ)
    env.pop("KMEANS2_DEBUG", None)
    env.pop("KMEANS2_DEBUG_BATCH_POINTS", None)
    if points is not None:
        env["KMEANS2_DEBUG"] = "1"
        env["KMEANS2_DEBUG_BATCH_POINTS"] = str(points)
    code = "ROOT = %r\nJOBS = %r\nBATCHED = %r\n" % (ROOT, JOBS, batched) + CASE
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_each_batched_tile_shape_equals_single_fits():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1351_gb300 import build
    build.build()
    build.build(debug=True)
    ref = _run(False)
    assert ref["lib"].endswith("libkmeans2.so")
    for points in ("1", "2", "4", "2x2", "4x2", "4x4"):
        got = _run(True, points)
        assert got["lib"].endswith("libkmeans2_debug.so")
        assert got["rc"] == 0, points
        for j, (a, b) in enumerate(zip(got["fits"], ref["fits"])):
            assert a == b, (points, JOBS[j])
