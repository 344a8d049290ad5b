"""The debug build (GPU): device-side index checks on every decided and old
label (-DKM2_DEBUG_CHECKS, reported as an error status, never a trap).

The same fits run in a child process that loads libkmeans2_debug.so
(KMEANS2_DEBUG=1) and in this process with the release library: every check
must pass (no error status) and the results must be identical."""
import json
import os
import subprocess
import sys

import pytest
import torch

import paper_1108_1351_gb300 as km

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r"""
import hashlib, json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import synth
km.load()
dev = torch.device("cuda", 0)
out = {"lib": km.LIB_PATH}
def digest(r):
    lab = torch.as_tensor(r.labels).cpu().numpy().astype(np.int32)
    return [r.J, r.iters_fast, r.iters_slow, hashlib.sha256(lab.tobytes()).hexdigest(),
            float(torch.as_tensor(r.centers).double().sum())]
X8 = synth.aniso_gaussian_noise(300_001, 8, 32, 1, device=dev)
X40 = synth.aniso_gaussian_noise(50_001, 40, 20, 2, device=dev)
Xv = synth.vmf_mixture(60_000, 64, 600, 3, device=dev)
out["fp32_small"] = digest(km.fit(X8, 32, 0.05, 1, 1e-6, 30, precision="fp32"))
out["fp32_large"] = digest(km.fit(X40, 20, 0.05, 1, 1e-6, 30, precision="fp32"))
out["tf32x3"] = digest(km.fit(X8, 32, 0.05, 1, 1e-6, 30, precision="tf32x3"))
out["bf16"] = digest(km.fit(Xv, 600, 0.1, 1, 1e-6, 20, precision="bf16"))
Xs = [X8[:100_000 + 1000 * j].contiguous() for j in range(6)]
res, rc = km.fit_batched(Xs, [4 + j for j in range(6)], 0.1, list(range(6)), 1e-6, 20)
out["batched"] = [rc] + [digest(r) for r in res]
print(json.dumps(out))
"""


def _run(debug: bool):
    env = dict(os.environ)
    env.pop("KMEANS2_DEBUG", None)
    if debug:
        env["KMEANS2_DEBUG"] = "1"
    code = "ROOT = %r\n" % ROOT + CASES
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_checks_pass_and_results_match_release():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1351_gb300 import build
    build.build()
    build.build(debug=True)
    dbg = _run(True)
    rel = _run(False)
    assert dbg.pop("lib").endswith("libkmeans2_debug.so")
    assert rel.pop("lib").endswith("libkmeans2.so")
    assert dbg == rel
