"""The bounded device-side waits of the tensor-core kernels (GPU).

Every mbarrier wait in the 16-bit and 3xTF32 tensor-core kernels has an iteration
limit; when it runs out the CTA records KMEANS2_ERR_TIMEOUT, the other roles
see the abort, each role lets its own bulk copies and MMAs finish, TMEM is
freed and the kernel returns.  The debug build (KMEANS2_DEBUG=1) takes the
limit of the consumer roles (MMA issuer and epilogues) from
KMEANS2_DEBUG_WAIT_TRIES; at 0 those waits give up at once, which is the
timeout path without any fault, trap or hang.  The call must report the
timeout status, and the next calls in the same process (limits restored)
must return the same labels, centers and J as the CUDA-core form."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASE = r"""
import json, os, sys
import torch
sys.path.insert(0, ROOT)
import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import synth
km.load()
dev = torch.device("cuda", 0)
Xb = synth.vmf_mixture(40_000, 64, 600, 5, device=dev)
Xt = synth.aniso_gaussian_noise(50_001, 8, 32, 6, device=dev)
out = {"lib": km.LIB_PATH}
for name, X, k in (("bf16", Xb, 600), ("fp16", Xb, 600), ("tf32x3", Xt, 32)):
    C = X[:k].double()
    os.environ["KMEANS2_DEBUG_WAIT_TRIES"] = "0"
    try:
        km.step(X, C, precision=name)
        status = 0
    except km.KMeans2Error as e:
        status = e.status
    del os.environ["KMEANS2_DEBUG_WAIT_TRIES"]
    torch.cuda.synchronize()                      # the context is still usable
    a = km.step(X, C, precision=name)
    b = km.step(X, C, precision="fp32")
    fa = km.fit(X, k, 0.1, 3, 1e-6, 10, precision=name)
    fb = km.fit(X, k, 0.1, 3, 1e-6, 10, precision="fp32")
    same = (bool(torch.equal(a[1], b[1])) and bool(torch.equal(a[0], b[0])) and a[2] == b[2]
            and bool(torch.equal(fa.labels, fb.labels)) and fa.J == fb.J)
    out[name] = [status, same]
print(json.dumps(out))
"""


def test_consumer_wait_timeout_reports_status_and_next_calls_are_correct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1351_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, KMEANS2_DEBUG="1")
    env.pop("KMEANS2_DEBUG_WAIT_TRIES", None)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CASE], capture_output=True,
                       text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out.pop("lib").endswith("libkmeans2_debug.so")
    for name in ("bf16", "fp16", "tf32x3"):
        status, same = out[name]
        assert status == -5, (name, status)            # KMEANS2_ERR_TIMEOUT
        assert same, name
