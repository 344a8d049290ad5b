"""Randomised shapes across the precision forms (GPU).

Every form decides a point only outside its own rounding bound and sends the
rest to the same FP64 recheck, so FP32, 3xTF32 and split-BF16 fits of the same
data must agree exactly (labels, centers, J, iteration counts), and agree with
the oracle.  The shapes are drawn at random (seeded) around the forms' internal
boundaries: d at and between the supported widths, k just below and above the
chunk widths (64, 128, 256, 512), ragged n, tiny and full subsets."""
import numpy as np
import pytest
import torch

import oracle
import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import synth
from tests.gpu_helpers import assert_centers_close, assert_J_close

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NT = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1351_gb300 import build
    build.build()
    oracle.build()
    km.load()


def _shapes(count=48, seed=2024):
    rng = np.random.default_rng(seed)
    ks = [2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513, 700]
    ds = [4, 8, 16, 32, 48, 64, 96, 112, 128]
    out = []
    for i in range(count):
        d = int(rng.choice(ds))
        k = int(rng.choice(ks))
        n = int(rng.integers(max(k, 1000), 40_000))
        f = float(rng.choice([0.05, 0.2, 1.0]))
        out.append((n, d, k, f, int(rng.integers(0, 1 << 30))))
    return out


def _forms(d, k):
    forms = ["fp32"]
    if d in (4, 8, 16, 32) and k <= 256:
        forms.append("tf32x3")
    if d % 16 == 0 and 16 <= d <= 128:
        forms.append("bf16")
        forms.append("fp16")
    return forms


@pytest.mark.parametrize("n,d,k,f,seed", _shapes())
def test_forms_agree_with_each_other_and_the_oracle(n, d, k, f, seed):
    X = synth.iso_gaussian_mixture(n, d, max(2, k // 3), seed % 1000, device=DEV)
    res = {form: km.fit(X, k, f, seed, 1e-6, 12, precision=form) for form in _forms(d, k)}
    ref = res["fp32"]
    for form, r in res.items():
        assert r.precision_used == form
        assert (r.iters_fast, r.iters_slow) == (ref.iters_fast, ref.iters_slow), form
        assert torch.equal(r.labels, ref.labels), form
        assert torch.equal(r.centers, ref.centers), form
        assert r.J == ref.J, form
    Xh = X.cpu().numpy()
    o = oracle.fit(Xh, k, f, seed, 1e-6, 12, nthreads=NT)
    assert (ref.iters_fast, ref.iters_slow) == (o["iters_fast"], o["iters_slow"])
    assert np.array_equal(ref.labels.cpu().numpy(), o["labels"])
    assert_centers_close(ref.centers.cpu().numpy(), o["centers"], Xh)
    assert_J_close(ref.J, o["J"], Xh)
