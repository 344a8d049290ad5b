"""kmeans2_fit_streamed: host-resident X streamed through the GPU in chunks (GPU).

The slow stage sees X one chunk at a time, but the arithmetic per point is the
same and the cluster sums are exact integers, so every result must equal the
resident kmeans2_fit (CUDA-core form) bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import synth
from tests.gpu_helpers import assert_centers_close, assert_J_close

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1351_gb300 import build
    build.build()
    oracle.build()
    km.load()


def _same(a, b):
    assert (a.iters_fast, a.iters_slow) == (b.iters_fast, b.iters_slow)
    assert np.array_equal(np.asarray(a.labels), np.asarray(b.labels))
    assert np.array_equal(np.asarray(a.centers), np.asarray(b.centers))
    assert a.J == b.J and a.distance_evals == b.distance_evals


@pytest.mark.parametrize("n,d,k,chunk", [(3_000_000, 8, 32, 1 << 18), (200_003, 16, 100, 50_000),
                                         (70_001, 3, 7, 70_001), (50_000, 64, 40, 4_099)])
def test_streamed_equals_resident(n, d, k, chunk):
    X = synth.aniso_gaussian_noise(n, d, k, 5, device="cpu", chunk=1 << 20).numpy()
    a = km.fit(X, k, 0.05, 11, 1e-6, 40, precision="fp32")
    b = km.fit_streamed(X, k, 0.05, 11, 1e-6, 40, chunk)
    _same(a, b)


def test_streamed_pinned_host_memory_and_oracle():
    n, d, k = 40_000, 4, 9
    Xt = synth.iso_gaussian_mixture(n, d, k, 21, device="cpu").pin_memory()
    b = km.fit_streamed(Xt, k, 0.1, 21, 1e-6, 60, 7_000)
    Xh = Xt.numpy()
    o = oracle.fit(Xh, k, 0.1, 21, 1e-6, 60, nthreads=max(1, oracle.max_threads()))
    assert (b.iters_fast, b.iters_slow) == (o["iters_fast"], o["iters_slow"])
    assert np.array_equal(b.labels, o["labels"])
    assert_centers_close(b.centers, o["centers"], Xh)
    assert_J_close(b.J, o["J"], Xh)


def test_streamed_rejects_device_x_and_invalid_shapes():
    X = torch.zeros((100, 8), device=DEV)
    with pytest.raises(TypeError):
        km.fit_streamed(X, 4, 0.5, 1, 1e-6, 5, 10)
    with pytest.raises(km.KMeans2Error):
        km.fit_streamed(np.zeros((100, 8), np.float32), 200, 0.5, 1, 1e-6, 5, 10)   # k > n


@pytest.mark.parametrize("pinned", [True, False])
def test_streamed_in_place_equals_resident(pinned):
    # chunk_points < 0: page-locked X is read by the kernels where it is;
    # pageable X falls back to staged chunks (as for 0).  All equal the
    # resident fit.
    n, d, k = 1_000_003, 8, 32
    Xt = synth.aniso_gaussian_noise(n, d, k, 12, device="cpu", chunk=1 << 20)
    if pinned:
        Xt = Xt.pin_memory()
    a = km.fit(Xt.numpy(), k, 0.02, 4, 1e-6, 40, precision="fp32")
    b = km.fit_streamed(Xt, k, 0.02, 4, 1e-6, 40, -1)
    _same(a, b)
    assert b.precision_used == "fp32"
    _same(a, km.fit_streamed(Xt, k, 0.02, 4, 1e-6, 40, 0))
