"""kmeans_step_noalloc against kmeans_step (GPU).

The no-allocation entry point serves callers that must not allocate device
memory during a call (for example a service whose device memory belongs to its
own pool).  It must give the same results as kmeans_step, call after call,
although every call reuses the same fixed scratch array.  This file is
collected last so that a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest
import torch

import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import synth
from tests.gpu_helpers import assert_centers_close, assert_J_close, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1351_gb300 import build
    build.build()
    km.load()


@pytest.mark.parametrize("n,d,k", [(200_000, 8, 32), (50_001, 32, 100)])
def test_noalloc_step_matches_step_on_consecutive_calls(n, d, k):
    dev = torch.device("cuda:0")
    X = synth.aniso_gaussian_noise(n, d, k, seed=n + d, device=dev)
    Xh = to_np(X)
    C = X[torch.randperm(n, generator=torch.Generator().manual_seed(1))[:k].to(dev)].double()
    for call in range(2):
        want = km.step(X, C)
        got = km.step_noalloc(X, C)
        assert np.array_equal(to_np(got[1]), to_np(want[1])), f"labels differ on call {call}"
        assert_centers_close(to_np(got[0]), to_np(want[0]), Xh)
        assert_J_close(got[2], want[2], Xh)
        assert abs(got[3] - want[3]) <= 1e-10 * max(want[3], 1.0)
        assert got[4] == want[4]
        C = want[0]                       # the second call starts from the updated centers


@pytest.mark.parametrize("d,k", [(128, 1024), (64, 512)])
def test_noalloc_step_at_its_size_limits(d, k):
    # n at the stated maximum, with d and k where kmeans_step would pick its
    # tensor-core form: the no-alloc step runs the CUDA-core form instead and
    # must return the same labels, centers and J as kmeans_step
    dev = torch.device("cuda:0")
    n = 4_194_304
    X = synth.vmf_mixture(n, d, k, seed=d, device=dev)
    C = X[torch.randperm(n, generator=torch.Generator().manual_seed(2))[:k].to(dev)].double()
    for call in range(2):
        want = km.step(X, C)
        got = km.step_noalloc(X, C)
        assert torch.equal(got[1], want[1]), f"labels differ on call {call}"
        assert torch.equal(got[0], want[0]), f"centers differ on call {call}"
        assert got[2] == want[2] and got[3] == want[3] and got[4] == want[4]
        C = want[0]


def test_noalloc_rejects_shapes_beyond_its_limits():
    dev = torch.device("cuda:0")
    X = torch.zeros((8, 129), dtype=torch.float32, device=dev)
    C = torch.zeros((2, 129), dtype=torch.float64, device=dev)
    with pytest.raises(km.KMeans2Error) as e:
        km.step_noalloc(X, C)
    assert e.value.status == -1 and "limits" in str(e.value)
