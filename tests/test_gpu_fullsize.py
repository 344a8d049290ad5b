"""Full-size workloads in the bench's launch configuration (GPU).

At n = 5e8 the oracle cannot redo a whole pass, so these tests check sampled
outputs one by one against the oracle (labels bit-exact) and properties that
hold at any size: the returned centers are the FP64 means of the points under
the returned labels, and J is the FP64 sum of the squared distances to the
centers the labels were assigned against."""
import numpy as np
import pytest
import torch

import oracle
import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import synth
from tests.gpu_helpers import grid_term

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda:0"
SAMPLE = 20_000


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1351_gb300 import build
    build.build()
    oracle.build()
    km.load()


def _means_fp64(X, labels, k, chunk=1 << 24):
    d = X.shape[1]
    S = torch.zeros(k, d, dtype=torch.float64, device=X.device)
    N = torch.zeros(k, dtype=torch.float64, device=X.device)
    for a in range(0, X.shape[0], chunk):
        lab = labels[a:a + chunk].long()
        S.index_add_(0, lab, X[a:a + chunk].double())
        N.index_add_(0, lab, torch.ones_like(lab, dtype=torch.float64))
    return S, N


def _J_fp64(X, labels, C, chunk=1 << 24):
    tot = torch.zeros((), dtype=torch.float64, device=X.device)
    for a in range(0, X.shape[0], chunk):
        diff = X[a:a + chunk].double() - C[labels[a:a + chunk].long()]
        tot += (diff * diff).sum()
    return float(tot)


def _grid(X):
    # fixed-point grid of the exact sums, from max |x| (reductions, no copy of X)
    return grid_term(np.array([max(abs(X.max().item()), abs(X.min().item()))]))


def _check_step(X, C_in, C_out, labels, J, k):
    n, d = X.shape
    # sampled labels, bit-exact against the oracle's FP64 argmin
    g = torch.Generator(device="cpu").manual_seed(7)
    idx = torch.randint(0, n, (SAMPLE,), generator=g)
    Xs = X[idx.to(X.device)].cpu().numpy()
    want = oracle.assign(Xs, C_in.cpu().numpy(), nthreads=max(1, oracle.max_threads()))[0]
    assert np.array_equal(labels[idx.to(X.device)].cpu().numpy(), want)
    # centers = FP64 means under the labels (empty clusters keep their center)
    S, N = _means_fp64(X, labels, k)
    mean = torch.where(N[:, None] > 0, S / N.clamp_min(1)[:, None], C_in)
    tol = 1e-10 * mean.abs().amax(dim=1, keepdim=True) + _grid(X)
    assert bool(((C_out - mean).abs() <= tol).all())
    # J of this assignment against the centers it was made with
    Jref = _J_fp64(X, labels, C_in)
    assert abs(J - Jref) <= 1e-9 * Jref, (J, Jref)


def test_default_workload_full_size_step_and_fit():
    # n = 5e8, d = 8, k = 32: anisotropic mixture with 2 % noise (the bench's default)
    n, d, k = 500_000_000, 8, 32
    X = synth.aniso_gaussian_noise(n, d, k, 0, device=DEV, chunk=1 << 24)
    fit = km.fit(X, k, 0.01, 0, 1e-5, 50)
    assert fit.iters_fast >= 1 and fit.iters_slow >= 1
    # the returned centers are the means of the points under the returned labels
    S, N = _means_fp64(X, fit.labels, k)
    assert int(N.sum().item()) == n
    nz = N > 0
    mean = S[nz] / N[nz][:, None]
    tol = 1e-10 * mean.abs().amax(dim=1, keepdim=True) + _grid(X)
    assert bool(((fit.centers[nz] - mean).abs() <= tol).all())
    # Lloyd: the mean minimises the within-cluster sum, so J (against the
    # pre-update centers) is at least the sum against the returned centers
    assert fit.J >= _J_fp64(X, fit.labels, fit.centers) * (1 - 1e-12)
    # one full-size step from the fit's centers, checked on samples and sums
    C_in = fit.centers.clone()
    C_out, labels, J, _, _ = km.step(X, C_in)
    _check_step(X, C_in, C_out, labels, J, k)


def test_precision_workload_full_size_bf16_step():
    # n = 5e7, d = 128, k = 1024: vMF mixture, split-BF16 tensor-core form
    n, d, k = 50_000_000, 128, 1024
    X = synth.vmf_mixture(n, d, k, 0, device=DEV, chunk=1 << 20)
    g = torch.Generator(device="cpu").manual_seed(3)
    C_in = X[torch.randperm(n, generator=g)[:k].to(DEV)].double()
    C_out, labels, J, _, _ = km.step(X, C_in, precision="bf16")
    _check_step(X, C_in, C_out, labels, J, k)
