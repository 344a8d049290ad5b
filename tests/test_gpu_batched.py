"""Batched form (kmeans2_fit_batched) vs the oracle and vs single fits (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import synth
from tests.gpu_helpers import assert_centers_close, assert_J_close, to_np

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


def _specs(count, seed, n_hi=20000, k_hi=40):
    specs = synth.instance_specs(count, seed=seed, n_lo=300, n_hi=n_hi, k_lo=1, k_hi=k_hi)
    return specs


def test_batched_matches_oracle_per_job():
    specs = _specs(48, 1)
    Xs = [synth.instance_data(s, device=DEV) for s in specs]
    res, rc = km.fit_batched(Xs, [s.k for s in specs], 0.1, [s.seed for s in specs], 1e-6, 40)
    assert rc == 0
    nt = max(1, oracle.max_threads())
    for s, X, r in zip(specs, Xs, res):
        Xh = to_np(X)
        o = oracle.fit(Xh, s.k, 0.1, s.seed, 1e-6, 40, nthreads=nt)
        assert (r.iters_fast, r.iters_slow) == (o["iters_fast"], o["iters_slow"]), s
        assert np.array_equal(to_np(r.labels), o["labels"]), s
        assert_centers_close(to_np(r.centers), o["centers"], Xh)
        assert_J_close(r.J, o["J"], Xh)
        assert r.distance_evals == o["distance_evals"]


def test_batched_equals_single_fits():
    specs = _specs(40, 2, n_hi=200_000, k_hi=256)
    Xs = [synth.instance_data(s, device=DEV) for s in specs]
    res, rc = km.fit_batched(Xs, [s.k for s in specs], 0.1, [s.seed for s in specs], 1e-5, 30,
                             tol_fast=1e-3)
    assert rc == 0
    for s, X, r in zip(specs, Xs, res):
        a = km.fit(X, s.k, 0.1, s.seed, 1e-5, 30, tol_fast=1e-3, precision="fp32")
        assert (r.iters_fast, r.iters_slow) == (a.iters_fast, a.iters_slow), s
        assert torch.equal(r.labels, a.labels), s
        assert torch.equal(r.centers, a.centers), s
        assert r.J == a.J


def test_batched_nonfinite_job_does_not_disturb_others():
    specs = _specs(6, 3)
    Xs = [synth.instance_data(s, device=DEV) for s in specs]
    Xs[2][min(5, Xs[2].shape[0] - 1), 0] = float("nan")
    res, rc = km.fit_batched(Xs, [s.k for s in specs], 0.2, [s.seed for s in specs], 1e-6, 30,
                             raise_on_error=False)
    assert rc == -4
    for j, (s, X, r) in enumerate(zip(specs, Xs, res)):
        if j == 2:
            continue
        a = km.fit(X, s.k, 0.2, s.seed, 1e-6, 30, precision="fp32")
        assert torch.equal(r.labels, a.labels) and r.J == a.J


def test_batched_profiled_host_loop_equals_graph():
    # the profiled (host-driven) loop runs the same kernels as the graph loop
    specs = _specs(24, 5, n_hi=100_000, k_hi=200)
    Xs = [synth.instance_data(s, device=DEV) for s in specs]
    args = ([s.k for s in specs], 0.1, [s.seed for s in specs], 1e-5, 40)
    a, rc_a = km.fit_batched(Xs, *args)
    prof = km.Profile()
    b, rc_b = km.fit_batched(Xs, *args, profile=prof)
    assert rc_a == rc_b == 0
    for ra, rb in zip(a, b):
        assert (ra.iters_fast, ra.iters_slow) == (rb.iters_fast, rb.iters_slow)
        assert torch.equal(ra.labels, rb.labels) and torch.equal(ra.centers, rb.centers)
        assert ra.J == rb.J
    assert prof.assign_launches > 0 and prof.assign_ms > 0 and prof.kernel_launches > 0
    want = sum(2.0 * (r.iters_fast * r.subset_size + r.iters_slow * s.n) * s.k * s.d
               for r, s in zip(b, specs))
    assert abs(prof.assign_flops - want) <= 1e-9 * want


def test_batched_reports_its_tile_shapes():
    """After a batched call the autotuner's choice is queryable per dimension
    class, and it is one of the shapes that class offers."""
    specs = [s for s in synth.instance_specs(64, seed=5, n_lo=2000, n_hi=20000, k_lo=2, k_hi=64)]
    Xs = [synth.instance_data(s, device=DEV) for s in specs]
    res, rc = km.fit_batched(Xs, [s.k for s in specs], 0.1, [s.seed for s in specs], 1e-5, 10)
    assert rc == 0
    offered = {2: {(2, 1), (4, 1)}, 8: {(2, 1), (4, 1)},
               32: {(1, 1), (2, 1), (4, 2), (4, 4)}, 64: {(1, 1), (2, 2), (4, 4)}}
    for d in sorted({s.d for s in specs}):
        got = km.batched_tile_shape(d)
        assert got is not None, d
        p, g, tiles = got
        assert (p, g) in offered[d], (d, got)
        assert tiles in (1, 2, 4, 8), (d, got)
