"""Data-parallel shards (GPU): the fit split over the rows of S_n.

Every rank keeps its own rows, labels and exact integer sums; the partials are
all-reduced per iteration.  Integer sums do not depend on the reduction order,
so for any number of ranks and any split the labels, centers, J and iteration
counts must equal the unsharded kmeans2_fit bit for bit (simulated multi-GPU:
the ranks run on this one GPU, reduced in rank order or by torch sums)."""
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
    assert torch.equal(torch.as_tensor(a.labels).cpu(), torch.as_tensor(b.labels).cpu())
    assert torch.equal(torch.as_tensor(a.centers).cpu(), torch.as_tensor(b.centers).cpu())
    assert a.J == b.J
    assert a.distance_evals == b.distance_evals
    assert a.precision_used == b.precision_used


@pytest.mark.parametrize("n,d,k,prec", [(200_003, 8, 32, "fp32"), (120_001, 64, 100, "bf16"),
                                        (90_001, 64, 300, "fp16"),
                                        (60_002, 16, 20, "tf32x3"), (30_001, 3, 7, "fp32")])
@pytest.mark.parametrize("shards", [1, 2, 3, 7])
def test_sharded_equals_unsharded(n, d, k, prec, shards):
    if prec in ("bf16", "fp16"):
        X = synth.vmf_mixture(n, d, k, 3, device=DEV)
    else:
        X = synth.aniso_gaussian_noise(n, d, k, 3, device=DEV)
    a = km.fit(X, k, 0.05, 17, 1e-6, 40, precision=prec)
    b = km.fit_sharded(X, k, 0.05, 17, 1e-6, 40, shards, precision=prec)
    _same(a, b)


def test_sharded_more_shards_than_rows_and_full_subset():
    # n = 10 over 7 ranks: boundaries on multiples of 4 rows leave empty ranks,
    # and f = 1 puts every row in S_s
    X = synth.iso_gaussian_mixture(10, 2, 3, 4, device=DEV)
    a = km.fit(X, 3, 1.0, 2, 0.0, 30)
    b = km.fit_sharded(X, 3, 1.0, 2, 0.0, 30, 7)
    _same(a, b)


def test_sharded_host_data_and_resume_from_given_centers():
    n, d, k = 50_000, 12, 16
    Xh = synth.aniso_gaussian_noise(n, d, k, 8, device="cpu").numpy()
    C0 = Xh[:k].astype(np.float64)
    a = km.fit(Xh, k, 0.1, 5, 1e-7, 60, init_centers=C0, start_stage=1)
    b = km.fit_sharded(Xh, k, 0.1, 5, 1e-7, 60, 4, init_centers=C0, start_stage=1)
    _same(a, b)
    a = km.fit(Xh, k, 0.1, 5, 1e-7, 60, init_centers=C0, tol_fast=1e-3)
    b = km.fit_sharded(Xh, k, 0.1, 5, 1e-7, 60, 5, init_centers=C0, tol_fast=1e-3)
    _same(a, b)


def test_sharded_matches_oracle():
    n, d, k = 20_000, 2, 4
    X = synth.iso_gaussian_mixture(n, d, k, 0, device=DEV)
    b = km.fit_sharded(X, k, 0.1, 0, 1e-6, 100, 3)
    Xh = X.cpu().numpy()
    o = oracle.fit(Xh, k, 0.1, 0, 1e-6, 100, nthreads=max(1, oracle.max_threads()))
    assert (b.iters_fast, b.iters_slow) == (o["iters_fast"], o["iters_slow"])
    assert np.array_equal(b.labels.cpu().numpy(), o["labels"])
    assert_centers_close(b.centers.cpu().numpy(), o["centers"], Xh)
    assert_J_close(b.J, o["J"], Xh)


def _reduce(bufs, op):
    # the all-reduce of an in-process group: sums in rank order
    tot = bufs[0].clone()
    for b in bufs[1:]:
        tot = torch.maximum(tot, b) if op == "max" else tot + b
    for b in bufs:
        b.copy_(tot)


@pytest.mark.parametrize("bounds", [(0, 1000, 33_333, 50_001), (0, 50_001)])
def test_shard_sessions_driven_from_python(bounds):
    # uneven, unaligned row ranges; the exchange done with torch ops
    n, d, k = bounds[-1], 32, 24
    X = synth.aniso_gaussian_noise(n, d, k, 6, device=DEV)
    a = km.fit(X, k, 0.1, 9, 1e-6, 50)
    shards = [km.Shard(X[lo:hi].clone(), lo, n, k, 0.1, 9, 1e-6, 50)
              for lo, hi in zip(bounds[:-1], bounds[1:])]
    exchanges = 0
    while True:
        xs = [s.advance() for s in shards]
        if all(x is None for x in xs):
            break
        assert all(x is not None and x[0] == xs[0][0] and x[1].numel() == xs[0][1].numel()
                   for x in xs)
        _reduce([x[1] for x in xs], xs[0][0])
        exchanges += 1
    res = [s.result() for s in shards]
    for s in shards:
        s.close()
    # init centers + one max|x| per stage + one partials exchange per iteration
    assert exchanges == 1 + 2 + a.iters_fast + a.iters_slow
    labels = torch.cat([r.labels for r in res])
    assert torch.equal(labels, a.labels)
    for r in res:
        assert torch.equal(r.centers, a.centers)
        assert r.J == a.J and (r.iters_fast, r.iters_slow) == (a.iters_fast, a.iters_slow)


def test_sharded_nonfinite_reaches_every_rank():
    X = synth.iso_gaussian_mixture(4_000, 4, 3, 1, device=DEV)
    X[3_900, 2] = float("nan")           # in the last rank's rows only
    with pytest.raises(km.KMeans2Error) as e:
        km.fit_sharded(X, 3, 1.0, 1, 1e-6, 10, 4)
    assert e.value.status == -4
