"""Serving form (kmeans2_server_*): continuous batching of independent fits (GPU).

Each job's result must be the same alone and in the mix: the server runs the
very kernels of a lone kmeans2_fit and the cluster sums are exact, so labels,
centers, J and iteration counts are compared bit for bit."""
import time

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


# (n, d, k, f, tol, max_iter, seed): CUDA-core and BF16 shapes, tiny to mid-size
MIX = [
    (20_000, 4, 16, 0.1, 1e-6, 60, 1),
    (150_000, 16, 200, 0.1, 1e-6, 40, 2),
    (60_000, 64, 64, 0.1, 1e-6, 40, 3),
    (200_000, 128, 512, 0.1, 1e-6, 30, 4),
    (3_000, 4, 4, 0.2, 1e-6, 100, 5),
    (90_000, 128, 1024, 0.1, 1e-6, 30, 6),
    (120_000, 16, 32, 0.05, 1e-6, 50, 7),
    (40_000, 64, 300, 0.1, 1e-6, 40, 8),
    (250_000, 4, 700, 0.1, 1e-5, 25, 9),
    (10_000, 16, 8, 0.3, 1e-6, 100, 10),
]


def _data(n, d, k, seed):
    return synth.iso_gaussian_mixture(n, d, k, seed, lo=-20.0, hi=20.0, device=DEV)


def _same(a, b):
    assert (a.iters_fast, a.iters_slow) == (b.iters_fast, b.iters_slow)
    assert torch.equal(a.labels, b.labels)
    assert torch.equal(a.centers, b.centers)
    assert a.J == b.J
    assert a.precision_used == b.precision_used


def test_server_results_equal_alone():
    Xs = [_data(n, d, k, s) for (n, d, k, f, tol, it, s) in MIX]
    alone = [km.fit(X, k, f, s, tol, it) for X, (n, d, k, f, tol, it, s) in zip(Xs, MIX)]
    torch.cuda.synchronize()
    with km.Server(max_slots=4) as srv:
        tickets = [srv.submit(X, k, f, s, tol, it) for X, (n, d, k, f, tol, it, s) in zip(Xs, MIX)]
        served = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(MIX) and st["failed"] == 0
    assert st["kernel_launches"] > 0
    for a, sv in zip(alone, served):
        assert sv.status == 0
        _same(sv.result, a)
        assert sv.t_submit <= sv.t_admit <= sv.t_done


def test_server_small_jobs_match_oracle():
    nt = max(1, oracle.max_threads())
    specs = [(3_000, 4, 4, 0.2, 1e-6, 100, 5), (10_000, 16, 8, 0.3, 1e-6, 100, 10),
             (6_000, 64, 12, 0.2, 1e-6, 100, 11)]
    with km.Server(max_slots=3) as srv:
        Xs = [_data(n, d, k, s) for (n, d, k, f, tol, it, s) in specs]
        tickets = [srv.submit(X, k, f, s, tol, it) for X, (n, d, k, f, tol, it, s) in zip(Xs, specs)]
        for X, t, (n, d, k, f, tol, it, s) in zip(Xs, tickets, specs):
            sv = srv.wait(t)
            assert sv.status == 0
            Xh = to_np(X)
            o = oracle.fit(Xh, k, f, s, tol, it, nthreads=nt)
            assert (sv.result.iters_fast, sv.result.iters_slow) == (o["iters_fast"], o["iters_slow"])
            assert np.array_equal(to_np(sv.result.labels), o["labels"])
            assert_centers_close(to_np(sv.result.centers), o["centers"], Xh)
            assert_J_close(sv.result.J, o["J"], Xh)


def test_server_admission_respects_budget():
    specs = [(100_000, 64, 128, 0.1, 1e-6, 30, 20 + j) for j in range(8)]
    fp = km.footprint(100_000, 64, 128, 0.1, 30) + 100_000 * 64 * 4
    budget = int(2.5 * fp)                       # two such jobs at a time
    Xs = [_data(n, d, k, s) for (n, d, k, f, tol, it, s) in specs]
    with km.Server(hbm_budget=budget, max_slots=6) as srv:
        tickets = [srv.submit(X, k, f, s, tol, it) for X, (n, d, k, f, tol, it, s) in zip(Xs, specs)]
        served = [srv.wait(t) for t in tickets]
        st = srv.stats()
        # a job larger than the whole budget is refused, not queued
        big = torch.empty((2_000_000, 64), dtype=torch.float32, device=DEV)
        with pytest.raises(km.KMeans2Error) as ei:
            srv.submit(big, 128, 0.1, 0, 1e-6, 30)
        assert ei.value.status == -6
        assert srv.stats()["rejected"] == 1
    assert all(s.status == 0 for s in served)
    assert st["hbm_peak"] <= budget
    assert st["hbm_peak"] >= fp
    for X, sv, (n, d, k, f, tol, it, s) in zip(Xs, served, specs):
        _same(sv.result, km.fit(X, k, f, s, tol, it))


def test_server_host_buffers():
    n, d, k, f, tol, it, s = 50_000, 16, 40, 0.1, 1e-6, 50, 31
    X = _data(n, d, k, s)
    a = km.fit(X, k, f, s, tol, it)
    Xh = X.cpu().numpy()
    with km.Server(max_slots=2) as srv:
        sv = srv.wait(srv.submit(Xh, k, f, s, tol, it))
    assert sv.status == 0
    assert np.array_equal(sv.result.labels, a.labels.cpu().numpy())
    assert np.array_equal(sv.result.centers, a.centers.cpu().numpy())
    assert sv.result.J == a.J


def test_server_admits_arrivals_while_running():
    # a long job first; a short one arriving while it runs starts before it ends
    # and, with the host-driven stage loops a server of several slots uses,
    # also finishes first (its kernels run between the long job's launches)
    XA = _data(2_000_000, 128, 1024, 41)
    XB = _data(20_000, 4, 8, 42)
    with km.Server(max_slots=2) as srv:
        ta = srv.submit(XA, 1024, 0.1, 41, 1e-7, 40)
        t0 = time.time()
        while srv.stats()["running"] < 1 and time.time() - t0 < 30:
            time.sleep(0.001)
        tb = srv.submit(XB, 8, 0.1, 42, 1e-6, 50)
        b = srv.wait(tb)
        a = srv.wait(ta)
    assert a.status == 0 and b.status == 0
    assert b.t_admit < a.t_done
    assert b.t_done < a.t_done
    _same(b.result, km.fit(XB, 8, 0.1, 42, 1e-6, 50))


def test_server_graph_stage_loops_match_fits():
    # the same jobs with the stage loops as while-graphs (use_graph=True)
    specs = [(60_000, 16, 24, 0.1, 1e-6, 40, 51), (30_000, 64, 520, 0.1, 1e-6, 20, 52),
             (8_000, 3, 5, 0.5, 1e-6, 60, 53)]
    Xs = [_data(n, d, k, s) for n, d, k, _, _, _, s in specs]
    with km.Server(max_slots=3, use_graph=True) as srv:
        tickets = [srv.submit(X, k, f, s, tol, it) for X, (n, d, k, f, tol, it, s) in zip(Xs, specs)]
        served = [srv.wait(t) for t in tickets]
    for X, sv, (n, d, k, f, tol, it, s) in zip(Xs, served, specs):
        assert sv.status == 0
        _same(sv.result, km.fit(X, k, f, s, tol, it))


def test_server_destroy_with_queued_jobs():
    Xs = [_data(300_000, 64, 256, 50 + j) for j in range(4)]
    srv = km.Server(max_slots=1)
    for j, X in enumerate(Xs):
        srv.submit(X, 256, 0.1, 50 + j, 1e-6, 30)
    srv.close()          # the running job completes, the waiting ones are cancelled
    torch.cuda.synchronize()


def test_server_faulty_job_leaves_the_others_unchanged():
    # a job holding a NaN fails with KMEANS2_ERR_NONFINITE; the jobs beside it
    # still equal their lone runs, and malformed requests are refused at submit
    specs = [(40_000, 16, 30, 0.1, 1e-6, 50, 61), (60_000, 64, 100, 0.1, 1e-6, 40, 62),
             (30_000, 4, 12, 0.1, 1e-6, 60, 63)]
    Xs = [_data(n, d, k, s) for (n, d, k, f, tol, it, s) in specs]
    bad = _data(50_000, 16, 20, 64)
    bad[123, 5] = float("nan")
    alone = [km.fit(X, k, f, s, tol, it) for X, (n, d, k, f, tol, it, s) in zip(Xs, specs)]
    with km.Server(max_slots=4) as srv:
        tb = srv.submit(bad, 20, 0.1, 64, 1e-6, 50)
        tickets = [srv.submit(X, k, f, s, tol, it) for X, (n, d, k, f, tol, it, s) in zip(Xs, specs)]
        for args in [(Xs[0], 0, 0.1, 1, 1e-6, 10), (Xs[0], 10, 0.0, 1, 1e-6, 10),
                     (Xs[0], 10, 0.1, 1, -1.0, 10), (Xs[0], 10, 0.1, 1, 1e-6, 0)]:
            with pytest.raises(km.KMeans2Error) as ei:
                srv.submit(*args)
            assert ei.value.status == -1
        fb = srv.wait(tb)
        served = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert fb.status == -4 and fb.result is None
    assert st["failed"] == 1 and st["completed"] == len(specs)
    for a, sv in zip(alone, served):
        assert sv.status == 0
        _same(sv.result, a)


@pytest.mark.parametrize("aging,order", [(1000.0, "CDB"), (0.0, "BCD")])
def test_server_shortest_policy_admission_order(aging, order):
    # one slot held by a long job; three jobs queue behind it.  SHORTEST admits
    # the least work per iteration first; with aging 0 every job is "old" and
    # the oldest goes first (arrival order)
    XA = _data(2_000_000, 128, 1024, 71)
    jobs = {"B": (100_000, 16, 64, 72), "C": (20_000, 4, 8, 73), "D": (50_000, 16, 16, 74)}
    Xs = {name: _data(n, d, k, s) for name, (n, d, k, s) in jobs.items()}
    with km.Server(max_slots=1, policy="shortest", aging_s=aging) as srv:
        ta = srv.submit(XA, 1024, 0.1, 71, 1e-7, 40)
        t0 = time.time()
        while srv.stats()["running"] < 1 and time.time() - t0 < 30:
            time.sleep(0.001)
        tickets = {name: srv.submit(Xs[name], k, 0.1, s, 1e-6, 50)
                   for name, (n, d, k, s) in jobs.items()}
        res = {name: srv.wait(t) for name, t in tickets.items()}
        a = srv.wait(ta)
    assert a.status == 0 and all(r.status == 0 for r in res.values())
    got = "".join(sorted(res, key=lambda nm: res[nm].t_admit))
    assert got == order
    for name, (n, d, k, s) in jobs.items():
        _same(res[name].result, km.fit(Xs[name], k, 0.1, s, 1e-6, 50))


def test_server_lazy_jobs_equal_eager_fits():
    # points produced at admission by a callback, outputs handed to a consumer:
    # same results as eager fits of the same data; a failing producer fails
    # only its own job
    specs = {"a": (40_000, 16, 30, 0.1, 1e-6, 50, 81), "b": (25_000, 64, 50, 0.1, 1e-6, 40, 82),
             "c": (60_000, 4, 12, 0.2, 1e-6, 60, 83)}
    outs = {}

    def make_for(n, d, k, s):
        def make(X):
            X.copy_(_data(n, d, k, s))
        return make

    def consume_for(name):
        def consume(C, L):
            outs[name] = (C.clone(), L.clone())
        return consume

    def broken(X):
        raise RuntimeError("no data")

    with km.Server(max_slots=3, policy="shortest", aging_s=5.0) as srv:
        tickets = {name: srv.submit_lazy(n, d, k, f, s, tol, it, make_for(n, d, k, s),
                                         consume_for(name))
                   for name, (n, d, k, f, tol, it, s) in specs.items()}
        tb = srv.submit_lazy(1000, 8, 4, 0.5, 1, 1e-6, 10, broken)
        res = {name: srv.wait(t) for name, t in tickets.items()}
        fb = srv.wait(tb)
        st = srv.stats()
    assert fb.status == -1 and st["failed"] == 1
    for name, (n, d, k, f, tol, it, s) in specs.items():
        assert res[name].status == 0
        a = km.fit(_data(n, d, k, s), k, f, s, tol, it)
        C, L = outs[name]
        assert torch.equal(C, a.centers) and torch.equal(L, a.labels)
        assert res[name].result.J == a.J
        assert (res[name].result.iters_fast, res[name].result.iters_slow) == (a.iters_fast, a.iters_slow)


def test_server_wait_any_returns_each_finished_job_once():
    specs = [(20_000, 4, 8, 0.1, 1e-6, 40, 91 + j) for j in range(6)]
    Xs = [_data(n, d, k, s) for (n, d, k, f, tol, it, s) in specs]
    with km.Server(max_slots=3) as srv:
        tickets = {srv.submit(X, k, f, s, tol, it) for X, (n, d, k, f, tol, it, s) in zip(Xs, specs)}
        seen = set()
        for _ in range(len(specs)):
            sv = srv.wait_any(60.0)
            assert sv is not None and sv.status == 0
            seen.add(sv.ticket)
        assert seen == tickets
        assert srv.wait_any(0.01) is None
