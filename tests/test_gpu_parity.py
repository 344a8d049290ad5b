"""CUDA path vs the FP64 oracle, element by element, on seeded inputs (GPU)."""
import numpy as np
import pytest
import torch

import oracle
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
    oracle.build()
    km.load()


DEV = "cuda:0"
NT = max(1, oracle.max_threads())


def _mixture(n, d, k, seed, spread=8.0):
    rng = np.random.default_rng(seed)
    means = rng.normal(size=(k, d)) * spread
    X = means[rng.integers(0, k, n)] + rng.normal(size=(n, d))
    return X.astype(np.float32)


def _centers_from(X, k, seed, jitter=0.0):
    rng = np.random.default_rng(seed + 99)
    idx = rng.choice(len(X), size=k, replace=False)
    C = X[idx].astype(np.float64)
    if jitter:
        C = C + jitter * rng.normal(size=C.shape)
    return C


def _step_both(X, C):
    Xd = torch.as_tensor(X, device=DEV)
    cn, lab, J, shift, empty = km.step(Xd, torch.as_tensor(C, device=DEV))
    ocn, olab, oJ, oshift, oempty = oracle.lloyd_step(X, C, nthreads=NT)
    return (to_np(cn), to_np(lab), J, shift, empty), (ocn, olab, oJ, oshift, oempty)


STEP_SHAPES = [
    # (n, d, k): small-d kernel (d <= 16) and large-d kernel; several tiles + ragged tails
    (5000, 1, 3), (20000, 2, 4), (10001, 3, 7), (9999, 5, 16), (70001, 8, 32), (12345, 13, 50),
    (30000, 16, 256), (5000, 17, 5), (20000, 32, 64), (10000, 64, 200), (4099, 128, 1024),
    (3000, 300, 10),
    # large enough that every CTA of the persistent grid walks several tiles
    (2_000_003, 8, 32), (1_500_001, 3, 7), (1_200_000, 16, 40), (700_001, 5, 100),
]


@pytest.mark.parametrize("n,d,k", STEP_SHAPES)
def test_step_matches_oracle(n, d, k):
    X = _mixture(n, d, k, seed=n + d + k)
    C = _centers_from(X, k, seed=d, jitter=0.3)
    (cn, lab, J, sh, em), (ocn, olab, oJ, osh, oem) = _step_both(X, C)
    assert np.array_equal(lab, olab)
    assert_centers_close(cn, ocn, X)
    assert_J_close(J, oJ, X)
    assert abs(sh - osh) <= 1e-10 * max(osh, 1.0)
    assert em == oem


TC_SHAPES = [(70001, 8, 32), (2_000_003, 8, 32), (50000, 4, 7), (300_001, 16, 100),
             (120_000, 32, 256), (33, 8, 1), (1000, 8, 256)]


@pytest.mark.parametrize("form", ["fp32", "tf32x3"])
@pytest.mark.parametrize("n,d,k", TC_SHAPES)
def test_step_each_form_matches_oracle(n, d, k, form):
    """Both distance-kernel forms (CUDA-core FP32 and tensor-core 3xTF32)."""
    X = _mixture(n, d, k, seed=3 * n + d + k)
    C = _centers_from(X, k, seed=d + 1, jitter=0.3)
    Xd = torch.as_tensor(X, device=DEV)
    cn, lab, J, sh, em = km.step(Xd, torch.as_tensor(C, device=DEV), precision=form)
    ocn, olab, oJ, osh, oem = oracle.lloyd_step(X, C, nthreads=NT)
    assert np.array_equal(to_np(lab), olab)
    assert_centers_close(to_np(cn), ocn, X)
    assert_J_close(J, oJ, X)
    assert em == oem


@pytest.mark.parametrize("form", ["fp32", "tf32x3"])
def test_fit_each_form_matches_oracle(form):
    X = to_np(synth.aniso_gaussian_noise(1_000_000, 8, 32, seed=23))
    Xd = torch.as_tensor(X, device=DEV)
    r = km.fit(Xd, 32, 0.02, 4, 1e-5, 30, precision=form, trajectories=True)
    o = oracle.fit(X, 32, 0.02, 4, 1e-5, 30, nthreads=NT)
    assert r.precision_used == form
    _assert_fit_equal(r, o, X)


BF16_SHAPES = [(20000, 16, 40), (50001, 64, 300), (30000, 128, 1024), (100_000, 128, 64),
               (10000, 112, 100), (5000, 32, 5), (1_000_001, 64, 32), (300, 128, 1),
               (200_003, 96, 777)]


@pytest.mark.parametrize("form", ["bf16", "fp16"])
@pytest.mark.parametrize("n,d,k", BF16_SHAPES)
def test_step_bf16_form_matches_oracle(n, d, k, form):
    """16-bit tensor-core cross term (split BF16; single-pass FP16 with its
    split-BF16 second pass) + FP64 recheck: labels still bit-exact."""
    X = _mixture(n, d, k, seed=5 * n + d + k, spread=3.0)
    C = _centers_from(X, k, seed=d + 2, jitter=0.3)
    Xd = torch.as_tensor(X, device=DEV)
    cn, lab, J, sh, em = km.step(Xd, torch.as_tensor(C, device=DEV), precision=form)
    ocn, olab, oJ, osh, oem = oracle.lloyd_step(X, C, nthreads=NT)
    assert np.array_equal(to_np(lab), olab)
    assert_centers_close(to_np(cn), ocn, X)
    assert_J_close(J, oJ, X)
    assert em == oem


@pytest.mark.parametrize("form", ["bf16", "fp16"])
def test_fit_bf16_vmf_matches_oracle(form):
    X = to_np(synth.vmf_mixture(60000, 128, 256, seed=7))
    Xd = torch.as_tensor(X, device=DEV)
    r = km.fit(Xd, 256, 0.05, 3, 1e-6, 15, precision=form, trajectories=True)
    o = oracle.fit(X, 256, 0.05, 3, 1e-6, 15, nthreads=NT)
    assert r.precision_used == form
    _assert_fit_equal(r, o, X)


@pytest.mark.parametrize("scale", [1e-20, 1e-12, 3e4, 1e13])
def test_step_fp16_scaled_operands_over_the_range(scale):
    # the single-pass FP16 form scales x and -2c by powers of two taken from
    # max|x| and max ||c||^2; tiny and huge data (outside FP16's own range)
    # and a set of centers much smaller than the data still give the oracle's
    # labels
    X0 = _mixture(40_000, 32, 20, seed=41, spread=3.0)
    C = _centers_from(X0, 20, seed=3, jitter=0.3)
    C[:5] *= 1e-3                                         # small centers
    X = (X0 * np.float32(scale)).astype(np.float32)
    C = C * scale
    Xd = torch.as_tensor(X, device=DEV)
    cn, lab, J, sh, em = km.step(Xd, torch.as_tensor(C, device=DEV), precision="fp16")
    ocn, olab, oJ, osh, oem = oracle.lloyd_step(X, C, nthreads=NT)
    assert np.array_equal(to_np(lab), olab)
    assert_centers_close(to_np(cn), ocn, X)
    assert_J_close(J, oJ, X)
    assert em == oem


def test_fp16_second_pass_overflow_goes_to_the_fp64_recheck():
    # every row a near tie (all points on the bisector of two centers): far
    # more undecided rows than the second pass takes (n / 4 + 1024), so the
    # FP64 recheck decides them all; labels still the oracle's
    rng = np.random.default_rng(77)
    n, d = 60_000, 32
    X = rng.normal(size=(n, d)).astype(np.float32)
    X[:, 0] = 0.0
    C = np.zeros((2, d))
    C[0, 0], C[1, 0] = 1.0, -1.0
    Xd = torch.as_tensor(X, device=DEV)
    cn, lab, J, sh, em = km.step(Xd, torch.as_tensor(C, device=DEV), precision="fp16")
    ocn, olab, oJ, osh, oem = oracle.lloyd_step(X, C, nthreads=NT)
    assert np.array_equal(to_np(lab), olab)
    assert_centers_close(to_np(cn), ocn, X)
    assert_J_close(J, oJ, X)


def test_tf32x3_rejects_unsupported_shape():
    X = torch.zeros((100, 5), dtype=torch.float32, device=DEV)
    with pytest.raises(km.KMeans2Error) as e:
        km.step(X, torch.zeros((3, 5), dtype=torch.float64, device=DEV), precision="tf32x3")
    assert e.value.status == -7


def test_step_exact_ties_duplicates_and_empty_cluster():
    rng = np.random.default_rng(5)
    base = rng.normal(size=(50, 4)).astype(np.float32)
    X = np.repeat(base, 40, axis=0)                      # every point 40 times
    C = np.concatenate([base[:6], base[:6], [[1e4] * 4]]).astype(np.float64)   # duplicated centers
    (cn, lab, J, sh, em), (ocn, olab, oJ, osh, oem) = _step_both(X, C)
    assert np.array_equal(lab, olab)
    assert lab.max() < 6                                  # ties go to the lowest index
    assert em == oem and em >= 7
    assert_centers_close(cn, ocn, X)
    assert_J_close(J, oJ, X)


def test_step_far_from_origin_forces_rechecks():
    rng = np.random.default_rng(6)
    X = (1000.0 + rng.normal(size=(40000, 3)) * 0.01).astype(np.float32)
    C = 1000.0 + rng.normal(size=(8, 3)) * 0.01
    (cn, lab, J, sh, em), (ocn, olab, oJ, osh, oem) = _step_both(X, C)
    assert np.array_equal(lab, olab)
    assert_centers_close(cn, ocn, X)
    assert_J_close(J, oJ, X)


@pytest.mark.parametrize("form", ["fp32", "tf32x3", "bf16", "fp16"])
def test_step_below_the_fixed_point_range(form):
    # max|x| ~ 1e-29 < 2^-74: the fixed-point scale stays at its cap 2^120, so
    # the cluster sums keep about 20 bits here.  Labels are still the oracle's;
    # centers meet the capped grid and J its rounding bound: each coordinate
    # moves by at most 2^-121 on the grid, i.e. |J - J_o| <= 1e-9 J_o +
    # 2^-120 sum_i ||x_i - c||_1 + n d 2^-242 (plus the same for the centers).
    X0 = _mixture(40_000, 32, 20, seed=43, spread=3.0)
    C = _centers_from(X0, 20, seed=4, jitter=0.3)
    X = (X0 * np.float32(1e-30)).astype(np.float32)
    C = C * 1e-30
    Xd = torch.as_tensor(X, device=DEV)
    cn, lab, J, sh, em = km.step(Xd, torch.as_tensor(C, device=DEV), precision=form)
    ocn, olab, oJ, osh, oem = oracle.lloyd_step(X, C, nthreads=NT)
    assert np.array_equal(to_np(lab), olab)
    assert_centers_close(to_np(cn), ocn, X)
    l1 = float(np.abs(X.astype(np.float64) - C[olab]).sum() + np.abs(X.astype(np.float64) - ocn[olab]).sum())
    assert abs(J - oJ) <= 1e-9 * oJ + 2.0 ** -120 * l1 + 2 * X.size * 2.0 ** -242, (J, oJ)
    assert em == oem


@pytest.mark.parametrize("form", ["fp32", "tf32x3", "bf16", "fp16"])
def test_step_far_from_origin_each_form(form):
    # x ~ 1e3 +- 1e-2 in d = 16: sum ||x||^2 / J ~ 1e10, so J must be formed
    # without cancellation to meet 1e-9 relative
    rng = np.random.default_rng(16)
    X = (1000.0 + rng.normal(size=(30000, 16)) * 0.01).astype(np.float32)
    C = 1000.0 + rng.normal(size=(12, 16)) * 0.01
    Xd = torch.as_tensor(X, device=DEV)
    cn, lab, J, sh, em = km.step(Xd, torch.as_tensor(C, device=DEV), precision=form)
    ocn, olab, oJ, osh, oem = oracle.lloyd_step(X, C, nthreads=NT)
    assert np.array_equal(to_np(lab), olab)
    assert_centers_close(to_np(cn), ocn, X)
    assert_J_close(J, oJ, X)
    assert abs(sh - osh) <= 1e-9 * osh


@pytest.mark.parametrize("case", ["1e3+-1e-2", "gauss2d+1e4"])
def test_fit_off_origin_matches_oracle(case):
    # Gaussian mixtures far from the origin (the second is the 20,000-point
    # d = 2, k = 4 workload shifted by +1e4): labels, centers, iteration counts
    # and every per-iteration J and movement equal the oracle's
    if case == "gauss2d+1e4":
        X = to_np(synth.iso_gaussian_mixture(20000, 2, 4, seed=0)) + np.float32(1e4)
        k = 4
    else:
        X = 1000.0 + _mixture(20000, 3, 5, seed=17) * 0.01
        k = 5
    X = np.ascontiguousarray(X, dtype=np.float32)
    r, o = _fit_both(X, k, 0.1, 0, 1e-6, 100)
    _assert_fit_equal(r, o, X)


def test_step_k_equals_n_and_k_one():
    X = _mixture(64, 3, 4, seed=7)
    C = X.astype(np.float64)
    (cn, lab, J, sh, em), (ocn, olab, oJ, osh, oem) = _step_both(X, C)
    assert np.array_equal(lab, olab) and np.array_equal(lab, np.arange(64))
    assert oJ == 0.0 and J == 0.0
    X = _mixture(3000, 6, 3, seed=8)
    C = X[:1].astype(np.float64)
    (cn, lab, J, sh, em), (ocn, olab, oJ, osh, oem) = _step_both(X, C)
    assert np.array_equal(lab, olab) and lab.max() == 0
    assert_centers_close(cn, ocn, X)


def test_step_host_buffers_match_device_buffers():
    X = _mixture(20000, 8, 16, seed=9)
    C = _centers_from(X, 16, seed=1)
    a = km.step(X, C)                                     # numpy in, numpy out (host staging)
    b = km.step(torch.as_tensor(X, device=DEV), torch.as_tensor(C, device=DEV))
    assert np.array_equal(a[1], to_np(b[1]))
    assert np.array_equal(a[0], to_np(b[0]))
    assert a[2] == b[2] and a[3] == b[3]


@pytest.mark.parametrize("n,k,f,seed", [(20000, 4, 0.1, 0), (1_000_000, 32, 0.01, 3),
                                        (1000, 256, 0.1, 5), (50, 50, 1.0, 1), (12345, 7, 0.37, 2**63 + 11)])
def test_sample_matches_oracle(n, k, f, seed):
    sub, pos = km.sample(n, k, f, seed, device=DEV)
    osub, opos = oracle.sample(n, k, f, seed)
    assert np.array_equal(to_np(sub), osub)
    assert np.array_equal(to_np(pos), opos)


def _fit_both(X, k, f, seed, tol, max_iter, tol_fast=0.0, **kw):
    Xd = torch.as_tensor(X, device=DEV)
    r = km.fit(Xd, k, f, seed, tol, max_iter, tol_fast=tol_fast, trajectories=True, **kw)
    o = oracle.fit(X, k, f, seed, tol, max_iter, tol_fast=tol_fast, nthreads=NT)
    return r, o


def _assert_fit_equal(r, o, X):
    assert (r.iters_fast, r.iters_slow) == (o["iters_fast"], o["iters_slow"])
    assert (r.converged_fast, r.converged_slow) == (o["converged_fast"], o["converged_slow"])
    assert np.array_equal(to_np(r.labels), o["labels"])
    assert_centers_close(to_np(r.centers), o["centers"], X)
    assert_J_close(r.J, o["J"], X)
    assert r.subset_size == o["subset_size"] and r.distance_evals == o["distance_evals"]
    assert r.empty_clusters == o["empty_clusters"]
    for key in ("J_fast", "J_slow"):
        for g, w in zip(r.traj[key], o["traj_" + key]):
            assert_J_close(g, w, X)
    for key in ("shift_fast", "shift_slow"):
        assert np.allclose(r.traj[key], o["traj_" + key], rtol=1e-9, atol=1e-10)


def test_fit_multi_tile_delta_iterations():
    """Enough points for many tiles per CTA and many incremental iterations."""
    X = to_np(synth.aniso_gaussian_noise(1_500_000, 8, 32, seed=21))
    r, o = _fit_both(X, 32, 0.05, 9, 1e-4, 25)
    _assert_fit_equal(r, o, X)


def test_fit_small_gaussian_config():
    """n = 20,000, d = 2, k = 4, isotropic Gaussians, 10% subset, tol 1e-6, seed 0."""
    X = to_np(synth.iso_gaussian_mixture(20000, 2, 4, seed=0))
    r, o = _fit_both(X, 4, 0.1, 0, 1e-6, 100)
    _assert_fit_equal(r, o, X)


@pytest.mark.parametrize("use_graph", [True, False])
def test_fit_aniso_noise_d8_k32(use_graph):
    X = to_np(synth.aniso_gaussian_noise(200_000, 8, 32, seed=1))
    r, o = _fit_both(X, 32, 0.01, 1, 1e-5, 50, use_graph=use_graph)
    _assert_fit_equal(r, o, X)


def test_fit_vmf_d32_k64():
    X = to_np(synth.vmf_mixture(30000, 32, 64, seed=2))
    r, o = _fit_both(X, 64, 0.05, 2, 1e-6, 40, tol_fast=1e-3)
    _assert_fit_equal(r, o, X)


def test_fit_full_subset_theorem():
    """Section 4.1 Theorem: with the whole set as S_s, the slow stage takes one
    iteration without movement."""
    X = _mixture(30000, 3, 5, seed=11)
    r, o = _fit_both(X, 5, 1.0, 4, 0.0, 300)
    _assert_fit_equal(r, o, X)
    assert r.iters_slow == 1 and r.traj["shift_slow"].tolist() == [0.0]


def test_fit_host_buffers_and_resume():
    X = _mixture(40000, 4, 6, seed=12)
    a = km.fit(X, 6, 0.1, 5, 1e-7, 60)                    # host in / host out
    b = km.fit(torch.as_tensor(X, device=DEV), 6, 0.1, 5, 1e-7, 60)
    assert np.array_equal(a.labels, to_np(b.labels)) and np.array_equal(a.centers, to_np(b.centers))
    assert a.J == b.J
    # resume the slow stage from given centers == oracle stage loop from them
    C0 = _centers_from(X, 6, seed=3)
    r = km.fit(X, 6, 0.1, 5, 1e-7, 60, init_centers=C0, start_stage=1)
    o = oracle.lloyd_stage(X, C0, 1e-7, 60, nthreads=NT)
    assert r.iters_fast == 0 and r.iters_slow == o["iters"]
    assert np.array_equal(r.labels, o["labels"])
    assert_centers_close(r.centers, o["centers"], X)
    assert_J_close(r.J, o["J"], X)


def test_fit_is_deterministic():
    X = torch.as_tensor(synth.aniso_gaussian_noise(300_000, 8, 32, seed=4), device=DEV)
    a = km.fit(X, 32, 0.02, 7, 1e-6, 30)
    b = km.fit(X, 32, 0.02, 7, 1e-6, 30)
    assert torch.equal(a.labels, b.labels) and torch.equal(a.centers, b.centers) and a.J == b.J


def test_nonfinite_input_is_rejected():
    X = _mixture(1000, 4, 3, seed=13)
    X[17, 2] = np.nan
    with pytest.raises(km.KMeans2Error) as e:
        km.fit(torch.as_tensor(X, device=DEV), 3, 0.5, 0, 1e-6, 10)
    assert e.value.status == -4


def test_release_memory_between_fits_keeps_results():
    # the library's scratch pool keeps freed memory mapped; trimming it between
    # calls changes nothing in the results
    X = torch.as_tensor(synth.aniso_gaussian_noise(200_000, 8, 16, seed=5), device=DEV)
    a = km.fit(X, 16, 0.05, 2, 1e-6, 30)
    km.release_memory()
    b = km.fit(X, 16, 0.05, 2, 1e-6, 30)
    assert torch.equal(a.labels, b.labels) and torch.equal(a.centers, b.centers) and a.J == b.J


@pytest.mark.parametrize("form", ["fp32", "bf16", "fp16"])
def test_step_many_near_ties_with_many_centers(form):
    # far from the origin with k * d = 38400: thousands of flagged points go
    # through the FP64 recheck (each reading all k d FP32 center values);
    # labels stay exact
    rng = np.random.default_rng(21)
    n, d, k = 30000, 64, 600
    X = (200.0 + rng.normal(size=(n, d)) * 0.05).astype(np.float32)
    C = 200.0 + rng.normal(size=(k, d)) * 0.05
    Xd = torch.as_tensor(X, device=DEV)
    cn, lab, J, sh, em = km.step(Xd, torch.as_tensor(C, device=DEV), precision=form)
    ocn, olab, oJ, osh, oem = oracle.lloyd_step(X, C, nthreads=NT)
    assert np.array_equal(to_np(lab), olab)
    assert_centers_close(to_np(cn), ocn, X)
    assert_J_close(J, oJ, X)
    assert em == oem


def test_center_and_count_trajectories_match_oracle_steps():
    # per iteration, the recorded centers and cluster sizes equal one oracle
    # Lloyd step from the previous recorded centers (the first from the drawn
    # initial centers, the slow stage's first from the fast stage's last)
    n, d, k, f, seed = 20_000, 3, 5, 0.1, 4
    X = _mixture(n, d, k, seed=31)
    Xd = torch.as_tensor(X, device=DEV)
    r = km.fit(Xd, k, f, seed, 1e-6, 40, trajectories=True, center_trajectories=True)
    tr = r.traj
    assert tr["centers_fast"].shape == (r.iters_fast, k, d)
    assert tr["counts_slow"].shape == (r.iters_slow, k)
    sub, pos = oracle.sample(n, k, f, seed)
    Xs = X[sub]
    C = Xs[pos].astype(np.float64)
    for stage, Xst, iters in (("fast", Xs, r.iters_fast), ("slow", X, r.iters_slow)):
        for i in range(iters):
            Cn, lab, J, shift, em = oracle.lloyd_step(Xst, C, nthreads=NT)
            assert np.array_equal(tr["counts_" + stage][i], np.bincount(lab, minlength=k))
            assert_centers_close(tr["centers_" + stage][i], Cn, Xst)
            assert_J_close(tr["J_" + stage][i], J, Xst)
            C = tr["centers_" + stage][i]
    assert np.array_equal(tr["centers_slow"][-1], r.centers.cpu().numpy())
    assert tr["counts_slow"][-1].sum() == n and tr["counts_fast"][-1].sum() == len(sub)
