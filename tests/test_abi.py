"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
entry point its header declares, and its host-only functions behave."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1108_1351_gb300 as km
from paper_1108_1351_gb300 import binding
from paper_1108_1351_gb300 import build as libbuild


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return km.load()


def test_exports_every_declared_symbol(lib):
    names = km.declared_symbols()
    assert {"kmeans2_fit", "kmeans_step", "kmeans2_sample", "kmeans2_subset_size",
            "kmeans2_strerror", "kmeans2_default_options", "kmeans2_version",
            "kmeans2_last_error"} <= set(names)
    raw = ctypes.CDLL(binding.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name


def test_subset_size_matches_oracle(lib):
    rng = np.random.default_rng(0)
    cases = [(20000, 4, 0.1), (500_000_000, 32, 0.01), (50_000_000, 1024, 0.02),
             (1000, 256, 0.1), (10, 3, 1.0), (7, 2, 0.5), (1, 1, 0.3)]
    cases += [(int(rng.integers(1, 10**7)), 1, float(rng.uniform(1e-4, 1))) for _ in range(200)]
    for n, k, f in cases:
        k = min(k, n)
        assert km.subset_size(n, k, f) == oracle.subset_size(n, k, f), (n, k, f)
    assert km.subset_size(10, 11, 0.5) == -1
    assert km.subset_size(10, 2, 0.0) == -1
    assert km.subset_size(10, 2, 1.5) == -1


def test_status_strings_and_version(lib):
    for code in range(0, -8, -1):
        assert km.strerror(code) not in ("", "unknown status")
    assert km.strerror(-99) == "unknown status"
    assert km.version() >= (1, 0)


def test_default_options(lib):
    o = binding.Options()
    lib.kmeans2_default_options(ctypes.byref(o))
    assert o.precision == 2 and o.use_graph == 1 and o.init_centers is None and o.stream is None


def test_invalid_arguments_rejected_before_device_work(lib):
    X = np.zeros((8, 2), dtype=np.float32)
    C = np.zeros((2, 2))
    lab = np.zeros(8, dtype=np.int32)
    res = binding.Result()
    p = X.ctypes.data
    bad = [
        (p, 8, 2, 9, 0.5, 0, 1e-6, 10),      # k > n
        (p, 8, 2, 2, 0.0, 0, 1e-6, 10),      # f = 0
        (p, 8, 2, 2, 1.5, 0, 1e-6, 10),      # f > 1
        (p, 8, 2, 2, 0.5, 0, -1.0, 10),      # tol < 0
        (p, 8, 2, 2, 0.5, 0, float("nan"), 10),
        (p, 8, 2, 2, 0.5, 0, 1e-6, 0),       # max_iter < 1
        (p, 8, 0, 2, 0.5, 0, 1e-6, 10),      # d < 1
        (None, 8, 2, 2, 0.5, 0, 1e-6, 10),   # NULL X
    ]
    for args in bad:
        rc = lib.kmeans2_fit(*args, C.ctypes.data, lab.ctypes.data, ctypes.byref(res), None)
        assert rc == -1, args
    assert lib.kmeans_step(p, 8, 2, 9, C.ctypes.data, C.ctypes.data, lab.ctypes.data,
                           None, None, None, None) == -1
    assert lib.kmeans2_sample(8, 9, 0.5, 0, lab.ctypes.data, lab.ctypes.data, None) == -1


def test_fit_footprint_host_arithmetic(lib):
    # device bytes of the buffers kmeans2_fit allocates: grows with n, d and k;
    # host-side X / labels add their staged copies; the BF16 form adds its copies
    base = km.footprint(1_000_000, 16, 64, 0.1, 50, precision="fp32")
    assert base > 1_000_000 * 4 * 2          # labels of S_n + recheck list at least
    assert km.footprint(2_000_000, 16, 64, 0.1, 50, precision="fp32") > base
    assert km.footprint(1_000_000, 32, 64, 0.1, 50, precision="fp32") > base
    assert km.footprint(1_000_000, 16, 512, 0.1, 50, precision="fp32") > base
    host_x = km.footprint(1_000_000, 16, 64, 0.1, 50, precision="fp32", x_on_host=True)
    assert host_x - base == 1_000_000 * 16 * 4 + 1024
    host_l = km.footprint(1_000_000, 16, 64, 0.1, 50, precision="fp32", labels_on_host=True)
    assert host_l - base == 1_000_000 * 4 + 1024
    f32 = km.footprint(1_000_000, 128, 1024, 0.1, 50, precision="fp32")
    b16 = km.footprint(1_000_000, 128, 1024, 0.1, 50, precision="bf16")
    assert b16 - f32 >= 2 * 1_100_000 * 128 * 2      # hi + lo BF16 copies of S_n and S_s
    # AUTO runs the fast stage in the single-pass FP16 form and the slow stage in
    # FP16 or split BF16: it counts the FP16 fast stage with its second pass and
    # the larger slow stage
    # (the FP16 slow stage, half-size tiles plus second-pass buffers for a
    # quarter of the rows, is the larger)
    f16 = km.footprint(1_000_000, 128, 1024, 0.1, 50, precision="fp16")
    assert f16 > b16
    assert km.footprint(1_000_000, 128, 1024, 0.1, 50, precision="auto") == f16
    assert km.footprint(1_000_000, 8, 32, 0.1, 50, precision="auto") == \
        km.footprint(1_000_000, 8, 32, 0.1, 50, precision="fp32")
    # invalid shapes and unsupported forms give 0
    assert km.footprint(10, 2, 11, 0.1, 50) == 0
    assert km.footprint(10, 2, 2, 0.0, 50) == 0
    assert km.footprint(10, 2, 2, 0.5, 0) == 0
    assert km.footprint(1000, 24, 8, 0.5, 10, precision="bf16") == 0


def test_server_create_without_device_or_bad_args(lib):
    o = binding.Options()
    lib.kmeans2_default_options(ctypes.byref(o))
    assert not lib.kmeans2_server_create(1 << 30, 0, ctypes.byref(o))
    assert not lib.kmeans2_server_create(1 << 30, 65, ctypes.byref(o))
    o.start_stage = 1
    assert not lib.kmeans2_server_create(1 << 30, 2, ctypes.byref(o))
    st = binding.ServerStats()
    assert lib.kmeans2_server_stats_get(None, ctypes.byref(st)) == -1
    assert lib.kmeans2_server_poll(None, 1, None, None) == -1
    assert lib.kmeans2_server_now(None) == 0.0
    lib.kmeans2_server_destroy(None)
    assert km.strerror(1) == "pending"


def test_binding_rejects_mismatched_buffers_before_any_device_work(lib):
    """The library writes exactly k*d FP64 centers and n int32 labels and reads
    k*d FP64 initial centers: the binding refuses buffers of another type, size
    or layout instead of passing them on."""
    X = np.random.default_rng(0).standard_normal((100, 4)).astype(np.float32)
    bad_out = [
        dict(centers_out=np.empty((5, 4), dtype=np.float32)),       # wrong type
        dict(centers_out=np.empty((4, 4), dtype=np.float64)),       # too small
        dict(centers_out=np.empty((4, 10), dtype=np.float64)[:, :5].T),  # not contiguous
        dict(labels_out=np.empty(99, dtype=np.int32)),              # too small
        dict(labels_out=np.empty(100, dtype=np.int64)),             # wrong type
        dict(init_centers=np.zeros((5, 3))),                        # wrong d
        dict(init_centers=np.zeros((4, 4))),                        # wrong k
    ]
    for kw in bad_out:
        with pytest.raises(ValueError):
            km.fit(X, 5, 0.5, 0, 1e-6, 10, **kw)
    ro = np.empty((5, 4), dtype=np.float64)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        km.fit(X, 5, 0.5, 0, 1e-6, 10, centers_out=ro)
    with pytest.raises(ValueError):
        km.step(X, np.zeros((5, 3)))                                # centers of another d


def test_batched_binding_accepts_an_empty_job_list(lib):
    assert km.fit_batched([], [], 0.1, [], 1e-6, 10) == ([], 0)


def test_batched_tile_shape_query_rejects_bad_arguments(lib):
    """kmeans2_batched_tile_shape is host-only: d outside [1, 64] or a NULL
    output is KMEANS2_ERR_INVALID, and before any batched call has tuned a
    dimension class there is nothing to report."""
    one = ctypes.c_int32(-7)
    out = [ctypes.c_int32(-7) for _ in range(3)]
    refs = [ctypes.byref(v) for v in out]
    invalid = lib.kmeans2_batched_tile_shape(0, *refs)
    assert invalid != 0 and km.strerror(invalid)
    assert lib.kmeans2_batched_tile_shape(65, *refs) == invalid
    assert lib.kmeans2_batched_tile_shape(8, None, ctypes.byref(one), ctypes.byref(one)) == invalid
    assert [v.value for v in out] == [-7, -7, -7] and one.value == -7
    assert km.batched_tile_shape(0) is None and km.batched_tile_shape(65) is None
    import torch
    if not torch.cuda.is_available():
        assert km.batched_tile_shape(8) is None
