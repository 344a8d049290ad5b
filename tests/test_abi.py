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
