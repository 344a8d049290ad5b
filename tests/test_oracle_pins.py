"""The oracle against its pins (CPU only)."""
import numpy as np
import pytest

import oracle
from tests import oracle_pins


@pytest.fixture(scope="module")
def o():
    return oracle._default_oracle()


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(o, pin):
    pin(o)


def test_thread_count_does_not_change_results(o):
    rng = np.random.default_rng(0)
    X = (rng.normal(size=(5000, 3)) + 8 * rng.normal(size=(6, 3))[rng.integers(0, 6, 5000)])
    X = X.astype(np.float32)
    a = o.fit(X, 6, 0.1, 1, tol=1e-7, max_iter=50, nthreads=1)
    b = o.fit(X, 6, 0.1, 1, tol=1e-7, max_iter=50, nthreads=max(2, o.max_threads()))
    assert np.array_equal(a["labels"], b["labels"])
    assert np.array_equal(a["centers"], b["centers"])
    assert a["J"] == b["J"] and a["iters_slow"] == b["iters_slow"]


def test_invalid_arguments_rejected(o):
    X = np.zeros((5, 2), dtype=np.float32)
    with pytest.raises(ValueError):
        o.fit(X, 6, 0.5, 0, 1e-6, 10)          # k > n
    with pytest.raises(ValueError):
        o.fit(X, 2, 0.0, 0, 1e-6, 10)          # f outside (0, 1]
    with pytest.raises(ValueError):
        o.fit(X, 2, 0.5, 0, -1.0, 10)          # tol < 0
    with pytest.raises(ValueError):
        o.fit(X, 2, 0.5, 0, 1e-6, 0)           # max_iter < 1
