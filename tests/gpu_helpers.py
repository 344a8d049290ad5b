"""Shared checks for the GPU parity tests (tolerances derived in the design notes).

* Labels: bit-exact (the library decides near ties in the oracle's own FP64 form).
* Centers: |c_gpu - c_oracle| <= 1e-10 * max_t |c_oracle[j, t]| + 2^-F per
  coordinate, F = min(120, 46 - E) where 2^E > max|x|: the second term is the
  documented fixed-point grid of the exact cluster sums.
* J: |J_gpu - J_oracle| <= 1e-9 * J_oracle (an exactly zero J must be zero).
  The library forms J without cancellation (exact integer within-cluster part
  plus double-word center displacements), so its error is a few FP64 ulps of J
  itself; only coordinates below the fixed-point grid (|x| < 2^(E-23)) could
  add more, and the test data hold none that matter.
"""
import math

import numpy as np


def grid_term(X) -> float:
    mx = float(np.max(np.abs(X))) if X.size else 0.0
    if mx == 0.0:
        return 0.0
    E = math.frexp(mx)[1]
    return 2.0 ** -min(120, 46 - E)


def assert_centers_close(got, want, X, rel=1e-10):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape
    scale = np.max(np.abs(want), axis=1, keepdims=True)
    tol = rel * scale + grid_term(X)
    bad = np.abs(got - want) > tol
    assert not bad.any(), f"{bad.sum()} center coordinates off; worst {np.max(np.abs(got - want) - tol)}"


def assert_J_close(got, want, X=None, rel=1e-9):
    assert abs(got - want) <= rel * abs(want), (got, want, abs(got - want) / max(abs(want), 1e-300))


def to_np(a):
    if hasattr(a, "detach"):
        return a.detach().cpu().numpy()
    return np.asarray(a)
