"""FP64 CPU oracle for the two-stage k-means (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and the
oracle never imports the product package: the two share no code.

The arithmetic lives in ``kmeans_oracle.c`` (plain C, FP64); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  Each function
cites the passage of the paper (arXiv 1108.1351) it follows:

* :func:`sample` -- the fast-stage subset S_s and the initial centers
  (the Algorithm's per% subset and its random initial centers; Section 2).
* :func:`assign` -- squared distance (Eq. 1 without the root, Algorithm) and
  nearest-center label.
* :func:`lloyd_step` -- one Lloyd iteration (Section 4.1): assignment, J
  (Eq. 3), means, largest center movement.
* :func:`lloyd_stage` / :func:`fit` -- the stage loop and the two-stage fit
  (Algorithm; Section 2: the slow stage starts from the fast stage's centers).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmeans_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libkmeans_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the .so path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-lm"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleResult(ctypes.Structure):
    _fields_ = [
        ("J", ctypes.c_double),
        ("iters_fast", ctypes.c_int32),
        ("iters_slow", ctypes.c_int32),
        ("converged_fast", ctypes.c_int32),
        ("converged_slow", ctypes.c_int32),
        ("empty_clusters", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("subset_size", ctypes.c_int64),
        ("distance_evals", ctypes.c_int64),
    ]


def _bind(lib):
    P = ctypes.c_void_p
    i64, i32, u64, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
    lib.oracle_splitmix64_at.restype = u64
    lib.oracle_splitmix64_at.argtypes = [u64, u64]
    lib.oracle_subset_size.restype = i64
    lib.oracle_subset_size.argtypes = [i64, i32, f64]
    lib.oracle_sample.restype = ctypes.c_int
    lib.oracle_sample.argtypes = [i64, i32, f64, u64, P, P]
    lib.oracle_assign.restype = ctypes.c_int
    lib.oracle_assign.argtypes = [P, i64, i32, i32, P, P, P, i32]
    lib.oracle_lloyd_step.restype = ctypes.c_int
    lib.oracle_lloyd_step.argtypes = [P, i64, i32, i32, P, P, P, P, P, P, i32]
    lib.oracle_lloyd_stage.restype = ctypes.c_int
    lib.oracle_lloyd_stage.argtypes = [P, i64, i32, i32, P, f64, i32, P, P, P, P, P,
                                       P, P, i32]
    lib.oracle_fit.restype = ctypes.c_int
    lib.oracle_fit.argtypes = [P, i64, i32, i32, f64, u64, f64, f64, i32, P, P, P,
                               P, P, P, P, ctypes.POINTER(OracleResult), i32]
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def build_variant(source_text: str, tag: str) -> "Oracle":
    """Compile a modified copy of the oracle source (used by the tests that
    plant a mistake in the oracle to show that the pins catch it)."""
    import tempfile
    d = tempfile.mkdtemp(prefix=f"oracle_{tag}_")
    src = os.path.join(d, "kmeans_oracle.c")
    with open(src, "w") as fh:
        fh.write(source_text)
    so = os.path.join(d, "liboracle_variant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", src,
                    "-lm", "-o", so], check=True)
    return Oracle(_bind(ctypes.CDLL(so)))


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f32(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("X must be 2-D (n, d)")
    return X


def _f64(C):
    return np.ascontiguousarray(C, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


class Oracle:
    """Bound oracle library; module-level functions use the default build."""

    def __init__(self, lib):
        self.lib = lib

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())

    def splitmix64_at(self, seed: int, i: int) -> int:
        """Output ``i`` of the SplitMix64 stream seeded with ``seed``."""
        return int(self.lib.oracle_splitmix64_at(seed & (2**64 - 1), i))

    def subset_size(self, n: int, k: int, f: float) -> int:
        """m = min(n, max(k, ceil(f*n)))."""
        return int(self.lib.oracle_subset_size(n, k, f))

    def sample(self, n: int, k: int, f: float, seed: int):
        """(subset indices ascending, init positions within the subset)."""
        m = self.subset_size(n, k, f)
        sub = np.empty(m, dtype=np.int64)
        pos = np.empty(k, dtype=np.int64)
        _check(self.lib.oracle_sample(n, k, f, seed & (2**64 - 1), _ptr(sub), _ptr(pos)), "sample")
        return sub, pos

    def assign(self, X, C, nthreads: int = 1):
        """(labels int32, minimal squared distance FP64) for each row of X."""
        X = _f32(X)
        C = _f64(C)
        n, d = X.shape
        k = C.shape[0]
        lab = np.empty(n, dtype=np.int32)
        dm = np.empty(n, dtype=np.float64)
        _check(self.lib.oracle_assign(_ptr(X), n, d, k, _ptr(C), _ptr(lab), _ptr(dm), nthreads),
               "assign")
        return lab, dm

    def lloyd_step(self, X, C, nthreads: int = 1):
        """One Lloyd iteration from centers C: (C_new, labels, J, shift, empty)."""
        X = _f32(X)
        C = _f64(C)
        n, d = X.shape
        k = C.shape[0]
        Cn = np.empty_like(C)
        lab = np.empty(n, dtype=np.int32)
        J = ctypes.c_double()
        sh = ctypes.c_double()
        em = ctypes.c_int32()
        _check(self.lib.oracle_lloyd_step(_ptr(X), n, d, k, _ptr(C), _ptr(Cn), _ptr(lab),
                                         ctypes.addressof(J), ctypes.addressof(sh),
                                         ctypes.addressof(em), nthreads), "lloyd_step")
        return Cn, lab, J.value, sh.value, em.value

    def lloyd_stage(self, X, C, tol: float, max_iter: int, nthreads: int = 1):
        """Lloyd loop from C: dict with centers, labels, J, iters, converged, trajectories."""
        X = _f32(X)
        C = _f64(C).copy()
        n, d = X.shape
        k = C.shape[0]
        lab = np.empty(n, dtype=np.int32)
        tJ = np.zeros(max_iter, dtype=np.float64)
        ts = np.zeros(max_iter, dtype=np.float64)
        J = ctypes.c_double()
        it = ctypes.c_int32()
        cv = ctypes.c_int32()
        em = ctypes.c_int32()
        _check(self.lib.oracle_lloyd_stage(_ptr(X), n, d, k, _ptr(C), tol, max_iter, _ptr(lab),
                                          ctypes.addressof(J), ctypes.addressof(it),
                                          ctypes.addressof(cv), ctypes.addressof(em),
                                          _ptr(tJ), _ptr(ts), nthreads), "lloyd_stage")
        q = it.value
        return dict(centers=C, labels=lab, J=J.value, iters=q, converged=bool(cv.value),
                    empty=em.value, traj_J=tJ[:q].copy(), traj_shift=ts[:q].copy())

    def fit(self, X, k: int, f: float, seed: int, tol: float, max_iter: int,
            tol_fast: float = 0.0, nthreads: int = 1):
        """Two-stage fit.  Returns a dict with centers, labels, J, per-stage counts,
        the fast stage's final centers and both stages' J / shift trajectories."""
        X = _f32(X)
        n, d = X.shape
        C = np.empty((k, d), dtype=np.float64)
        Cf = np.empty((k, d), dtype=np.float64)
        lab = np.empty(n, dtype=np.int32)
        tJf = np.zeros(max_iter)
        tsf = np.zeros(max_iter)
        tJs = np.zeros(max_iter)
        tss = np.zeros(max_iter)
        r = OracleResult()
        _check(self.lib.oracle_fit(_ptr(X), n, d, k, f, seed & (2**64 - 1), tol_fast, tol, max_iter,
                                  _ptr(C), _ptr(lab), _ptr(Cf), _ptr(tJf), _ptr(tsf), _ptr(tJs),
                                  _ptr(tss), ctypes.byref(r), nthreads), "fit")
        return dict(centers=C, labels=lab, J=r.J, iters_fast=r.iters_fast, iters_slow=r.iters_slow,
                    converged_fast=bool(r.converged_fast), converged_slow=bool(r.converged_slow),
                    empty_clusters=r.empty_clusters, subset_size=r.subset_size,
                    distance_evals=r.distance_evals, fast_centers=Cf,
                    traj_J_fast=tJf[:r.iters_fast].copy(), traj_shift_fast=tsf[:r.iters_fast].copy(),
                    traj_J_slow=tJs[:r.iters_slow].copy(), traj_shift_slow=tss[:r.iters_slow].copy())


_default = None


def _default_oracle() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(_load())
    return _default


def max_threads() -> int:
    return _default_oracle().max_threads()


def splitmix64_at(seed: int, i: int) -> int:
    return _default_oracle().splitmix64_at(seed, i)


def subset_size(n: int, k: int, f: float) -> int:
    return _default_oracle().subset_size(n, k, f)


def sample(n: int, k: int, f: float, seed: int):
    return _default_oracle().sample(n, k, f, seed)


def assign(X, C, nthreads: int = 1):
    return _default_oracle().assign(X, C, nthreads)


def lloyd_step(X, C, nthreads: int = 1):
    return _default_oracle().lloyd_step(X, C, nthreads)


def lloyd_stage(X, C, tol: float, max_iter: int, nthreads: int = 1):
    return _default_oracle().lloyd_stage(X, C, tol, max_iter, nthreads)


def fit(X, k: int, f: float, seed: int, tol: float, max_iter: int, tol_fast: float = 0.0,
        nthreads: int = 1):
    return _default_oracle().fit(X, k, f, seed, tol, max_iter, tol_fast, nthreads)
