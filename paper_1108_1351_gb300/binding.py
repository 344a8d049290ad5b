"""ctypes binding of libkmeans2 (argument marshalling only).

Every step of the method runs in the CUDA library; this module converts torch
tensors / numpy arrays to pointers, picks torch's current stream and wraps the
results.  It never falls back to another implementation: if the shared object
is missing it raises, telling the caller to build it.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from dataclasses import dataclass, field

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# KMEANS2_DEBUG=1 loads the debug build (device-side index checks that report
# an error status instead of trapping; build it with build.build(debug=True))
LIB_PATH = os.path.join(_HERE, "libkmeans2_debug.so" if os.environ.get("KMEANS2_DEBUG") == "1"
                        else "libkmeans2.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "kmeans2.h")

PRECISION = {"fp32": 0, "bf16": 1, "auto": 2, "tf32x3": 3, "fp16": 4}
_lock = threading.Lock()
_lib = None


class KMeans2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.kmeans2_strerror(status).decode()
        detail = lib.kmeans2_last_error().decode()
        super().__init__(f"{where}: {msg} (status {status})" + (f" [{detail}]" if detail else ""))
        self.status = status


class Profile(ctypes.Structure):
    _fields_ = [
        ("kernel_launches", ctypes.c_int64),
        ("assign_launches", ctypes.c_int64),
        ("assign_ms", ctypes.c_double),
        ("assign_flops", ctypes.c_double),
        ("assign_bytes", ctypes.c_double),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("deterministic", ctypes.c_int32),
        ("tol_fast", ctypes.c_double),
        ("init_centers", ctypes.c_void_p),
        ("start_stage", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("traj_J_fast", ctypes.c_void_p),
        ("traj_shift_fast", ctypes.c_void_p),
        ("traj_J_slow", ctypes.c_void_p),
        ("traj_shift_slow", ctypes.c_void_p),
        ("profile", ctypes.c_void_p),
        ("traj_centers_fast", ctypes.c_void_p),
        ("traj_centers_slow", ctypes.c_void_p),
        ("traj_counts_fast", ctypes.c_void_p),
        ("traj_counts_slow", ctypes.c_void_p),
    ]


class Job(ctypes.Structure):
    _fields_ = [
        ("X", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("d", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("subset_fraction", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("centers_out", ctypes.c_void_p),
        ("labels_out", ctypes.c_void_p),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("J", ctypes.c_double),
        ("iters_fast", ctypes.c_int32),
        ("iters_slow", ctypes.c_int32),
        ("converged_fast", ctypes.c_int32),
        ("converged_slow", ctypes.c_int32),
        ("empty_clusters", ctypes.c_int32),
        ("precision_used", ctypes.c_int32),
        ("subset_size", ctypes.c_int64),
        ("rechecked_points", ctypes.c_int64),
        ("distance_evals", ctypes.c_int64),
        ("shift_fast", ctypes.c_double),
        ("shift_slow", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("undecided_fast", ctypes.c_int64),
        ("undecided_slow", ctypes.c_int64),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("admitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("failed", ctypes.c_int64),
        ("rejected", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("queued", ctypes.c_int32),
        ("running", ctypes.c_int32),
        ("slots", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("hbm_budget", ctypes.c_uint64),
        ("hbm_in_use", ctypes.c_uint64),
        ("hbm_peak", ctypes.c_uint64),
    ]


class TicketTimes(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class Exchange(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("reserved", ctypes.c_int32), ("count", ctypes.c_int64)]


PENDING = 1
XCHG_SUM_I64, XCHG_MAX_I64, XCHG_SUM_F64 = 0, 1, 2

MATERIALIZE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
CONSUME_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p)


class _DeviceView:
    """__cuda_array_interface__ of library-owned device memory (zero-copy view)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def load():
    """Load libkmeans2.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u64, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_uint64, ctypes.c_double)
        lib.kmeans2_default_options.restype = None
        lib.kmeans2_default_options.argtypes = [ctypes.POINTER(Options)]
        lib.kmeans2_fit.restype = ctypes.c_int
        lib.kmeans2_fit.argtypes = [P, i64, i32, i32, f64, u64, f64, i32, P, P,
                                    ctypes.POINTER(Result), ctypes.POINTER(Options)]
        lib.kmeans2_fit_streamed.restype = ctypes.c_int
        lib.kmeans2_fit_streamed.argtypes = [P, i64, i32, i32, f64, u64, f64, i32, i64, P, P,
                                             ctypes.POINTER(Result), ctypes.POINTER(Options)]
        lib.kmeans2_fit_sharded.restype = ctypes.c_int
        lib.kmeans2_fit_sharded.argtypes = [P, i64, i32, i32, f64, u64, f64, i32, i32, P, P,
                                            ctypes.POINTER(Result), ctypes.POINTER(Options)]
        lib.kmeans2_shard_exchange_elems.restype = i64
        lib.kmeans2_shard_exchange_elems.argtypes = [i32, i32]
        lib.kmeans2_shard_create.restype = ctypes.c_int
        lib.kmeans2_shard_create.argtypes = [P, i64, i64, i64, i32, i32, f64, u64, f64, i32, P,
                                             ctypes.POINTER(Options), ctypes.POINTER(P)]
        lib.kmeans2_shard_advance.restype = ctypes.c_int
        lib.kmeans2_shard_advance.argtypes = [P, ctypes.POINTER(Exchange)]
        lib.kmeans2_shard_result.restype = ctypes.c_int
        lib.kmeans2_shard_result.argtypes = [P, P, P, ctypes.POINTER(Result)]
        lib.kmeans2_shard_destroy.restype = None
        lib.kmeans2_shard_destroy.argtypes = [P]
        lib.kmeans_step.restype = ctypes.c_int
        lib.kmeans_step.argtypes = [P, i64, i32, i32, P, P, P, P, P, P, ctypes.POINTER(Options)]
        lib.kmeans2_fit_batched.restype = ctypes.c_int
        lib.kmeans2_fit_batched.argtypes = [i32, ctypes.POINTER(Job), ctypes.POINTER(Result),
                                            ctypes.POINTER(Options)]
        lib.kmeans2_batched_tile_shape.restype = ctypes.c_int
        lib.kmeans2_batched_tile_shape.argtypes = [i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                                   ctypes.POINTER(i32)]
        lib.kmeans_step_noalloc.restype = ctypes.c_int
        lib.kmeans_step_noalloc.argtypes = [P, i64, i32, i32, P, P, P, P, P, P, P]
        lib.kmeans2_fit_footprint.restype = u64
        lib.kmeans2_fit_footprint.argtypes = [i64, i32, i32, f64, i32, i32, i32, i32]
        lib.kmeans2_server_create.restype = P
        lib.kmeans2_server_create.argtypes = [u64, i32, ctypes.POINTER(Options)]
        lib.kmeans2_server_submit.restype = ctypes.c_int
        lib.kmeans2_server_submit.argtypes = [P, ctypes.POINTER(Job), ctypes.POINTER(u64)]
        lib.kmeans2_server_submit_lazy.restype = ctypes.c_int
        lib.kmeans2_server_submit_lazy.argtypes = [P, ctypes.POINTER(Job), MATERIALIZE_FN,
                                                   CONSUME_FN, P, ctypes.POINTER(u64)]
        lib.kmeans2_server_wait_any.restype = ctypes.c_int
        lib.kmeans2_server_wait_any.argtypes = [P, f64, ctypes.POINTER(u64)]
        lib.kmeans2_server_poll.restype = ctypes.c_int
        lib.kmeans2_server_poll.argtypes = [P, u64, ctypes.POINTER(Result),
                                            ctypes.POINTER(TicketTimes)]
        lib.kmeans2_server_wait.restype = ctypes.c_int
        lib.kmeans2_server_wait.argtypes = [P, u64, f64, ctypes.POINTER(Result),
                                            ctypes.POINTER(TicketTimes)]
        lib.kmeans2_server_stats_get.restype = ctypes.c_int
        lib.kmeans2_server_stats_get.argtypes = [P, ctypes.POINTER(ServerStats)]
        lib.kmeans2_server_set_policy.restype = ctypes.c_int
        lib.kmeans2_server_set_policy.argtypes = [P, i32, f64]
        lib.kmeans2_server_now.restype = f64
        lib.kmeans2_server_now.argtypes = [P]
        lib.kmeans2_server_destroy.restype = None
        lib.kmeans2_server_destroy.argtypes = [P]
        lib.kmeans2_subset_size.restype = i64
        lib.kmeans2_subset_size.argtypes = [i64, i32, f64]
        lib.kmeans2_sample.restype = ctypes.c_int
        lib.kmeans2_sample.argtypes = [i64, i32, f64, u64, P, P, P]
        lib.kmeans2_strerror.restype = ctypes.c_char_p
        lib.kmeans2_strerror.argtypes = [ctypes.c_int]
        lib.kmeans2_last_error.restype = ctypes.c_char_p
        lib.kmeans2_last_error.argtypes = []
        lib.kmeans2_release_memory.restype = ctypes.c_int
        lib.kmeans2_release_memory.argtypes = []
        lib.kmeans2_version.restype = i32
        lib.kmeans2_version.argtypes = []
        _lib = lib
    return _lib


def declared_symbols() -> list[str]:
    """Names of the entry points declared in include/kmeans2.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"KMEANS2_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)))


# ------------------------------------------------------------------ marshalling

def _is_torch(a) -> bool:
    return isinstance(a, torch.Tensor)


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _as_points(X):
    if _is_torch(X):
        if X.dtype != torch.float32 or X.dim() != 2:
            raise TypeError("X must be a 2-D float32 tensor")
        return X.contiguous()
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise TypeError("X must be 2-D")
    return X


def _as_centers(C, like, k=None, d=None):
    """FP64 contiguous centers (k x d; k taken from C when not given)."""
    if C is None:
        return None
    if _is_torch(C):
        C = C.to(dtype=torch.float64).contiguous()
    else:
        C = np.ascontiguousarray(C, dtype=np.float64)
        if _is_torch(like) and like.is_cuda:
            C = torch.as_tensor(C, device=like.device)
    kk = C.shape[0] if (k is None and C.ndim == 2) else k
    if C.ndim != 2 or (d is not None and C.shape[1] != d) or C.shape[0] != kk:
        raise ValueError(f"centers must have shape ({kk}, {d}), got {tuple(C.shape)}")
    return C


_TORCH_KIND = {"f64": torch.float64, "i32": torch.int32, "i64": torch.int64}
_NP_KIND = {"f64": np.float64, "i32": np.int32, "i64": np.int64}


def _empty(like, shape, kind):
    if _is_torch(like):
        return torch.empty(shape, dtype=_TORCH_KIND[kind], device=like.device)
    return np.empty(shape, dtype=_NP_KIND[kind])


def _out(buf, like, shape, kind, name):
    """A caller-given output buffer after checking its type, size and layout
    (the library writes exactly prod(shape) elements), else a new one where
    `like` lives."""
    if buf is None:
        return _empty(like, shape, kind)
    count = int(np.prod(shape))
    if _is_torch(buf):
        ok = buf.dtype == _TORCH_KIND[kind] and buf.is_contiguous() and buf.numel() == count
    else:
        ok = (isinstance(buf, np.ndarray) and buf.dtype == _NP_KIND[kind]
              and buf.flags.c_contiguous and buf.flags.writeable and buf.size == count)
    if not ok:
        raise ValueError(f"{name} must be a contiguous, writable {kind} buffer of {count} elements")
    return buf


def _stream_of(X, stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if _is_torch(X) and X.is_cuda:
        return torch.cuda.current_stream(X.device).cuda_stream
    return None


def _check_devices(X, *bufs):
    """Every CUDA tensor of a call must live on the device the call runs on
    (X's device, else the current one): the kernels read and write them
    directly, and another GPU's memory is not addressable without peer access."""
    dev = X.device if (_is_torch(X) and X.is_cuda) else None
    if dev is None and torch.cuda.is_available():
        dev = torch.device("cuda", torch.cuda.current_device())
    for b in bufs:
        if _is_torch(b) and b.is_cuda and b.device != dev:
            raise ValueError(f"a CUDA tensor on {b.device} was passed to a call running on {dev}")


class _device_of:
    """Make X's device current for the call (the library uses the current device)."""

    def __init__(self, X):
        self.dev = X.device if (_is_torch(X) and X.is_cuda) else None

    def __enter__(self):
        self.ctx = torch.cuda.device(self.dev) if self.dev is not None else None
        if self.ctx is not None:
            self.ctx.__enter__()

    def __exit__(self, *a):
        if self.ctx is not None:
            self.ctx.__exit__(*a)


@dataclass
class FitResult:
    centers: object
    labels: object
    J: float
    iters_fast: int
    iters_slow: int
    converged_fast: bool
    converged_slow: bool
    empty_clusters: int
    subset_size: int
    rechecked_points: int
    distance_evals: int
    shift_fast: float
    shift_slow: float
    seconds: float
    precision_used: str
    traj: dict = field(default_factory=dict)
    undecided: tuple = (0, 0)     # FP16 form: rows its single pass left undecided per stage


def fit(X, k: int, subset_fraction: float, seed: int, tol: float, max_iter: int, *,
        tol_fast: float = 0.0, precision: str = "auto", init_centers=None, start_stage: int = 0,
        use_graph: bool = True, stream=None, trajectories: bool = False,
        center_trajectories: bool = False, centers_out=None, labels_out=None,
        profile: "Profile | None" = None) -> FitResult:
    """Two-stage k-means (kmeans2_fit).  Outputs live where X lives (device
    tensors for a CUDA tensor, host arrays otherwise) unless given.
    trajectories: per-iteration J and max center movement of both stages;
    center_trajectories: also the updated centers (iterations x k x d) and the
    cluster sizes (iterations x k) of every iteration."""
    lib = load()
    X = _as_points(X)
    n, d = X.shape
    C0 = _as_centers(init_centers, X, k, d)
    cen = _out(centers_out, X, (k, d), "f64", "centers_out")
    lab = _out(labels_out, X, (n,), "i32", "labels_out")
    _check_devices(X, C0, cen, lab)
    opt = Options()
    lib.kmeans2_default_options(ctypes.byref(opt))
    opt.precision = PRECISION[precision]
    opt.tol_fast = tol_fast
    opt.init_centers = _ptr(C0)
    opt.start_stage = start_stage
    opt.use_graph = 1 if use_graph else 0
    opt.stream = _stream_of(X, stream)
    opt.profile = ctypes.addressof(profile) if profile is not None else None
    traj = {}
    if trajectories:
        for key in ("J_fast", "shift_fast", "J_slow", "shift_slow"):
            traj[key] = np.zeros(max_iter, dtype=np.float64)
            setattr(opt, "traj_" + key, traj[key].ctypes.data)
    if center_trajectories:
        for st in ("fast", "slow"):
            traj["centers_" + st] = np.zeros((max_iter, k, d), dtype=np.float64)
            traj["counts_" + st] = np.zeros((max_iter, k), dtype=np.int64)
            setattr(opt, "traj_centers_" + st, traj["centers_" + st].ctypes.data)
            setattr(opt, "traj_counts_" + st, traj["counts_" + st].ctypes.data)
    res = Result()
    with _device_of(X):
        rc = lib.kmeans2_fit(_ptr(X), n, d, k, subset_fraction, seed & (2**64 - 1), tol, max_iter,
                             _ptr(cen), _ptr(lab), ctypes.byref(res), ctypes.byref(opt))
    if rc != 0:
        raise KMeans2Error(rc, "kmeans2_fit")
    if traj:
        lim = {"fast": res.iters_fast, "slow": res.iters_slow}
        traj = {key: v[:lim[key.rsplit("_", 1)[1]]] for key, v in traj.items()}
    return FitResult(centers=cen, labels=lab, J=res.J, iters_fast=res.iters_fast,
                     iters_slow=res.iters_slow, converged_fast=bool(res.converged_fast),
                     converged_slow=bool(res.converged_slow), empty_clusters=res.empty_clusters,
                     subset_size=res.subset_size, rechecked_points=res.rechecked_points,
                     distance_evals=res.distance_evals, shift_fast=res.shift_fast,
                     shift_slow=res.shift_slow, seconds=res.seconds,
                     precision_used={0: "fp32", 1: "bf16", 3: "tf32x3", 4: "fp16"}.get(res.precision_used, "?"),
                     traj=traj, undecided=(res.undecided_fast, res.undecided_slow))


def fit_streamed(X, k: int, subset_fraction: float, seed: int, tol: float, max_iter: int,
                 chunk_points: int, *, tol_fast: float = 0.0, init_centers=None,
                 start_stage: int = 0, stream=None, centers_out=None,
                 labels_out=None, profile: "Profile | None" = None) -> "FitResult":
    """Two-stage k-means on host-resident X (kmeans2_fit_streamed); same
    results as fit().  chunk_points > 0: X is staged through the GPU in chunks
    of that many rows (0: 2^26 rows); < 0: page-locked X is read in place by
    the kernels over the CPU-GPU link (pageable X falls back to chunks).
    X: a numpy array or a CPU tensor (pinned for in-place reads and
    asynchronous copies).  Outputs are host arrays unless given."""
    lib = load()
    if _is_torch(X) and X.is_cuda:
        raise TypeError("fit_streamed takes host-resident X")
    X = _as_points(X)
    n, d = X.shape
    C0 = _as_centers(init_centers, X, k, d)
    cen = _out(centers_out, None, (k, d), "f64", "centers_out")
    lab = _out(labels_out, None, (n,), "i32", "labels_out")
    _check_devices(X, C0, cen, lab)
    opt = Options()
    lib.kmeans2_default_options(ctypes.byref(opt))
    opt.precision = PRECISION["fp32"]
    opt.tol_fast = tol_fast
    opt.init_centers = _ptr(C0) if C0 is not None else None
    opt.start_stage = start_stage
    opt.profile = ctypes.addressof(profile) if profile is not None else None
    dev = torch.device("cuda", torch.cuda.current_device())
    opt.stream = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    res = Result()
    with torch.cuda.device(dev):
        rc = lib.kmeans2_fit_streamed(_ptr(X), n, d, k, subset_fraction, seed & (2**64 - 1), tol,
                                      max_iter, int(chunk_points), _ptr(cen), _ptr(lab),
                                      ctypes.byref(res), ctypes.byref(opt))
    if rc != 0:
        raise KMeans2Error(rc, "kmeans2_fit_streamed")
    return _fit_result(res, cen, lab)


def fit_sharded(X, k: int, subset_fraction: float, seed: int, tol: float, max_iter: int,
                shards: int, *, tol_fast: float = 0.0, precision: str = "auto",
                init_centers=None, start_stage: int = 0, stream=None, centers_out=None,
                labels_out=None) -> FitResult:
    """fit() run as `shards` data-parallel ranks on this GPU (kmeans2_fit_sharded):
    row blocks with their own sums and labels, partials all-reduced in rank
    order each iteration.  Equal to fit() bit for bit."""
    lib = load()
    X = _as_points(X)
    n, d = X.shape
    C0 = _as_centers(init_centers, X, k, d)
    cen = _out(centers_out, X, (k, d), "f64", "centers_out")
    lab = _out(labels_out, X, (n,), "i32", "labels_out")
    _check_devices(X, C0, cen, lab)
    opt = Options()
    lib.kmeans2_default_options(ctypes.byref(opt))
    opt.precision = PRECISION[precision]
    opt.tol_fast = tol_fast
    opt.init_centers = _ptr(C0)
    opt.start_stage = start_stage
    opt.stream = _stream_of(X, stream)
    res = Result()
    with _device_of(X):
        rc = lib.kmeans2_fit_sharded(_ptr(X), n, d, k, subset_fraction, seed & (2**64 - 1), tol,
                                     max_iter, int(shards), _ptr(cen), _ptr(lab),
                                     ctypes.byref(res), ctypes.byref(opt))
    if rc != 0:
        raise KMeans2Error(rc, "kmeans2_fit_sharded")
    return _fit_result(res, cen, lab)


class Shard:
    """One rank's session of a data-parallel fit (kmeans2_shard_*).

    ``advance()`` runs the rank to its next exchange point and returns
    ``(op, buf)``: buf (a view of the session's device exchange buffer, int64
    or float64) must be all-reduced across ranks with op ("sum" or "max") in
    place before the next ``advance()``; None once the fit has finished."""

    def __init__(self, X_local, row0: int, n_total: int, k: int, subset_fraction: float,
                 seed: int, tol: float, max_iter: int, *, tol_fast: float = 0.0,
                 precision: str = "auto", init_centers=None, start_stage: int = 0, stream=None,
                 profile: "Profile | None" = None):
        lib = load()
        if not (_is_torch(X_local) and X_local.is_cuda):
            raise TypeError("Shard takes a CUDA tensor of this rank's rows")
        self.X = _as_points(X_local)
        self.n_local, self.d = self.X.shape
        self.k = int(k)
        self.device = self.X.device
        E = int(lib.kmeans2_shard_exchange_elems(self.d, self.k))
        self.xbuf = torch.zeros(E, dtype=torch.int64, device=self.device)
        self._C0 = _as_centers(init_centers, self.X, self.k, self.d)
        _check_devices(self.X, self._C0)
        opt = Options()
        lib.kmeans2_default_options(ctypes.byref(opt))
        opt.precision = PRECISION[precision]
        opt.tol_fast = tol_fast
        opt.init_centers = _ptr(self._C0)
        opt.start_stage = start_stage
        opt.stream = _stream_of(self.X, stream)
        if profile is not None:
            opt.profile = ctypes.addressof(profile)      # kernel launches of the session
        h = ctypes.c_void_p()
        with _device_of(self.X):
            rc = lib.kmeans2_shard_create(_ptr(self.X) if self.n_local else None, self.n_local,
                                          int(row0), int(n_total), self.d, self.k,
                                          subset_fraction, seed & (2**64 - 1), tol, max_iter,
                                          self.xbuf.data_ptr(), ctypes.byref(opt),
                                          ctypes.byref(h))
        if rc != 0:
            raise KMeans2Error(rc, "kmeans2_shard_create")
        self._h = h

    def advance(self):
        x = Exchange()
        with _device_of(self.X):
            rc = load().kmeans2_shard_advance(self._h, ctypes.byref(x))
        if rc == 0:
            return None
        if rc != PENDING:
            raise KMeans2Error(rc, "kmeans2_shard_advance")
        buf = self.xbuf.view(torch.float64) if x.op == XCHG_SUM_F64 else self.xbuf
        return ("max" if x.op == XCHG_MAX_I64 else "sum"), buf[:x.count]

    def result(self) -> FitResult:
        cen = torch.empty((self.k, self.d), dtype=torch.float64, device=self.device)
        lab = torch.empty((self.n_local,), dtype=torch.int32, device=self.device)
        res = Result()
        with _device_of(self.X):
            rc = load().kmeans2_shard_result(self._h, cen.data_ptr(), lab.data_ptr(),
                                             ctypes.byref(res))
        if rc != 0:
            raise KMeans2Error(rc, "kmeans2_shard_result")
        return _fit_result(res, cen, lab)

    def close(self):
        if getattr(self, "_h", None):
            load().kmeans2_shard_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fit_data_parallel(X_local, row0: int, n_total: int, k: int, subset_fraction: float,
                      seed: int, tol: float, max_iter: int, *, group=None, shard_factory=None,
                      **kw) -> FitResult:
    """The fit of the rows [row0, row0 + len(X_local)) of a data set split over
    the ranks of a torch.distributed group (one rank per GPU): each rank runs
    its Shard and every exchange is one all_reduce over the group.  Returns
    this rank's labels and the replicated centers; all equal fit() on the
    whole data.  ``shard_factory`` replaces Shard (same constructor and
    methods)."""
    import torch.distributed as dist

    make = shard_factory or Shard
    sh = make(X_local, row0, n_total, k, subset_fraction, seed, tol, max_iter, **kw)
    ops = {"sum": dist.ReduceOp.SUM, "max": dist.ReduceOp.MAX}
    # a gloo group reduces host tensors: stage a device buffer through host
    # memory (the shard's stream is synchronised when advance() returns, and
    # the copy back is ordered before its next kernels on the same stream)
    stage = dist.get_backend(group) == "gloo"
    try:
        while True:
            x = sh.advance()
            if x is None:
                break
            op, buf = x
            if stage and buf.is_cuda:
                h = buf.cpu()
                dist.all_reduce(h, op=ops[op], group=group)
                buf.copy_(h)
            else:
                dist.all_reduce(buf, op=ops[op], group=group)
        return sh.result()
    finally:
        sh.close()


def release_memory() -> None:
    """Return the library's unused device scratch to the driver
    (kmeans2_release_memory; waits for the current device)."""
    rc = load().kmeans2_release_memory()
    if rc != 0:
        raise KMeans2Error(rc, "kmeans2_release_memory")


def _fit_result(r, cen, lab, traj=None) -> FitResult:
    return FitResult(centers=cen, labels=lab, J=r.J, iters_fast=r.iters_fast,
                     iters_slow=r.iters_slow, converged_fast=bool(r.converged_fast),
                     converged_slow=bool(r.converged_slow), empty_clusters=r.empty_clusters,
                     subset_size=r.subset_size, rechecked_points=r.rechecked_points,
                     distance_evals=r.distance_evals, shift_fast=r.shift_fast,
                     shift_slow=r.shift_slow, seconds=r.seconds,
                     precision_used={0: "fp32", 1: "bf16", 3: "tf32x3", 4: "fp16"}.get(r.precision_used, "?"),
                     traj=traj or {})


def footprint(n: int, d: int, k: int, subset_fraction: float, max_iter: int, *,
              precision: str = "auto", x_on_host: bool = False,
              labels_on_host: bool = False) -> int:
    """Device bytes kmeans2_fit allocates for one problem (kmeans2_fit_footprint)."""
    return int(load().kmeans2_fit_footprint(n, d, k, subset_fraction, max_iter,
                                            PRECISION[precision], int(x_on_host),
                                            int(labels_on_host)))


@dataclass
class Served:
    """A finished server job: its status, result (None on failure) and the
    server-clock times of submission, admission and completion."""
    ticket: int
    status: int
    result: "FitResult | None"
    t_submit: float
    t_admit: float
    t_done: float


class Server:
    """Continuous-batching request loop (kmeans2_server_*).

    ``submit`` queues a job and returns its ticket at once; ``poll`` / ``wait``
    return a ``Served`` once the job has finished.  The server holds references
    to each job's tensors until the job has been collected.  ``use_graph``:
    stage loops as while-graphs (True) or host-driven (False); None picks
    host-driven loops for several slots, so that jobs interleave."""

    POLICY = {"fifo": 0, "shortest": 1}

    def __init__(self, hbm_budget: int = 0, max_slots: int = 4, *, precision: str = "auto",
                 tol_fast: float = 0.0, policy: str = "fifo", aging_s: float = 30.0,
                 use_graph: "bool | None" = None, device=None):
        lib = load()
        opt = Options()
        lib.kmeans2_default_options(ctypes.byref(opt))
        opt.precision = PRECISION[precision]
        opt.tol_fast = tol_fast
        # None: host-driven stage loops when several jobs run at once (another
        # job's while-graph waits for a running one), graphs for a single slot
        if use_graph is None:
            use_graph = max_slots == 1
        opt.use_graph = 1 if use_graph else 0
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.device = dev
        with torch.cuda.device(dev):
            self._h = lib.kmeans2_server_create(int(hbm_budget), int(max_slots), ctypes.byref(opt))
        if not self._h:
            raise KMeans2Error(-1, "kmeans2_server_create")
        rc = lib.kmeans2_server_set_policy(self._h, self.POLICY[policy], float(aging_s))
        if rc != 0:
            lib.kmeans2_server_destroy(self._h)
            self._h = None
            raise KMeans2Error(rc, "kmeans2_server_set_policy")
        self._refs: dict[int, tuple] = {}
        self._mu = threading.Lock()

    def submit(self, X, k: int, subset_fraction: float, seed: int, tol: float, max_iter: int, *,
               centers_out=None, labels_out=None) -> int:
        lib = load()
        X = _as_points(X)
        n, d = X.shape
        cen = _out(centers_out, X, (k, d), "f64", "centers_out")
        lab = _out(labels_out, X, (n,), "i32", "labels_out")
        _check_devices(X, cen, lab)
        job = Job(X=_ptr(X), n=n, d=d, k=int(k), subset_fraction=float(subset_fraction),
                  seed=int(seed) & (2**64 - 1), tol=float(tol), max_iter=int(max_iter), reserved=0,
                  centers_out=_ptr(cen), labels_out=_ptr(lab))
        t = ctypes.c_uint64(0)
        with self._mu:
            rc = lib.kmeans2_server_submit(self._h, ctypes.byref(job), ctypes.byref(t))
            if rc != 0:
                raise KMeans2Error(rc, "kmeans2_server_submit")
            self._refs[t.value] = (X, cen, lab)
        return t.value

    def submit_lazy(self, n: int, d: int, k: int, subset_fraction: float, seed: int, tol: float,
                    max_iter: int, make, consume=None) -> int:
        """Queue a job whose points are produced only at admission:
        ``make(X)`` fills the (n, d) float32 CUDA tensor X in place on the
        current stream (the worker's); ``consume(centers, labels)``, if given,
        receives the fit's device outputs (valid during the call; copy them
        on the current stream)."""
        lib = load()
        dev = self.device

        def _run(stream, fn):
            with torch.cuda.device(dev):
                st = torch.cuda.ExternalStream(int(stream or 0), device=dev)
                with torch.cuda.stream(st):
                    fn()

        def _mat(user, xptr, stream):
            try:
                X = torch.as_tensor(_DeviceView(xptr, (n, d), "<f4"), device=dev)
                _run(stream, lambda: make(X))
                return 0
            except Exception:       # the library fails the job
                return 1

        def _con(user, cptr, lptr, stream):
            try:
                C = torch.as_tensor(_DeviceView(cptr, (k, d), "<f8"), device=dev)
                L = torch.as_tensor(_DeviceView(lptr, (n,), "<i4"), device=dev)
                _run(stream, lambda: consume(C, L))
            except Exception:
                pass

        cb_m = MATERIALIZE_FN(_mat)
        cb_c = CONSUME_FN(_con) if consume is not None else CONSUME_FN()
        job = Job(X=None, n=int(n), d=int(d), k=int(k), subset_fraction=float(subset_fraction),
                  seed=int(seed) & (2**64 - 1), tol=float(tol), max_iter=int(max_iter),
                  reserved=0, centers_out=None, labels_out=None)
        t = ctypes.c_uint64(0)
        with self._mu:
            rc = lib.kmeans2_server_submit_lazy(self._h, ctypes.byref(job), cb_m, cb_c, None,
                                                ctypes.byref(t))
            if rc != 0:
                raise KMeans2Error(rc, "kmeans2_server_submit_lazy")
            self._refs[t.value] = (cb_m, cb_c, None)
        return t.value

    def _collect(self, ticket, rc, r, tt):
        if rc == PENDING:
            return None
        with self._mu:
            X, cen, lab = self._refs.pop(ticket, (None, None, None))
        if not (_is_torch(cen) or isinstance(cen, np.ndarray)):
            cen = lab = None            # lazy job: the outputs went to its consume callback
        res = _fit_result(r, cen, lab) if rc == 0 else None
        return Served(ticket=ticket, status=rc, result=res, t_submit=tt.t_submit,
                      t_admit=tt.t_admit, t_done=tt.t_done)

    def poll(self, ticket: int) -> "Served | None":
        r, tt = Result(), TicketTimes()
        rc = load().kmeans2_server_poll(self._h, ticket, ctypes.byref(r), ctypes.byref(tt))
        if rc == -1 and ticket not in self._refs:
            raise KMeans2Error(rc, "kmeans2_server_poll")
        return self._collect(ticket, rc, r, tt)

    def wait(self, ticket: int, timeout: float = -1.0) -> "Served | None":
        r, tt = Result(), TicketTimes()
        rc = load().kmeans2_server_wait(self._h, ticket, float(timeout), ctypes.byref(r),
                                        ctypes.byref(tt))
        if rc == -1 and ticket not in self._refs:
            raise KMeans2Error(rc, "kmeans2_server_wait")
        return self._collect(ticket, rc, r, tt)

    def wait_any(self, timeout: float = -1.0) -> "Served | None":
        """The next finished job not yet returned by wait_any (collected), or
        None if none finishes within `timeout` seconds."""
        t = ctypes.c_uint64(0)
        rc = load().kmeans2_server_wait_any(self._h, float(timeout), ctypes.byref(t))
        if rc != 0:
            return None
        return self.poll(t.value)

    def stats(self) -> dict:
        st = ServerStats()
        load().kmeans2_server_stats_get(self._h, ctypes.byref(st))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_ if name != "pad_"}

    def now(self) -> float:
        return float(load().kmeans2_server_now(self._h))

    def close(self):
        if self._h:
            load().kmeans2_server_destroy(self._h)
            self._h = None
            self._refs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fit_batched(Xs, ks, subset_fraction, seeds, tol, max_iter, *, tol_fast: float = 0.0,
                stream=None, raise_on_error: bool = True, profile: "Profile | None" = None):
    """Batched two-stage fits (kmeans2_fit_batched) of independent problems.

    Xs: list of 2-D float32 CUDA tensors; ks, seeds: per-job lists; the other
    arguments are scalars or per-job lists.  Returns a list of FitResult (with
    device centers and labels) and the status code."""
    lib = load()
    cnt = len(Xs)
    if cnt == 0:
        return [], 0

    def per_job(v):
        return list(v) if isinstance(v, (list, tuple)) else [v] * cnt

    fs, tols, its = per_job(subset_fraction), per_job(tol), per_job(max_iter)
    jobs = (Job * cnt)()
    outs = []
    for j, X in enumerate(Xs):
        if not (_is_torch(X) and X.is_cuda):
            raise TypeError("fit_batched needs CUDA tensors")
        if X.device != Xs[0].device:
            raise ValueError("fit_batched needs every job's X on the same device")
        X = _as_points(X)
        n, d = X.shape
        cen = _empty(X, (ks[j], d), "f64")
        lab = _empty(X, (n,), "i32")
        outs.append((X, cen, lab))
        jobs[j] = Job(X=X.data_ptr(), n=n, d=d, k=int(ks[j]), subset_fraction=float(fs[j]),
                      seed=int(seeds[j]) & (2**64 - 1), tol=float(tols[j]), max_iter=int(its[j]),
                      reserved=0, centers_out=cen.data_ptr(), labels_out=lab.data_ptr())
    res = (Result * cnt)()
    opt = Options()
    lib.kmeans2_default_options(ctypes.byref(opt))
    opt.precision = PRECISION["fp32"]
    opt.tol_fast = tol_fast
    opt.stream = _stream_of(Xs[0], stream)
    opt.profile = ctypes.addressof(profile) if profile is not None else None
    with _device_of(Xs[0]):
        rc = lib.kmeans2_fit_batched(cnt, jobs, res, ctypes.byref(opt))
    if rc != 0 and raise_on_error:
        raise KMeans2Error(rc, "kmeans2_fit_batched")
    out = []
    for j in range(cnt):
        r = res[j]
        out.append(FitResult(centers=outs[j][1], labels=outs[j][2], J=r.J, iters_fast=r.iters_fast,
                             iters_slow=r.iters_slow, converged_fast=bool(r.converged_fast),
                             converged_slow=bool(r.converged_slow),
                             empty_clusters=r.empty_clusters, subset_size=r.subset_size,
                             rechecked_points=r.rechecked_points,
                             distance_evals=r.distance_evals, shift_fast=r.shift_fast,
                             shift_slow=r.shift_slow, seconds=r.seconds, precision_used="fp32"))
    return out, rc


def batched_tile_shape(d: int):
    """The batched autotuner's choice for the dimension class of d in this
    process (kmeans2_batched_tile_shape): (point slots per lane, lanes per
    point, tiles per work item), or None before a batched call has tuned it."""
    lib = load()
    p, g, t = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib.kmeans2_batched_tile_shape(int(d), ctypes.byref(p), ctypes.byref(g), ctypes.byref(t))
    return (p.value, g.value, t.value) if rc == 0 else None


def step(X, centers, *, precision: str = "auto", stream=None, centers_out=None, labels_out=None,
         profile: "Profile | None" = None):
    """One Lloyd iteration (kmeans_step): returns (centers', labels, J, shift, empty)."""
    lib = load()
    X = _as_points(X)
    n, d = X.shape
    C = _as_centers(centers, X, None, d)
    k = C.shape[0]
    cen = _out(centers_out, X, (k, d), "f64", "centers_out")
    lab = _out(labels_out, X, (n,), "i32", "labels_out")
    _check_devices(X, C, cen, lab)
    J = ctypes.c_double()
    sh = ctypes.c_double()
    em = ctypes.c_int32()
    opt = Options()
    lib.kmeans2_default_options(ctypes.byref(opt))
    opt.precision = PRECISION[precision]
    opt.stream = _stream_of(X, stream)
    opt.profile = ctypes.addressof(profile) if profile is not None else None
    with _device_of(X):
        rc = lib.kmeans_step(_ptr(X), n, d, k, _ptr(C), _ptr(cen), _ptr(lab), ctypes.addressof(J),
                             ctypes.addressof(sh), ctypes.addressof(em), ctypes.byref(opt))
    if rc != 0:
        raise KMeans2Error(rc, "kmeans_step")
    return cen, lab, J.value, sh.value, em.value


def step_noalloc(X, centers, *, stream=None, centers_out=None, labels_out=None):
    """kmeans_step_noalloc: one Lloyd iteration whose scratch is the library's
    fixed device array (no device allocation inside the call).  X and centers
    must be CUDA tensors; returns (centers', labels, J, shift, empty)."""
    lib = load()
    if not (_is_torch(X) and X.is_cuda):
        raise TypeError("step_noalloc needs X on a CUDA device")
    X = _as_points(X)
    n, d = X.shape
    C = _as_centers(centers, X, None, d)
    k = C.shape[0]
    cen = _out(centers_out, X, (k, d), "f64", "centers_out")
    lab = _out(labels_out, X, (n,), "i32", "labels_out")
    _check_devices(X, C, cen, lab)
    J = ctypes.c_double()
    sh = ctypes.c_double()
    em = ctypes.c_int32()
    with _device_of(X):
        rc = lib.kmeans_step_noalloc(_ptr(X), n, d, k, _ptr(C), _ptr(cen), _ptr(lab),
                                     ctypes.addressof(J), ctypes.addressof(sh),
                                     ctypes.addressof(em), _stream_of(X, stream))
    if rc != 0:
        raise KMeans2Error(rc, "kmeans_step_noalloc")
    return cen, lab, J.value, sh.value, em.value


def subset_size(n: int, k: int, subset_fraction: float) -> int:
    return int(load().kmeans2_subset_size(n, k, subset_fraction))


def sample(n: int, k: int, subset_fraction: float, seed: int, device="cuda", stream=None):
    """GPU draw of S_s and of the initial-center positions (kmeans2_sample)."""
    lib = load()
    m = subset_size(n, k, subset_fraction)
    if m < 0:
        raise ValueError("invalid sampling arguments")
    dev = torch.device(device)
    sub = torch.empty(m, dtype=torch.int64, device=dev)
    pos = torch.empty(k, dtype=torch.int64, device=dev)
    s = _stream_of(sub, stream)
    with _device_of(sub):
        rc = lib.kmeans2_sample(n, k, subset_fraction, seed & (2**64 - 1), sub.data_ptr(),
                                pos.data_ptr(), s)
    if rc != 0:
        raise KMeans2Error(rc, "kmeans2_sample")
    return sub, pos


def strerror(status: int) -> str:
    return load().kmeans2_strerror(status).decode()


def version() -> tuple[int, int]:
    v = int(load().kmeans2_version())
    return v >> 16, v & 0xFFFF
