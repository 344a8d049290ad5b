"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no k-means arithmetic: it only draws points.  Both the CUDA
library's callers (tests, benchmark) and the FP64 oracle receive the SAME
tensors from here, so neither side regenerates the other's inputs.

The paper's datasets (a 150-point 3-D set, UCI "Synthetic Control Chart",
its unnamed "Synthetic" 100,000 x 10 and 1M-10M x 12 sets) are not available;
these generators stand in for them with the shapes the paper uses
(Section 4: randomly placed clusters of uniform size; Section 6: 100,000 x 10;
Section 6.1: up to 10M points in 12-D; Abstract: 500M+ points).

Mixture parameters (means, rotations, weights, concentrations) are drawn on
the CPU in float64 from ``numpy.random.default_rng(seed)``; per-point draws use
a ``torch.Generator`` on the target device seeded with ``seed``.  The same
seed therefore gives the same parameters everywhere and the same points on the
same device type.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

__all__ = [
    "iso_gaussian_mixture", "aniso_gaussian_noise", "vmf_mixture",
    "InstanceSpec", "instance_specs", "instance_data", "JobSpec", "arrival_trace",
]


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed) & 0x7FFF_FFFF_FFFF_FFFF)
    return g


def iso_gaussian_mixture(n: int, d: int, k: int, seed: int, *, lo: float = -10.0,
                         hi: float = 10.0, sigma: float = 1.0, device="cpu",
                         return_truth: bool = False):
    """k isotropic Gaussians N(mu_j, sigma^2 I), mu_j ~ U[lo, hi]^d, equal weights.

    Returns X (n, d) float32 on ``device``; with ``return_truth`` also the
    component of each point (int64) and the means (float64 numpy)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(lo, hi, size=(k, d))
    g = _gen(device, seed)
    comp = torch.randint(0, k, (n,), generator=g, device=device)
    z = torch.randn(n, d, generator=g, device=device, dtype=torch.float32)
    mu = torch.as_tensor(means, dtype=torch.float32, device=device)
    X = (mu[comp] + sigma * z).contiguous()
    if return_truth:
        return X, comp, means
    return X


def _haar_rotation(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix, signs fixed
    so that R has a positive diagonal (Mezzadri 2007)."""
    A = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))[None, :]


def aniso_gaussian_noise(n: int, d: int, k: int, seed: int, *, eig_lo: float = 0.1,
                         eig_hi: float = 2.0, alpha: float = 1.0, noise: float = 0.02,
                         lo: float = -10.0, hi: float = 10.0, device="cpu",
                         chunk: int = 1 << 22, out: torch.Tensor | None = None,
                         return_truth: bool = False, sample_seed: int | None = None):
    """Anisotropic Gaussian mixture with uniform background noise.

    Component j: mean ~ U[lo, hi]^d, covariance R_j diag(lambda) R_j^T with
    lambda log-uniform in [eig_lo, eig_hi] and R_j Haar-random; weights
    ~ Dirichlet(alpha).  Each point is noise with probability ``noise``; noise
    points are uniform over the per-dimension bounding box of the mixture
    points.  Generated in chunks so that n = 5e8 fits beside its output.
    The mixture comes from ``seed``, the points from ``sample_seed`` (default
    ``seed``): blocks with the same seed and different sample seeds are
    independent samples of one mixture (the row blocks of a data set split
    over several GPUs)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(lo, hi, size=(k, d))
    L = np.empty((k, d, d))
    for j in range(k):
        lam = np.exp(rng.uniform(math.log(eig_lo), math.log(eig_hi), size=d))
        L[j] = _haar_rotation(rng, d) * np.sqrt(lam)[None, :]
    w = rng.gamma(alpha, 1.0, size=k)
    w = w / w.sum()
    cum = torch.as_tensor(np.cumsum(w)[:-1], dtype=torch.float32, device=device)
    mu = torch.as_tensor(means, dtype=torch.float32, device=device)
    Lt = torch.as_tensor(L, dtype=torch.float32, device=device)

    g = _gen(device, seed if sample_seed is None else sample_seed)
    X = out if out is not None else torch.empty(n, d, dtype=torch.float32, device=device)
    is_noise = torch.rand(n, generator=g, device=device) < noise
    comp_all = torch.empty(n, dtype=torch.int32, device=device) if return_truth else None
    bmin = torch.full((d,), float("inf"), device=device)
    bmax = torch.full((d,), float("-inf"), device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        u = torch.rand(b - a, generator=g, device=device)
        comp = torch.searchsorted(cum, u)
        z = torch.randn(b - a, d, 1, generator=g, device=device)
        x = mu[comp] + torch.bmm(Lt[comp], z).squeeze(2)
        X[a:b] = x
        keep = ~is_noise[a:b]
        if bool(keep.any()):
            xs = x[keep]
            bmin = torch.minimum(bmin, xs.min(0).values)
            bmax = torch.maximum(bmax, xs.max(0).values)
        if comp_all is not None:
            comp_all[a:b] = comp.to(torch.int32)
        del x, z, comp, u
    idx = is_noise.nonzero().squeeze(1)
    for a in range(0, idx.numel(), chunk):
        sel = idx[a:a + chunk]
        r = torch.rand(sel.numel(), d, generator=g, device=device)
        X[sel] = bmin + (bmax - bmin) * r
        if comp_all is not None:
            comp_all[sel] = -1
    if return_truth:
        return X, comp_all, means
    return X


def vmf_mixture(n: int, d: int, k: int, seed: int, *, kappa_lo: float = 50.0,
                kappa_hi: float = 500.0, device="cpu", chunk: int = 1 << 20,
                out: torch.Tensor | None = None, return_truth: bool = False):
    """Unit-norm points from k equal-weight von Mises-Fisher components.

    Mean directions are uniform on the sphere, concentrations uniform in
    [kappa_lo, kappa_hi].  The cosine w to the mean direction is drawn with
    Wood's rejection sampler (Wood 1994), whose Beta((d-1)/2, (d-1)/2) proposal
    is taken as (1 + t)/2, t the first coordinate of a uniform point on the
    sphere; the remaining coordinates of that point give the tangent
    direction.  A Householder reflection maps e_1 onto the mean direction."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((k, d))
    M /= np.linalg.norm(M, axis=1, keepdims=True)
    kap = rng.uniform(kappa_lo, kappa_hi, size=k)
    Mt = torch.as_tensor(M, dtype=torch.float32, device=device)
    U = Mt.clone()
    U[:, 0] -= 1.0                                 # Householder vector e_1 - mu, sign-flipped
    Un = (U * U).sum(1)
    kt = torch.as_tensor(kap, dtype=torch.float64, device=device)
    dm1 = float(d - 1)
    bt = (-2.0 * kt + torch.sqrt(4.0 * kt * kt + dm1 * dm1)) / dm1
    x0t = (1.0 - bt) / (1.0 + bt)
    ct = kt * x0t + dm1 * torch.log(1.0 - x0t * x0t)

    g = _gen(device, seed)
    X = out if out is not None else torch.empty(n, d, dtype=torch.float32, device=device)
    comp_all = torch.empty(n, dtype=torch.int64, device=device) if return_truth else None
    for a in range(0, n, chunk):
        m = min(n, a + chunk) - a
        comp = torch.randint(0, k, (m,), generator=g, device=device)
        kap_c, b_c, x0_c, c_c = kt[comp], bt[comp], x0t[comp], ct[comp]
        w = torch.empty(m, dtype=torch.float64, device=device)
        tang = torch.empty(m, d - 1, dtype=torch.float32, device=device)
        todo = torch.arange(m, device=device)
        while todo.numel() > 0:
            gg = torch.randn(todo.numel(), d, generator=g, device=device)
            t = (gg[:, 0] / gg.norm(dim=1)).double()
            z = 0.5 * (1.0 + t)
            bb, xx, cc, kk = b_c[todo], x0_c[todo], c_c[todo], kap_c[todo]
            ww = (1.0 - (1.0 + bb) * z) / (1.0 - (1.0 - bb) * z)
            u = torch.rand(todo.numel(), generator=g, device=device, dtype=torch.float64)
            ok = kk * ww + dm1 * torch.log(1.0 - xx * ww) - cc >= torch.log(u)
            acc = todo[ok]
            w[acc] = ww[ok]
            tv = gg[ok, 1:]
            tang[acc] = tv / tv.norm(dim=1, keepdim=True)
            todo = todo[~ok]
        y = torch.empty(m, d, dtype=torch.float32, device=device)
        y[:, 0] = w.float()
        y[:, 1:] = tang * torch.sqrt(torch.clamp(1.0 - w * w, min=0.0)).float()[:, None]
        Uc, Unc = U[comp], Un[comp]
        proj = (Uc * y).sum(1)
        scale = torch.where(Unc > 0, 2.0 * proj / torch.clamp(Unc, min=1e-30),
                            torch.zeros_like(proj))
        x = y - scale[:, None] * Uc
        X[a:a + m] = x / x.norm(dim=1, keepdim=True)
        if comp_all is not None:
            comp_all[a:a + m] = comp
    if return_truth:
        return X, comp_all, M
    return X


@dataclass(frozen=True)
class InstanceSpec:
    """One independent k-means instance of the batched workload."""
    n: int
    d: int
    k: int
    seed: int


def instance_specs(count: int = 4096, seed: int = 0, *, n_lo: float = 1e3, n_hi: float = 1e6,
                   dims=(2, 8, 32, 64), k_lo: int = 2, k_hi: int = 256):
    """Batched workload: n log-uniform in [n_lo, n_hi], d uniform over ``dims``,
    k uniform in [k_lo, k_hi]; instance i carries seed i (+ ``seed``)."""
    rng = np.random.default_rng(seed + 0x5EED)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    ds = rng.choice(np.asarray(dims), size=count)
    ks = rng.integers(k_lo, k_hi + 1, size=count)
    out = []
    for i in range(count):
        n = int(max(ns[i], 1))
        k = int(min(ks[i], n))
        out.append(InstanceSpec(n=n, d=int(ds[i]), k=k, seed=seed + i))
    return out


def instance_data(spec: InstanceSpec, device="cpu", *, lo: float = -20.0, hi: float = 20.0):
    """Gaussian mixture with spec.k components, sigma = 1, means U[lo, hi]^d."""
    return iso_gaussian_mixture(spec.n, spec.d, spec.k, spec.seed, lo=lo, hi=hi, device=device)


@dataclass(frozen=True)
class JobSpec:
    """One clustering request of the serving workload."""
    t_arrival: float
    n: int
    d: int
    k: int
    seed: int


def arrival_trace(rate: float = 200.0, duration: float = 60.0, seed: int = 0, *,
                  n_lo: float = 1e4, n_hi: float = 2e7, dims=(4, 16, 64, 128),
                  k_lo: float = 4, k_hi: float = 1024):
    """Poisson arrivals at ``rate`` jobs/s for ``duration`` s; n and k
    log-uniform, d uniform over ``dims``; job j's data seed is seed + j."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
        d = int(rng.choice(np.asarray(dims)))
        k = int(round(math.exp(rng.uniform(math.log(k_lo), math.log(k_hi)))))
        jobs.append(JobSpec(t_arrival=t, n=n, d=d, k=min(k, n), seed=seed + len(jobs)))
    return jobs
