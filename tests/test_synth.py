"""The seeded input generators (CPU): shapes, determinism, distribution facts."""
import numpy as np
import torch

from paper_1108_1351_gb300 import synth


def test_iso_mixture_deterministic_and_shaped():
    a = synth.iso_gaussian_mixture(1000, 2, 4, seed=0)
    b = synth.iso_gaussian_mixture(1000, 2, 4, seed=0)
    c = synth.iso_gaussian_mixture(1000, 2, 4, seed=1)
    assert a.shape == (1000, 2) and a.dtype == torch.float32 and a.is_contiguous()
    assert torch.equal(a, b) and not torch.equal(a, c)
    X, comp, means = synth.iso_gaussian_mixture(20000, 2, 4, seed=0, return_truth=True)
    assert np.all((means >= -10) & (means <= 10))
    for j in range(4):
        pts = X[comp == j].double().numpy()
        assert abs(pts.std(0).mean() - 1.0) < 0.05
        assert np.allclose(pts.mean(0), means[j], atol=0.1)


def test_aniso_noise_fraction_and_box():
    X, comp, means = synth.aniso_gaussian_noise(40000, 8, 32, seed=0, chunk=10000,
                                                return_truth=True)
    assert X.shape == (40000, 8) and torch.isfinite(X).all()
    frac = float((comp < 0).float().mean())
    assert 0.015 < frac < 0.025
    mix = X[comp >= 0]
    noise = X[comp < 0]
    assert (noise >= mix.min(0).values).all() and (noise <= mix.max(0).values).all()


def test_vmf_unit_norm_and_concentration():
    X, comp, M = synth.vmf_mixture(4000, 16, 8, seed=3, chunk=1500, return_truth=True)
    assert torch.allclose(X.norm(dim=1), torch.ones(4000), atol=1e-5)
    cos = (X.double() * torch.as_tensor(M)[comp]).sum(1)
    assert float(cos.mean()) > 0.9           # kappa >= 50 in 16-D is tightly concentrated


def test_instance_specs_and_arrivals():
    specs = synth.instance_specs(256, seed=0)
    assert len(specs) == 256
    assert all(1000 <= s.n <= 1_000_000 and s.d in (2, 8, 32, 64) and 2 <= s.k <= 256
               for s in specs)
    assert len({s.seed for s in specs}) == 256
    jobs = synth.arrival_trace(rate=200, duration=5, seed=0)
    assert 800 < len(jobs) < 1200
    assert all(10_000 <= j.n <= 20_000_000 and j.d in (4, 16, 64, 128) and 4 <= j.k <= 1024
               for j in jobs)
    assert all(a.t_arrival < b.t_arrival for a, b in zip(jobs, jobs[1:]))
