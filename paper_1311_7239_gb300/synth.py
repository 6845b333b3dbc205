"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module draws random numbers and shapes them into media fields; it holds none of the
lattice Boltzmann arithmetic (no equilibria, no collision, no streaming), so both the CUDA path
and the FP64 oracle can take their inputs from it without sharing any of the method.

Recipes (the workloads the paper's validation flows suggest, Sec. 3):
  * ``gaussian_random_field``: white noise filtered in Fourier space by a Gaussian kernel of the
    given correlation length, normalised to zero mean and unit standard deviation.
  * ``heterogeneous_medium``: log K = log(Da_mean * H^2) + sigma * GRF, eps = clip(eps0 + s * GRF', lo, hi)
    with an independent seed for eps.
  * ``ensemble_domains``: side lengths, flow kind and Reynolds number of a batch of domains.
"""
from __future__ import annotations

import numpy as np


def gaussian_random_field(ny: int, nx: int, corr_len: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance stationary field with a Gaussian covariance of length corr_len (cells)."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.rfftfreq(nx)[None, :]
    kernel = np.exp(-0.5 * (2.0 * np.pi * corr_len) ** 2 * (kx * kx + ky * ky))
    field = np.fft.irfft2(np.fft.rfft2(noise) * kernel, s=(ny, nx))
    field -= field.mean()
    sd = field.std()
    return field / sd if sd > 0 else field


def heterogeneous_medium(
    ny: int,
    nx: int,
    H: float,
    seed: int,
    da_mean: float = 1e-3,
    sigma_logk: float = 1.0,
    corr_len: float = 32.0,
    eps_mean: float = 0.3,
    eps_sd: float = 0.1,
    eps_lo: float = 0.1,
    eps_hi: float = 0.9,
):
    """(eps, K) float64 fields of shape (ny, nx): log-normal permeability and clipped porosity."""
    logk = np.log(da_mean * H * H) + sigma_logk * gaussian_random_field(ny, nx, corr_len, seed)
    eps = np.clip(eps_mean + eps_sd * gaussian_random_field(ny, nx, corr_len, seed + 7919), eps_lo, eps_hi)
    return eps, np.exp(logk)


def ensemble_domains(n: int, seed: int, lo: int = 64, hi: int = 1024):
    """List of dicts (nx, ny, kind, Re, seed) for a batch of independent domains."""
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n):
        out.append(
            {
                "nx": int(rng.integers(lo, hi + 1)),
                "ny": int(rng.integers(lo, hi + 1)),
                "kind": "cavity" if rng.random() < 0.5 else "channel",
                "Re": float(rng.uniform(10.0, 400.0)),
                "seed": int(seed * 100003 + d),
            }
        )
    return out


def random_populations(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Standard-normal array times scale (perturbations for brute-force parity cases)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)
