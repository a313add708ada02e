"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds no arithmetic of the method itself (no covariance function,
no ordering, no factorization, no solve).  It only draws the random inputs
that the paper's synthetic experiments describe: irregular 2D locations in
]0,1[ and measurement vectors (Section "Synthetic Datasets"), plus the
parameter draws of the batched workload.  Every generator takes an explicit
seed and uses numpy's PCG64 bit generator, so both sides of a comparison see
the same arrays.

Measurement vectors for large n are drawn by a spectral (random Fourier
feature) simulation of a Matern field: the field is a sum of cosines whose
frequencies follow the Matern spectral density, a multivariate Student-t with
2*nu degrees of freedom and scale 1/(beta*sqrt(2*nu)).  As the number of
features grows the sample converges to a Gaussian field with exactly the
Matern covariance; at any finite count it is a smooth stationary field of the
right range and variance, which is all the likelihood evaluation needs (the
likelihood is defined for every Z).  Small cases that want Z = L w exactly
build it in the tests from the oracle's own factor and the white noise drawn
here.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "jittered_grid",
    "uniform_points",
    "line_points",
    "white_noise",
    "matern_field_rff",
    "batch_specs",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def jittered_grid(m: int, seed: int, jitter: float = 0.4):
    """m*m locations: cell centres ((i+1/2)/m, (j+1/2)/m) moved by U(-jitter/m, jitter/m).

    Returned in grid (row-major) order as float64 arrays x, y of length m*m.
    With jitter < 1/2 every point stays strictly inside ]0,1[ and no two
    points coincide.
    """
    g = _rng(seed)
    i, j = np.meshgrid(np.arange(m, dtype=np.float64), np.arange(m, dtype=np.float64), indexing="ij")
    jx = g.uniform(-jitter, jitter, size=(m, m))
    jy = g.uniform(-jitter, jitter, size=(m, m))
    x = (i + 0.5 + jx) / m
    y = (j + 0.5 + jy) / m
    return x.ravel().copy(), y.ravel().copy()


def uniform_points(n: int, seed: int):
    """n locations drawn uniformly on ]0,1[^2 (float64 x, y)."""
    g = _rng(seed)
    x = g.uniform(0.0, 1.0, size=n)
    y = g.uniform(0.0, 1.0, size=n)
    return x, y


def line_points(n: int, seed: int, min_gap: float = 0.0):
    """n sorted locations on the segment y = 0, x in ]0,1[ (float64 x, y).

    Gaps are i.i.d. exponential, rescaled so the points span ]0,1[; `min_gap`
    is added to every gap before rescaling to bound the spacing from below.
    """
    g = _rng(seed)
    gaps = g.exponential(1.0, size=n + 1) + min_gap
    x = np.cumsum(gaps)[:n] / gaps.sum()
    return x.astype(np.float64), np.zeros(n, dtype=np.float64)


def white_noise(n: int, seed: int):
    """n i.i.d. standard normal draws (float64)."""
    return _rng(seed).standard_normal(n)


def matern_field_rff(x, y, sigma2: float, beta: float, nu: float, seed: int,
                     n_features: int = 1024, nugget: float = 0.0, chunk: int = 1 << 15):
    """Approximate Matern-field sample at (x, y) by random Fourier features.

    Z(s) = sqrt(2*sigma2/M) * sum_m cos(w_m . s + phi_m) (+ sqrt(nugget)*e), with
    w_m = g_m / (beta*sqrt(2*nu)) / sqrt(chi2_{2nu}/(2nu)), g_m ~ N(0, I_2),
    phi_m ~ U(0, 2*pi).  Values are a deterministic function of each point's
    coordinates and the seed, so any reordering of the points carries Z along.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    g = _rng(seed)
    dof = 2.0 * nu
    gauss = g.standard_normal((n_features, 2))
    chi2 = g.chisquare(dof, size=n_features)
    w = gauss / (beta * np.sqrt(dof)) / np.sqrt(chi2 / dof)[:, None]
    phi = g.uniform(0.0, 2.0 * np.pi, size=n_features)
    out = np.empty(x.shape[0], dtype=np.float64)
    amp = np.sqrt(2.0 * sigma2 / n_features)
    for s in range(0, x.shape[0], chunk):
        arg = np.outer(x[s:s + chunk], w[:, 0]) + np.outer(y[s:s + chunk], w[:, 1]) + phi[None, :]
        out[s:s + chunk] = amp * np.cos(arg).sum(axis=1)
    if nugget > 0.0:
        out += np.sqrt(nugget) * g.standard_normal(x.shape[0])
    return out


def batch_specs(count: int, seed: int, n_lo: int = 500, n_hi: int = 8000):
    """Per-problem draws of the batched workload.

    Returns a list of dicts with n ~ U[n_lo, n_hi] (integer), sigma2 ~ U[0.5, 2],
    beta ~ U[0.02, 0.3], nu drawn from {0.5, 1.0, 1.5}, and a per-problem seed.
    """
    g = _rng(seed)
    out = []
    for i in range(count):
        out.append(dict(
            n=int(g.integers(n_lo, n_hi + 1)),
            sigma2=float(g.uniform(0.5, 2.0)),
            beta=float(g.uniform(0.02, 0.3)),
            nu=float(g.choice([0.5, 1.0, 1.5])),
            seed=int(seed * 1000 + i),
        ))
    return out
