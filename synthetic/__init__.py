"""Seeded synthetic inputs shaped like the paper's workloads.

This module only makes inputs; it holds none of the resampling arithmetic
(no chain, no bound, no gather) and imports neither the CUDA package nor the
oracle.  Both sides of every parity test take their inputs from here.

Recipes (Section 5, "Numerical Experimental Settings"):
  * gaussian_weights: x_i ~ N(0,1), w_i = exp(-(x_i - y)^2 / 2) (Eq. 12 up to
    its constant factor), computed in double and rounded to float32.  Larger
    y concentrates the weight on fewer particles.
  * gamma_weights: w_i ~ Gamma(alpha, rate 1) (Eq. 13), float32.
  * gaussian_state: an SoA [dim, N] float32 array with N(0,1) entries (three
    positions and three velocities for dim = 6).
  * filter_sizes / request_stream: batched and served workloads (many
    independent filters of log-uniform size).
All draws come from numpy's PCG64 generator seeded with the given seed and a
per-recipe salt, so each recipe's stream is independent of the others.
"""
from __future__ import annotations

import numpy as np

_SALT_GAUSS_W = 0x5747
_SALT_GAMMA_W = 0x4741
_SALT_STATE = 0x5354
_SALT_FILTERS = 0x4649
_SALT_REQUESTS = 0x5251
_SALT_TRUTH = 0x5452
_SALT_NOISE = 0x4E4F


def _rng(seed: int, salt: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(salt)]))


def gaussian_weights(n: int, y: float, seed: int) -> np.ndarray:
    x = _rng(seed, _SALT_GAUSS_W).standard_normal(int(n))
    return np.exp(-0.5 * (x - float(y)) ** 2).astype(np.float32)


def gamma_weights(n: int, alpha: float, seed: int) -> np.ndarray:
    return _rng(seed, _SALT_GAMMA_W).gamma(float(alpha), 1.0, int(n)).astype(np.float32)


def gaussian_state(n: int, dim: int, seed: int) -> np.ndarray:
    return _rng(seed, _SALT_STATE).standard_normal((int(dim), int(n))).astype(np.float32)


def filter_sizes(count: int, lo_log2: float, hi_log2: float, seed: int):
    """count sizes N = floor(2^U[lo, hi]) and per-filter y ~ U[0, 4]."""
    g = _rng(seed, _SALT_FILTERS)
    sizes = np.floor(2.0 ** g.uniform(lo_log2, hi_log2, int(count))).astype(np.int64)
    ys = g.uniform(0.0, 4.0, int(count))
    return sizes, ys


def request_stream(count: int, rate_per_s: float, lo_log2: float, hi_log2: float,
                   seed: int):
    """Poisson arrivals: (arrival times in s, sizes N, per-request y = 2)."""
    g = _rng(seed, _SALT_REQUESTS)
    gaps = g.exponential(1.0 / float(rate_per_s), int(count))
    t = np.cumsum(gaps)
    sizes = np.floor(2.0 ** g.uniform(lo_log2, hi_log2, int(count))).astype(np.int64)
    return t, sizes


def uniform_weights(n: int, seed: int) -> np.ndarray:
    """w_i ~ U[0, 1) float32 (cheap inputs for the largest sizes)."""
    return _rng(seed, 0x554E).random(int(n), dtype=np.float32)


def sir_truth(T: int, seed: int, x0: float = 0.1):
    """A ground-truth trajectory of the model of Eqs. 22-23 (double):
    x_t = x_{t-1}/2 + 25 x_{t-1}/(1 + x_{t-1}^2) + 8 cos(1.2 t) + v, v ~ N(0, 10);
    z_t = x_t^2 / 20 + n, n ~ N(0, 1).  Returns (x[0..T], z[0..T]); z[0] unused."""
    g = _rng(seed, _SALT_TRUTH)
    x = np.empty(T + 1)
    z = np.empty(T + 1)
    x[0] = x0
    z[0] = np.nan
    for t in range(1, T + 1):
        xp = x[t - 1]
        x[t] = xp / 2 + 25 * xp / (1 + xp * xp) + 8 * np.cos(1.2 * t) + np.sqrt(10.0) * g.standard_normal()
        z[t] = x[t] * x[t] / 20 + g.standard_normal()
    return x, z


def sir_initial_particles(n: int, seed: int) -> np.ndarray:
    """Initial particles x_0 ~ N(0, 2), float32."""
    return (np.sqrt(2.0) * _rng(seed, _SALT_STATE + 1).standard_normal(int(n))).astype(np.float32)


def sir_process_noise(n: int, T: int, seed: int, device=None):
    """Process noise v ~ N(0, 10) for T steps of n particles, float32 [T, n].
    device=None: numpy on the host; a CUDA device: torch's generator there
    (for large runs)."""
    if device is None:
        return (np.sqrt(10.0) * _rng(seed, _SALT_NOISE).standard_normal((int(T), int(n)))).astype(np.float32)
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1_000_003 + _SALT_NOISE)
    return torch.randn((int(T), int(n)), generator=gen, device=device, dtype=torch.float32) * float(np.sqrt(10.0))
