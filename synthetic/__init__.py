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
