"""Offspring statistics of Section 5.1 (Eqs. 14-21).  Test infrastructure.

For K ancestor vectors of one weight vector w (length N):
  offspring  o_k^(i) = #{ particles whose ancestor is i in run k }
  SE(o_k)    = sum_i (o_k^(i) - N w_i / sum_j w_j)^2             (Eq. 14)
  MSE        = (1/K) sum_k SE(o_k)                               (Eq. 15)
  o_hat^(i)  = (1/K) sum_k o_k^(i)                               (Eq. 19)
  Var        = sum_i (1/(K-1)) sum_k (o_k^(i) - o_hat^(i))^2     (Eqs. 17, 20)
  |Bias|^2   = sum_i (o_hat^(i) - N w_i / sum_j w_j)^2           (Eq. 18)
  bias contribution = |Bias|^2 / MSE                             (Eq. 21)
The paper reports MSE/N.  Eq. 18 prints a hat over the w in the numerator;
it is read as the plain weight w (there is no estimated weight anywhere
else in the paper), and Var uses the 1/(K-1) of Eq. 20, so
MSE = Var + |Bias|^2 (Eq. 16) holds only up to the factor (K-1)/K on Var.
"""
from __future__ import annotations

import numpy as np


def offspring(anc: np.ndarray, n: int) -> np.ndarray:
    return np.bincount(np.asarray(anc, dtype=np.int64), minlength=n)[:n]


def expected_offspring(w) -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    return w.shape[0] * w / w.sum()


def offspring_stats(w, ancestor_runs) -> dict:
    """Statistics over K runs; ancestor_runs is a [K, N] array-like."""
    w = np.asarray(w, dtype=np.float64)
    n = w.shape[0]
    runs = [offspring(a, n).astype(np.float64) for a in ancestor_runs]
    K = len(runs)
    o = np.stack(runs)                      # [K, N]
    e = expected_offspring(w)               # [N]
    se = ((o - e[None, :]) ** 2).sum(axis=1)
    mse = float(se.mean())
    o_hat = o.mean(axis=0)
    var = float(((o - o_hat[None, :]) ** 2).sum(axis=0).sum() / (K - 1)) if K > 1 else float("nan")
    bias2 = float(((o_hat - e) ** 2).sum())
    return {
        "K": K,
        "N": n,
        "mse": mse,
        "mse_per_n": mse / n,
        "var": var,
        "bias2": bias2,
        "bias_contribution": bias2 / mse if mse > 0 else float("nan"),
        "max_offspring": int(o.max()),
    }
