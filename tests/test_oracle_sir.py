"""Pins for the oracle's SIR filter stages (Algorithm 6; Eqs. 22-23) against
the model's closed form evaluated in double, and for the mean estimator."""
import math

import numpy as np

import oracle
import synthetic


def test_predict_matches_model_within_rounding():
    rng = np.random.default_rng(1)
    x = rng.normal(0, 8, 5000).astype(np.float32)
    x[:4] = [0.0, 1.0, -1.0, 3.0]
    v = rng.normal(0, math.sqrt(10), 5000).astype(np.float32)
    drift = np.float32(8 * math.cos(1.2 * 7))
    z = np.float32(4.5)
    xp, w = oracle.sir_predict_update(x, v, float(drift), float(z))
    xd = x.astype(np.float64)
    ref = xd / 2 + 25 * xd / (1 + xd * xd) + float(drift) + v.astype(np.float64)
    scale = np.abs(xd) / 2 + np.abs(25 * xd / (1 + xd * xd)) + abs(float(drift)) + np.abs(v)
    assert (np.abs(xp - ref) <= 8 * 2.0 ** -24 * scale + 1e-30).all()
    assert xp[0] == np.float32(drift + v[0])        # x = 0: only drift and noise
    # weight: exp(-(z - x'^2/20)^2 / 2) of the predicted particle, as computed
    d = float(z) - xp.astype(np.float64) ** 2 / 20
    wref = np.exp(-0.5 * d * d)
    # error of d = z - x'^2/20 in binary32 (two roundings of x'^2/20, one of
    # the difference) times |d|, the rounding of a = d^2/2, and exp's rounding
    a = 0.5 * d * d
    tol = (4 + 4 * np.abs(d) * (xp.astype(np.float64) ** 2 / 20) + 2 * a) * 2.0 ** -23 * wref + 2.0 ** -149
    assert (np.abs(w - wref) <= tol).all()
    assert (w >= 0).all() and (w <= 1).all()


def test_weight_is_one_at_the_measurement():
    x = np.array([2.0, -3.0], np.float32)
    v = np.zeros(2, np.float32)
    xp, _ = oracle.sir_predict_update(x, v, 0.0, 0.0)
    z = np.float32(np.float32(xp[0] * xp[0]) / np.float32(20.0))
    _, w = oracle.sir_predict_update(x, v, 0.0, float(z))
    assert w[0] == 1.0


def test_mean_against_exact_sum():
    x = synthetic.gaussian_state(100_001, 1, 3)[0] * 7 + 2
    assert abs(oracle.mean(x) - math.fsum(x.astype(np.float64).tolist()) / x.size) < 1e-12


def test_truth_trajectory_follows_the_model():
    x, z = synthetic.sir_truth(50, 4)
    resid = x[1:] - (x[:-1] / 2 + 25 * x[:-1] / (1 + x[:-1] ** 2) + 8 * np.cos(1.2 * np.arange(1, 51)))
    assert abs(resid.std() - math.sqrt(10)) < 1.5          # N(0, 10) process noise
    assert abs((z[1:] - x[1:] ** 2 / 20).std() - 1.0) < 0.5
