"""Pins for the oracle's gather (x_bar^(i) = x^(k)) and likelihood weight."""
import math

import numpy as np

import oracle
import synthetic


def test_gather_soa_matches_fancy_indexing():
    x = synthetic.gaussian_state(777, 6, 1)
    rng = np.random.default_rng(2)
    anc = rng.integers(0, 777, 777).astype(np.int32)
    assert np.array_equal(oracle.gather_soa(x, anc), x[:, anc])
    ident = np.arange(777, dtype=np.int32)
    assert np.array_equal(oracle.gather_soa(x, ident), x)


def test_gather_aos4_matches_fancy_indexing():
    x = synthetic.gaussian_state(4 * 513, 1, 3).reshape(513, 4)
    anc = np.random.default_rng(4).integers(0, 513, 513).astype(np.int32)
    assert np.array_equal(oracle.gather_aos4(x, anc), x[anc])


def test_likelihood_closed_form_points_and_symmetry():
    # w(x) = exp(-(x - y)^2 / 2): at x - y = 0 the weight is exactly 1; at
    # |x - y| = 1, 2 and 4 it is e^(-1/2), e^(-2) and e^(-8) (powers of the
    # constant e, not of the function under test); it depends on x - y only
    # through its square (symmetry about y); a dropped 1/2, a sign error or
    # an (x + y) would break one of these.
    y = 2.0
    d = np.array([0.0, 1.0, -1.0, 2.0, -2.0, 4.0, -4.0], dtype=np.float32)
    w = oracle.likelihood(np.float32(y) + d, y).astype(np.float64)
    e = math.e
    want = [1.0, e ** -0.5, e ** -0.5, e ** -2, e ** -2, e ** -8, e ** -8]
    assert w[0] == 1.0
    assert np.allclose(w, want, rtol=2.0 ** -23, atol=0.0)
    # |x - y| = sqrt(2): e^-1 (x - y not exactly representable: first order)
    dx = np.float32(math.sqrt(2.0))
    w2 = oracle.likelihood(np.array([y + dx, y - dx], np.float32), y).astype(np.float64)
    d_exact = np.array([np.float64(np.float32(y + dx)) - y, np.float64(np.float32(y - dx)) - y])
    assert np.all(np.abs(w2 - 1.0 / e) <= 2.0 * np.abs(np.abs(d_exact) - math.sqrt(2.0)) / e
                  + 2.0 ** -24)
    x = synthetic.gaussian_state(10_000, 1, 5)[0]
    mirrored = (np.float32(2.0 * y) - x).astype(np.float32)
    exact = (np.float64(2.0 * y) - x.astype(np.float64)) == mirrored.astype(np.float64)
    assert exact.sum() > 1000
    assert np.array_equal(oracle.likelihood(x, y)[exact], oracle.likelihood(mirrored, y)[exact])
    ww = oracle.likelihood(x, y)
    assert (ww >= 0).all() and (ww <= 1).all()


def test_likelihood_half_maximum_and_integral():
    # Textbook facts of the unit-variance Gaussian: the full width at half
    # maximum is 2 sqrt(2 ln 2) = 2.3548200450309493, and the integral of
    # exp(-t^2 / 2) over the line is sqrt(2 pi) = 2.5066282746310002.
    y = -1.5
    half = np.float32(2.3548200450309493 / 2)
    w = oracle.likelihood(np.array([y + half, y - half], np.float32), y)
    assert np.allclose(w, 0.5, rtol=1e-6)
    h = 1.0 / 256
    t = (y + h * np.arange(-12 * 256, 12 * 256 + 1)).astype(np.float32)
    assert np.all(t.astype(np.float64) == y + h * np.arange(-12 * 256, 12 * 256 + 1))
    integral = float(oracle.likelihood(t, y).astype(np.float64).sum()) * h
    assert abs(integral - 2.5066282746310002) < 1e-6
