"""Pins for the oracle's gather (x_bar^(i) = x^(k)) and likelihood weight."""
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


def test_likelihood_closed_form():
    x = synthetic.gaussian_state(10_000, 1, 5)[0]
    x[:4] = [2.0, 0.0, -3.0, 12.0]
    w = oracle.likelihood(x, 2.0)
    ref = np.exp(-0.5 * (x.astype(np.float64) - 2.0) ** 2)
    assert w[0] == 1.0
    assert np.array_equal(w, ref.astype(np.float32))
    assert (w >= 0).all() and (w <= 1).all()
