"""Pins for the iteration bound B (Eq. 3; Proposition 1, Eq. 4).

* Closed form: for the weights of Eq. 12, E(w)/max(w) = exp(-y^2/4)/sqrt(2)
  (Section 6.3), so the population B at eps = 0.01 is 4, 6, 16, 60, 354 for
  y = 0..4.  The bound computed from 2^20 samples must land within a few
  iterations of it (the sample maximum is a little below the population
  maximum).
* One nonzero weight among N: E(w)/w_p = 1/N, so B is the least integer
  with (1 - 1/N)^B <= eps, and the absorbed fraction after B iterations is
  at least 1 - eps (Proposition 1's recurrence is exact here).
* Special cases: equal weights give B = 0; eps = 1 gives B = 0; invalid
  weights and eps are rejected.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic


def _population_B(y, eps):
    r = math.exp(-y * y / 4.0) / math.sqrt(2.0)
    return math.ceil(math.log(eps) / math.log(1.0 - r))


def test_population_closed_form_values():
    assert [_population_B(y, 0.01) for y in range(5)] == [4, 6, 16, 60, 354]
    assert [_population_B(y, 0.1) for y in range(5)] == [2, 3, 8, 30, 177]


@pytest.mark.parametrize("y", [0, 1, 2, 3, 4])
def test_sample_bound_near_population_bound(y):
    w = synthetic.gaussian_weights(1 << 20, y, 1)
    st, B, q = oracle.compute_B(w, 0.01)
    assert st == oracle.OK
    assert B == math.ceil(q)
    assert abs(B - _population_B(y, 0.01)) <= 3


def test_bound_matches_exact_sum():
    # The double sum in index order against an exactly rounded sum.
    for y in range(5):
        w = synthetic.gaussian_weights(50_000, y, 2)
        st, B, q = oracle.compute_B(w, 0.01)
        r = (math.fsum(w.astype(np.float64).tolist()) / w.size) / float(w.max())
        q_ref = math.log(0.01) / math.log1p(-r)
        assert abs(q - q_ref) <= 1e-9 * q_ref
        assert B == math.ceil(q_ref)


@pytest.mark.parametrize("n", [8, 64, 500])
@pytest.mark.parametrize("eps", [0.5, 0.1, 0.01])
def test_single_nonzero_weight_bound_and_coverage(n, eps):
    w = np.zeros(n, dtype=np.float32)
    w[n // 2] = 3.0
    st, B, q = oracle.compute_B(w, eps)
    assert st == oracle.OK
    assert (1.0 - 1.0 / n) ** B <= eps * (1 + 1e-12)
    assert (1.0 - 1.0 / n) ** (B - 1) > eps
    for variant in (oracle.MEGOPOLIS, oracle.METROPOLIS):
        hits = 0
        total = 0
        for s in range(max(4, 4000 // n)):
            anc = oracle.resample(w, B, 500 + s, variant)
            hits += int((anc == n // 2).sum())
            total += n
        # E[absorbed] = 1 - (1-1/N)^B >= 1 - eps; allow sampling slack
        assert hits / total >= 1.0 - eps - 0.05


def test_special_cases():
    w = np.full(1000, 0.25, dtype=np.float32)
    assert oracle.compute_B(w, 0.01)[:2] == (oracle.OK, 0)
    w = synthetic.gaussian_weights(1000, 2.0, 1)
    assert oracle.compute_B(w, 1.0)[:2] == (oracle.OK, 0)
    assert oracle.compute_B(w, 0.0)[0] == oracle.EINVAL
    assert oracle.compute_B(w, 1.5)[0] == oracle.EINVAL
    for bad in (np.nan, np.inf, -1.0):
        v = w.copy()
        v[10] = bad
        assert oracle.compute_B(v, 0.01)[0] == oracle.EWEIGHTS
    assert oracle.compute_B(np.zeros(10, np.float32), 0.01)[0] == oracle.EWEIGHTS
    # a bound beyond the cap is reported, not silently clamped
    w = np.zeros(1 << 16, dtype=np.float32)
    w[0] = 1.0
    assert oracle.compute_B(w, 0.01, b_max=1000)[0] == oracle.EWEIGHTS
    # unnormalised weights: B is scale-free
    w = synthetic.gaussian_weights(4096, 3.0, 5)
    assert oracle.compute_B(w, 0.01)[1] == oracle.compute_B(w * np.float32(64.0), 0.01)[1]
