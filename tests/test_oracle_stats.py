"""Pins for the offspring statistics (Section 5.1) and for the oracle's
resampling quality against the paper's printed MSE/N (Tables 3 and 4).

* Statistics code: on multinomial resampling (numpy's sampler) the
  expected SE is N * sum_i p_i (1 - p_i), so MSE/N -> 1 - sum p_i^2, and the
  squared bias is only the sampling floor Var/K.
* Tables 3-4: MSE/N depends on y but hardly on N (2^15..2^22); the
  oracle at N = 2^15 must agree within its own sampling error.
"""
import json
import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np
import pytest

import oracle
import synthetic
from oracle.stats import offspring_stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_mse_tables.json")


def test_stats_against_multinomial_closed_form():
    rng = np.random.default_rng(3)
    n = 5000
    w = synthetic.gaussian_weights(n, 2.0, 6)
    p = w.astype(np.float64) / w.sum()
    K = 200
    runs = []
    for _ in range(K):
        counts = rng.multinomial(n, p)
        runs.append(np.repeat(np.arange(n), counts))
    s = offspring_stats(w, runs)
    expect = 1.0 - (p ** 2).sum()
    assert abs(s["mse_per_n"] - expect) < 0.01
    # unbiased sampler: |Bias|^2 is about Var/K
    assert s["bias2"] < 3.0 * s["var"] / K
    assert abs(s["mse"] - (s["var"] * (K - 1) / K + s["bias2"])) < 1e-6 * s["mse"]


def test_stats_hand_example():
    w = np.array([1.0, 1.0, 2.0], dtype=np.float32)       # expected 0.75, 0.75, 1.5
    runs = [np.array([2, 2, 2]), np.array([0, 1, 2])]     # offspring (0,0,3), (1,1,1)
    s = offspring_stats(w, runs)
    se1 = 0.75 ** 2 + 0.75 ** 2 + 1.5 ** 2
    se2 = 0.25 ** 2 + 0.25 ** 2 + 0.5 ** 2
    assert s["mse"] == pytest.approx((se1 + se2) / 2)
    assert s["bias2"] == pytest.approx(0.25 ** 2 * 2 + 0.5 ** 2)
    assert s["var"] == pytest.approx(0.5 + 0.5 + 2.0)
    assert s["max_offspring"] == 3


def _mse_job(args):
    y, variant, k0, K, wseed, n = args
    import oracle as o
    import synthetic as syn
    from oracle.stats import offspring_stats as st
    w = syn.gaussian_weights(n, y, wseed)
    _, B, _ = o.compute_B(w, 0.01)
    per_run = []
    for k in range(k0, k0 + K):
        s = st(w, [o.resample(w, B, 10_000 + k, variant)])
        per_run.append(s["mse_per_n"])
    return y, variant, per_run


@pytest.fixture(scope="module")
def paper():
    with open(GOLDEN) as f:
        return json.load(f)


def test_mse_per_n_matches_paper_tables(paper):
    n = 1 << 15
    K = 24
    jobs = []
    for variant in (oracle.MEGOPOLIS, oracle.METROPOLIS):
        for y in range(5):
            for wseed in (1, 2):
                for k0 in (0, K // 2):
                    jobs.append((y, variant, k0 + 100 * wseed, K // 2, wseed, n))
    oracle.build()
    res = {}
    with ProcessPoolExecutor(min(8, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        for y, variant, per_run in ex.map(_mse_job, jobs):
            res.setdefault((variant, y), []).extend(per_run)
    for (variant, y), vals in sorted(res.items()):
        name = "megopolis" if variant == oracle.MEGOPOLIS else "metropolis"
        want = paper[name]["all"][str(n)]["mse_per_n"][y]
        vals = np.asarray(vals)
        se = vals.std(ddof=1) / np.sqrt(vals.size)
        got = vals.mean()
        assert abs(got - want) <= 4.0 * se + 0.004, (name, y, got, want, se)


def _c_job(args):
    y, variant, ps, k0, K, wseed, n = args
    import oracle as o
    import synthetic as syn
    from oracle.stats import offspring_stats as st
    w = syn.gaussian_weights(n, y, wseed)
    _, B, _ = o.compute_B(w, 0.01)
    return y, variant, ps, [st(w, [o.resample(w, B, 20_000 + k, variant, psize_bytes=ps)])["mse_per_n"]
                            for k in range(k0, k0 + K)]


def test_partition_variants_match_paper_tables(paper):
    """Metropolis-C1/C2 (Algorithms 3, 4) at N = 2^15 against Tables 5-6 for
    the smallest and largest partition sizes, where both differ most from
    plain Metropolis (e.g. C1 with 128-byte partitions at y = 4: MSE/N 15.4)."""
    n = 1 << 15
    jobs = [(y, v, ps, 100 * ws, 6, ws, n) for v in (oracle.C1, oracle.C2)
            for ps in (128, 2048) for y in (0, 2, 4) for ws in (1, 2)]
    oracle.build()
    res = {}
    with ProcessPoolExecutor(min(8, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        for y, v, ps, vals in ex.map(_c_job, jobs):
            res.setdefault((v, ps, y), []).extend(vals)
    for (v, ps, y), vals in sorted(res.items()):
        name = "c1" if v == oracle.C1 else "c2"
        want = paper[name][str(ps)][str(n)]["mse_per_n"][y]
        vals = np.asarray(vals)
        se = vals.std(ddof=1) / np.sqrt(vals.size)
        assert abs(vals.mean() - want) <= 4.0 * se + 0.01 * want, (name, ps, y, vals.mean(), want)
