"""Pins for the oracle's resampling chains (Algorithms 2 and 5).

* Equal weights: every proposal is accepted (u <= 1), so the final ancestor
  is the last proposal.
* One nonzero weight: a chain there never leaves (u > 0); any other chain
  is absorbed the first time the heavy particle is proposed, so
  P(absorbed after B) = 1 - (1 - 1/N)^B (the recurrence of Proposition 1,
  which is exact in this case).
* N = 4: each particle's ancestor law after B iterations is e_i P^B for the
  exact one-step kernel P of the discrete acceptance rule, computed here by
  brute force over all 2^23 values of u; the oracle's empirical frequencies
  over 10^6 seeds must agree (chi-squared).
* Offspring bound: with 32 | N every particle is proposed exactly once per
  Megopolis iteration, so no particle gets more than B + 1 offspring.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
import synthetic

VARIANTS = [oracle.MEGOPOLIS, oracle.METROPOLIS]


@pytest.mark.parametrize("n", [1, 5, 64, 1000])
@pytest.mark.parametrize("B", [1, 7, 32])
def test_equal_weights_take_the_last_proposal(n, B):
    w = np.full(n, 0.37, dtype=np.float32)
    seed = 77
    anc = oracle.resample(w, B, seed, oracle.MEGOPOLIS)
    o_last = oracle.offset(seed, 0, B - 1, n)
    want = [oracle.megopolis_index(i, o_last, n) for i in range(n)]
    assert anc.tolist() == want
    anc = oracle.resample(w, B, seed, oracle.METROPOLIS)
    want = [oracle.metropolis_draw(seed, 0, i, B - 1, n)[0] for i in range(n)]
    assert anc.tolist() == want


@pytest.mark.parametrize("variant", VARIANTS)
def test_zero_iterations_is_identity_and_single_particle(variant):
    w = synthetic.gaussian_weights(100, 2.0, 3)
    assert oracle.resample(w, 0, 1, variant).tolist() == list(range(100))
    assert oracle.resample(np.ones(1, np.float32), 50, 1, variant).tolist() == [0]


@pytest.mark.parametrize("variant", VARIANTS)
def test_subrange_matches_full_run(variant):
    w = synthetic.gaussian_weights(3000, 1.0, 4)
    full = oracle.resample(w, 12, 5, variant)
    part = np.concatenate([oracle.resample(w, 12, 5, variant, i0=a, i1=b)
                           for a, b in [(0, 1000), (1000, 1001), (1001, 3000)]])
    assert np.array_equal(full, part)
    idx = [0, 31, 32, 2999]
    assert oracle.resample_at(w, 12, 5, idx, variant).tolist() == full[idx].tolist()


@pytest.mark.parametrize("variant", VARIANTS)
def test_host_thread_split_matches_single_thread(variant):
    # The split run that checks full-size GPU results uses many contiguous
    # [i0, i1) ranges on host threads; it must give the single-threaded array.
    n = 50_000 + 13
    w = synthetic.gaussian_weights(n, 3.0, 8)
    full = oracle.resample(w, 21, 6, variant, stream_id=4)
    for threads in (2, 3, 8):
        assert np.array_equal(oracle.resample(w, 21, 6, variant, stream_id=4,
                                              threads=threads), full)
    sub = oracle.resample(w, 21, 6, variant, stream_id=4, i0=777, i1=n - 5, threads=5)
    assert np.array_equal(sub, full[777:n - 5])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,B", [(16, 5), (100, 40), (1024, 300)])
def test_single_heavy_particle_absorption_rate(variant, n, B):
    p = n // 3
    w = np.zeros(n, dtype=np.float32)
    w[p] = 0.75
    absorbed = 0
    total = 0
    seeds = max(1, 20000 // n)
    for s in range(seeds):
        anc = oracle.resample(w, B, 1000 + s, variant)
        assert anc[p] == p                      # the heavy chain never leaves
        others = np.delete(anc, p)
        absorbed += int((others == p).sum())
        total += others.size
    prob = 1.0 - (1.0 - 1.0 / n) ** B
    if variant == oracle.METROPOLIS:
        # independent chains: exact binomial test
        assert stats.binomtest(absorbed, total, prob).pvalue > 1e-3
    else:
        # Megopolis chains share offsets (correlated): compare the mean with
        # a looser bound based on per-seed dispersion.
        assert abs(absorbed / total - prob) < 0.03 + 4 * np.sqrt(prob * (1 - prob) / seeds)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", [4, 32, 64, 256])
def test_large_B_absorbs_every_chain(variant, n):
    B = int(np.ceil(n * (np.log(n) + 20.0)))
    w = np.zeros(n, dtype=np.float32)
    w[n - 1] = 2.0
    anc = oracle.resample(w, B, 4242, variant)
    assert (anc == n - 1).all()


def _acceptance_prob(wk: np.float32, wj: np.float32) -> float:
    """#{m in [1, 2^23] : fl(m 2^-23 * wk) <= wj} / 2^23, by bisection
    (fl(m 2^-23 * wk) is non-decreasing in m)."""
    wk = np.float32(wk)
    wj = np.float32(wj)

    def ok(m):
        u = np.float32(m) * np.float32(2.0 ** -23)     # exact
        return np.float32(u * wk) <= wj

    lo, hi = 0, 1 << 23                       # ok(lo) is vacuous, find max m
    if ok(hi):
        return 1.0
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo / float(1 << 23)


def _exact_marginals(w, B):
    n = len(w)
    P = np.zeros((n, n))
    for k in range(n):
        for j in range(n):
            if j != k:
                P[k, j] = _acceptance_prob(w[k], w[j]) / n
        P[k, k] = 1.0 - P[k].sum()
    return np.linalg.matrix_power(P, B)


@pytest.mark.parametrize("variant", VARIANTS)
def test_n4_exact_distribution(variant):
    w = np.array([0.1, 1.0, 0.35, 2.5], dtype=np.float32)
    B = 3
    nseeds = 1_000_000
    counts = oracle.ancestor_counts(w, B, 1, nseeds, variant).astype(np.float64)
    PB = _exact_marginals(w, B)
    chi2 = 0.0
    for i in range(4):
        expect = PB[i] * nseeds
        assert counts[i].sum() == nseeds
        chi2 += float(((counts[i] - expect) ** 2 / expect).sum())
    p = stats.chi2.sf(chi2, df=4 * 3)
    assert p > 0.01, (chi2, p)


@pytest.mark.parametrize("variant", VARIANTS)
def test_n4_exact_distribution_subnormal_weights(variant):
    # All four weights subnormal, so every product u w_k is subnormal or
    # underflows: the exact law (numpy's IEEE binary32 with gradual
    # underflow) holds only if the oracle neither flushes subnormals to zero
    # (which would accept every proposal) nor rounds differently.
    w = np.array([2.0 ** -140, 2.0 ** -128, 2.0 ** -135, 0.75 * 2.0 ** -126], dtype=np.float32)
    assert np.all(w < np.float32(2.0 ** -126)) and np.all(w > 0)
    B = 3
    nseeds = 1_000_000
    counts = oracle.ancestor_counts(w, B, 5, nseeds, variant).astype(np.float64)
    PB = _exact_marginals(w, B)
    flushed = _exact_marginals(np.ones(4, dtype=np.float32), B)   # what FTZ would give
    assert np.abs(PB - flushed).max() > 0.1
    chi2 = 0.0
    for i in range(4):
        expect = PB[i] * nseeds
        chi2 += float(((counts[i] - expect) ** 2 / np.maximum(expect, 1e-12)).sum())
    p = stats.chi2.sf(chi2, df=4 * 3)
    assert p > 0.01, (chi2, p)


def test_n4_detects_a_reversed_acceptance():
    # The exact law is sensitive to the direction of the acceptance test:
    # the reversed rule (accept iff u*w_j <= w_k) gives a different P^B.
    w = np.array([0.1, 1.0, 0.35, 2.5], dtype=np.float32)
    right = _exact_marginals(w, 3)
    wrong = _exact_marginals(1.0 / w, 3)
    assert np.abs(right - wrong).max() > 0.05


@pytest.mark.parametrize("n", [64, 4096])
def test_megopolis_offspring_bound(n):
    for y, B in [(3.0, 60), (4.0, 200)]:
        w = synthetic.gaussian_weights(n, y, 8)
        anc = oracle.resample(w, B, 9, oracle.MEGOPOLIS)
        assert np.bincount(anc, minlength=n).max() <= B + 1
