"""Pins for the Megopolis proposal index (Algorithm 5, Section 4).

Section 4 states what the index achieves rather than only how it is
computed: a warp's 32 threads read inside one aligned 32-weight partition
(the "wrapped sequential" pattern, four 32-byte transactions), each offset
still gives each particle a distinct index, and each particle sees every
particle with the same probability.  These tests check those properties of
the oracle's index; they do not retype its formula.
"""
import numpy as np
import pytest

import oracle


def _index_map(n, o):
    return np.array([oracle.megopolis_index(i, o, n) for i in range(n)])


@pytest.mark.parametrize("n", [32, 64, 96, 4096])
@pytest.mark.parametrize("o_sel", [0, 5, 31, 32, 1000, -1])
def test_each_offset_permutes_particles(n, o_sel):
    o = (n - 1) if o_sel == -1 else o_sel % n
    j = _index_map(n, o)
    assert j.min() >= 0 and j.max() < n
    assert np.array_equal(np.sort(j), np.arange(n))


@pytest.mark.parametrize("n", [64, 4096])
def test_warp_reads_one_aligned_partition_as_a_rotation(n):
    rng = np.random.default_rng(0)
    for o in rng.integers(0, n, 20).tolist():
        j = _index_map(n, o)
        for w0 in range(0, n, 32):
            jw = j[w0:w0 + 32]
            base = jw.min()
            # one aligned 128-byte partition: 4 sectors of 32 bytes
            assert base % 32 == 0 and jw.max() == base + 31
            assert len(set((jw * 4 // 32).tolist())) == 4
            # lane l reads lane (l + o) mod 32 of the partition
            assert np.array_equal(jw - base, (np.arange(32) + o) % 32)
            # the partition moves by whole partitions: floor(o/32) of them
            assert base // 32 == (w0 // 32 + o // 32) % (n // 32)


@pytest.mark.parametrize("n", [4, 16, 32, 96, 4096])
def test_each_particle_sees_every_index_once_over_offsets(n):
    # For a uniform offset the proposal of any fixed particle is uniform.
    for i in sorted({0, 1, n // 2, n - 1}):
        j = np.array([oracle.megopolis_index(i, o, n) for o in range(n)])
        assert np.array_equal(np.sort(j), np.arange(n))


def test_congruence_mod_32():
    n = 1 << 12
    rng = np.random.default_rng(7)
    for _ in range(2000):
        i, o = (int(v) for v in rng.integers(0, n, 2))
        j = oracle.megopolis_index(i, o, n)
        assert j % 32 == (i + o) % 32


@pytest.mark.parametrize("n,tv_max", [(33, 0.1), (100, 0.1), (1000, 0.02)])
def test_ragged_n_marginal_close_to_uniform(n, tv_max):
    # When 32 does not divide N the index is still in range, and the
    # marginal over a uniform offset departs from uniform only a little.
    worst = 0.0
    for i in range(n):
        j = np.array([oracle.megopolis_index(i, o, n) for o in range(n)])
        assert j.min() >= 0 and j.max() < n
        p = np.bincount(j, minlength=n) / n
        worst = max(worst, 0.5 * np.abs(p - 1.0 / n).sum())
    assert worst < tv_max
