"""Pins for the oracle's random generator and its mappings.

Philox4x32-10 is checked against an independent library implementation
(Triton's, run by its CPU interpreter in a child process); the u and index
mappings against their distributional and range properties.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def _k(out_ptr, c_ptr, key_ptr, n: tl.constexpr):
    offs = tl.arange(0, n)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    k0 = tl.load(key_ptr + offs * 0)
    k1 = tl.load(key_ptr + 1 + offs * 0)
    a, b, c, d = tl.philox_impl(c0, c1, c2, c3, k0, k1)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)

cases = json.loads(sys.stdin.read())
res = []
for key, ctrs in cases:
    n = len(ctrs)
    c = torch.tensor([v for ctr in ctrs for v in ctr], dtype=torch.int64).to(torch.uint32)
    out = torch.zeros(4 * n, dtype=torch.uint32)
    k = torch.tensor(key, dtype=torch.int64).to(torch.uint32)
    _k[(1,)](out, c, k, n)
    res.append([int(v) & 0xFFFFFFFF for v in out.to(torch.int64).tolist()])
print(json.dumps(res))
"""


def test_philox_matches_library_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    cases = []
    for _ in range(4):
        key = [int(v) for v in rng.integers(0, 2**32, 2, dtype=np.uint64)]
        ctrs = [[int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64)]
                for _ in range(8)]
        cases.append((key, ctrs))
    # Edge counters and keys.
    cases.append(([0, 0], [[0, 0, 0, 0]] * 8))
    cases.append(([0xFFFFFFFF, 0xFFFFFFFF], [[0xFFFFFFFF] * 4] * 8))
    cases.append(([1, 0], [[i, 7, 0, 2] for i in range(8)]))
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT],
                          input=json.dumps(cases), capture_output=True, text=True,
                          timeout=600, env=dict(os.environ, TRITON_INTERPRET="1"))
    assert proc.returncode == 0, proc.stderr[-2000:]
    expect = json.loads(proc.stdout.strip().splitlines()[-1])
    for (key, ctrs), want in zip(cases, expect):
        got = []
        for ctr in ctrs:
            got.extend(int(v) for v in oracle.philox4x32_10(ctr, key))
        assert got == want, (key, ctrs)


def test_u_mapping_range_and_grid():
    assert oracle.u_from_word(0) == 1.0
    assert oracle.u_from_word(0x000001FF) == 1.0          # low 9 bits unused
    assert oracle.u_from_word(0xFFFFFE00) == 2.0 ** -23    # smallest u > 0
    assert oracle.u_from_word(0xFFFFFFFF) == 2.0 ** -23
    assert oracle.u_from_word(0x00000200) == 1.0 - 2.0 ** -23
    assert oracle.u_from_word(0x80000000) == 0.5
    rng = np.random.default_rng(5)
    for word in rng.integers(0, 2**32, 2000, dtype=np.uint64).tolist():
        u = oracle.u_from_word(word)
        assert 0.0 < u <= 1.0
        m = u * 2.0 ** 23
        assert m == int(m) and 1 <= m <= 2 ** 23
        # u depends only on the top 23 bits, and maps them one-to-one
        assert m == 2 ** 23 - (word >> 9)


def test_megopolis_u_uniform():
    us = np.array([oracle.megopolis_u(9, 0, i, b) for i in range(500) for b in range(40)])
    assert us.min() > 0.0 and us.max() <= 1.0
    ks = stats.kstest(us, "uniform")
    assert ks.pvalue > 1e-3
    # the five uniforms of one call are used by five consecutive iterations
    assert len(set(us.tolist())) > 0.99 * us.size


def test_megopolis_u_word_layout():
    """Iteration b of particle i reads call (i, b // 5, sid, 2): words 0..3
    for b mod 5 < 4; for b mod 5 = 4, the word whose bytes 1..3 are the low
    bytes of words 0..2."""
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for sid in (0, 7):
        for i in (0, 1, 31, 1000, 2**30 - 1):
            for b in range(12):
                x = [int(v) for v in oracle.philox4x32_10([i, b // 5, sid, 2], key)]
                q = b % 5
                word = x[q] if q < 4 else ((x[0] & 0xFF) << 8 | (x[1] & 0xFF) << 16
                                           | (x[2] & 0xFF) << 24)
                assert oracle.megopolis_u(seed, sid, i, b) == np.float32(oracle.u_from_word(word))


def test_megopolis_five_uniforms_independent():
    """The five uniforms of one Philox call come from disjoint bits: each is
    uniform on the 2^-23 grid and they are uncorrelated with one another
    (a fifth word that reused bits of the first three would correlate)."""
    m = 4000
    u = np.array([[oracle.megopolis_u(3, 1, i, 5 * g + q) for q in range(5)]
                  for i in range(m // 4) for g in range(4)], dtype=np.float64)
    for q in range(5):
        assert stats.kstest(u[:, q], "uniform").pvalue > 1e-3
        grid = u[:, q] * 2.0 ** 23
        assert np.all(grid == np.round(grid))
    c = np.corrcoef(u.T)
    off = c[~np.eye(5, dtype=bool)]
    # sd of a sample correlation of independent uniforms is 1/sqrt(m)
    assert np.abs(off).max() < 5.0 / np.sqrt(m)
    # Bit by bit: the 23 random bits behind each uniform (recovered exactly
    # from u) agree with any bit of another uniform of the call about half
    # the time; a shared bit would agree always (or never).
    bits = (2 ** 23 - np.round(u * 2.0 ** 23).astype(np.int64)) & 0x7FFFFF
    planes = ((bits[:, :, None] >> np.arange(23)) & 1).astype(np.float64)  # [m, 5, 23]
    for q in range(4):
        agree = (planes[:, 4, :, None] == planes[:, q, None, :]).mean(axis=0)  # [23, 23]
        assert np.abs(agree - 0.5).max() < 0.1, q


@pytest.mark.parametrize("n", [4, 37, 1000, 4096])
def test_offsets_uniform_and_in_range(n):
    B = 20000 if n <= 1000 else 40000
    o = oracle.offsets(3, 1, B, n)
    assert o.min() >= 0 and o.max() < n
    counts = np.bincount(o, minlength=n)
    chi = stats.chisquare(counts)
    assert chi.pvalue > 1e-3


def test_offsets_depend_on_seed_and_stream():
    a = oracle.offsets(1, 0, 64, 1 << 20)
    b = oracle.offsets(2, 0, 64, 1 << 20)
    c = oracle.offsets(1, 1, 64, 1 << 20)
    assert (a != b).mean() > 0.9 and (a != c).mean() > 0.9


@pytest.mark.parametrize("n", [4, 100, 4096])
def test_metropolis_proposals_uniform(n):
    js = []
    us = []
    for i in range(200):
        for b in range(100):
            j, u = oracle.metropolis_draw(11, 0, i, b, n)
            js.append(j)
            us.append(u)
    js = np.array(js)
    assert js.min() >= 0 and js.max() < n
    assert stats.chisquare(np.bincount(js, minlength=n)).pvalue > 1e-3
    assert stats.kstest(np.array(us), "uniform").pvalue > 1e-3
