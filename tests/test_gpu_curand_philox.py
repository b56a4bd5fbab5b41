"""The oracle's Philox4x32-10 against cuRAND's, run on the GPU.

cuRAND's Philox4_32_10 generator (its device API, compiled here into a small
test-only library) is a third implementation of the same function, beside
the oracle's and Triton's (the CPU pin in test_oracle_generator.py).  A
counter (c0, c1, sid, tag) and key (lo32(seed), hi32(seed)) map onto cuRAND's
state as offset = 4 (c1 * 2^32 + c0), subsequence = tag * 2^32 + sid; the
first four words cuRAND then returns must equal the oracle's words.  The
counters cover the ranges the resampler draws from: particle index c0 up to
2^30, group index c1 (cuRAND's offset / 4 has 62 bits, so c1 < 2^30), every
tag and arbitrary stream ids and seeds.  The kernels' own Philox is pinned to
the oracle by the bit-exact parity tests.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox_check.so")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
           "-Xcompiler", "-fPIC", os.path.join(HERE, "curand_philox_check.cu"), "-o", out]
    proc = subprocess.run(cmd, capture_output=True, text=True)
    assert proc.returncode == 0, proc.stderr[-2000:]
    lib = ctypes.CDLL(out)
    u64p = ctypes.POINTER(ctypes.c_ulonglong)
    lib.curand_philox_words.argtypes = [ctypes.c_ulonglong, u64p, u64p,
                                        ctypes.POINTER(ctypes.c_uint), ctypes.c_int]
    lib.curand_philox_words.restype = ctypes.c_int
    return lib


def _curand(lib, seed, ctrs):
    sub = np.array([(t << 32) | s for _, _, s, t in ctrs], dtype=np.uint64)
    off = np.array([4 * ((c1 << 32) | c0) for c0, c1, _, _ in ctrs], dtype=np.uint64)
    out = np.zeros(4 * len(ctrs), dtype=np.uint32)
    u64p = ctypes.POINTER(ctypes.c_ulonglong)
    rc = lib.curand_philox_words(seed, sub.ctypes.data_as(u64p), off.ctypes.data_as(u64p),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)), len(ctrs))
    assert rc == 0, rc
    return out.reshape(-1, 4)


def test_oracle_philox_equals_curand_philox(lib):
    rng = np.random.default_rng(2109)
    seeds = [0, 1, 7, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF] + \
        [int(v) for v in rng.integers(0, 2**63, 3, dtype=np.uint64)]
    for seed in seeds:
        ctrs = [(0, 0, 0, 1), (1, 0, 0, 2), (2**30 - 1, 2**24, 7, 3), (5, 2**30 - 1, 2**32 - 1, 5)]
        for tag in (1, 2, 3, 4, 5):
            for _ in range(16):
                ctrs.append((int(rng.integers(0, 2**30)), int(rng.integers(0, 2**24)),
                             int(rng.integers(0, 2**32)), tag))
        got = _curand(lib, seed, ctrs)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for row, ctr in zip(got, ctrs):
            want = [int(v) for v in oracle.philox4x32_10(list(ctr), key)]
            assert [int(v) for v in row] == want, (hex(seed), ctr)


def test_oracle_draws_use_the_same_words_as_curand(lib):
    # One step further: the Megopolis offset and u the oracle derives from a
    # call equal those derived from cuRAND's words for the same counter.
    seed, sid = 0x5EED, 3
    n = 1000003
    ctrs = [(b, 0, sid, 1) for b in range(64)]
    words = _curand(lib, seed, ctrs)
    offs = oracle.offsets(seed, sid, len(ctrs), n)
    for b, w in enumerate(words):
        x = (int(w[1]) << 32) | int(w[0])
        assert offs[b] == (x * n) >> 64
    ctrs = [(i, g, sid, 2) for i in (0, 17, 4095) for g in range(3)]
    words = _curand(lib, seed, ctrs)
    for (i, g, _, _), w in zip(ctrs, words):
        for q in range(4):
            assert oracle.megopolis_u(seed, sid, i, 5 * g + q) == \
                np.float32(oracle.u_from_word(int(w[q])))
