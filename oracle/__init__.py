"""CPU oracle for the Megopolis / Metropolis resampling hot path.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import this package.  The CUDA path never loads it, and it shares no code
with the CUDA path.

The arithmetic lives in ``megopolis_oracle.c`` (plain C, single-threaded,
``-O2 -ffp-contract=off``), compiled on first use into
``oracle/_build/libmegopolis_oracle.so`` and called through ctypes.  The
offspring statistics of Section 5.1 (Eqs. 14-21) live in ``oracle.stats``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "megopolis_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libmegopolis_oracle.so")

MEGOPOLIS = 0
METROPOLIS = 1
C1 = 2
C2 = 3

OK = 0
EINVAL = 1
ENOMEM = 2
EWEIGHTS = 5

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc; return its path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u32, i32, u64, f64 = (ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64,
                              ctypes.c_double)
        vp = ctypes.c_void_p
        lib.oracle_philox4x32_10.argtypes = [vp, vp, vp]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_u_from_word.argtypes = [u32]
        lib.oracle_u_from_word.restype = ctypes.c_float
        lib.oracle_offset.argtypes = [u64, u32, u32, u32]
        lib.oracle_offset.restype = u32
        lib.oracle_megopolis_u.argtypes = [u64, u32, u32, u32]
        lib.oracle_megopolis_u.restype = ctypes.c_float
        lib.oracle_metropolis_draw.argtypes = [u64, u32, u32, u32, u32, vp, vp]
        lib.oracle_metropolis_draw.restype = None
        lib.oracle_megopolis_index.argtypes = [u32, u32, u32]
        lib.oracle_megopolis_index.restype = u32
        lib.oracle_resample.argtypes = [vp, u32, i32, u64, u32, ctypes.c_int,
                                        u32, u32, u32, vp]
        lib.oracle_resample.restype = ctypes.c_int
        lib.oracle_ancestor_counts.argtypes = [vp, u32, i32, u64, u64, u32,
                                               ctypes.c_int, u32, vp]
        lib.oracle_ancestor_counts.restype = ctypes.c_int
        lib.oracle_reduce.argtypes = [vp, u32, vp, vp]
        lib.oracle_reduce.restype = ctypes.c_int
        lib.oracle_compute_B.argtypes = [vp, u32, f64, i32, vp, vp]
        lib.oracle_compute_B.restype = ctypes.c_int
        lib.oracle_gather_soa.argtypes = [vp, vp, vp, u32, u32, u64]
        lib.oracle_gather_soa.restype = ctypes.c_int
        lib.oracle_gather_aos4.argtypes = [vp, vp, vp, u32]
        lib.oracle_gather_aos4.restype = ctypes.c_int
        lib.oracle_likelihood.argtypes = [vp, u32, ctypes.c_float, vp]
        lib.oracle_likelihood.restype = None
        lib.oracle_sir_predict_update.argtypes = [vp, vp, u32, ctypes.c_float, ctypes.c_float,
                                                  vp, vp]
        lib.oracle_sir_predict_update.restype = None
        lib.oracle_mean.argtypes = [vp, u32]
        lib.oracle_mean.restype = f64
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def _check(status: int, what: str) -> None:
    if status != OK:
        raise OracleError("%s failed with status %d" % (what, status))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------
# Generator and mappings


def philox4x32_10(counter, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u_from_word(word: int) -> float:
    return float(np.float32(_load().oracle_u_from_word(int(word) & 0xFFFFFFFF)))


def offset(seed: int, stream_id: int, b: int, n: int) -> int:
    """The Megopolis offset o^(b) (Algorithm 5, first loop)."""
    return int(_load().oracle_offset(seed, stream_id, b, n))


def offsets(seed: int, stream_id: int, B: int, n: int) -> np.ndarray:
    lib = _load()
    return np.array([lib.oracle_offset(seed, stream_id, b, n) for b in range(B)],
                    dtype=np.int64)


def megopolis_u(seed: int, stream_id: int, i: int, b: int) -> np.float32:
    return np.float32(_load().oracle_megopolis_u(seed, stream_id, i, b))


def metropolis_draw(seed: int, stream_id: int, i: int, b: int, n: int):
    j = ctypes.c_uint32()
    u = ctypes.c_float()
    _load().oracle_metropolis_draw(seed, stream_id, i, b, n,
                                   ctypes.addressof(j), ctypes.addressof(u))
    return int(j.value), np.float32(u.value)


def megopolis_index(i: int, o: int, n: int) -> int:
    """j of Algorithm 5 for particle i under offset o."""
    return int(_load().oracle_megopolis_index(i, o, n))


# --------------------------------------------------------------------------
# Resampling


def host_threads() -> int:
    """Host threads a split oracle run uses: every core of this machine."""
    return max(1, os.cpu_count() or 1)


def resample(w, B: int, seed: int, variant: int = MEGOPOLIS, stream_id: int = 0,
             i0: int = 0, i1: int | None = None, psize_bytes: int = 0,
             threads: int = 1) -> np.ndarray:
    """Ancestors of particles [i0, i1) (default: all) as int32.

    threads > 1 splits [i0, i1) into contiguous sub-ranges and runs the
    single-threaded C oracle on each from a pool of host threads (ctypes
    releases the interpreter lock during the call).  Every particle's chain
    depends only on (w, B, seed, stream id, its own index), so the result is
    the same array as the single-threaded run; only the wall time changes.
    """
    lib = _load()
    w = _f32(w)
    n = w.shape[0]
    if i1 is None:
        i1 = n
    out = np.empty(max(i1 - i0, 0), dtype=np.int32)
    if threads <= 1 or i1 - i0 < 4096:
        st = lib.oracle_resample(_ptr(w), n, int(B), int(seed), int(stream_id),
                                 int(variant), int(psize_bytes), int(i0), int(i1),
                                 _ptr(out))
        _check(st, "oracle_resample")
        return out
    # Four ranges per thread, so that uneven per-range times still balance.
    pieces = min(4 * int(threads), (i1 - i0) // 1024)
    cuts = [i0 + (i1 - i0) * k // pieces for k in range(pieces + 1)]

    def one(k):
        a, b = cuts[k], cuts[k + 1]
        return lib.oracle_resample(_ptr(w), n, int(B), int(seed), int(stream_id),
                                   int(variant), int(psize_bytes), a, b,
                                   _ptr(out) + 4 * (a - i0))

    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=int(threads)) as ex:
        for st in ex.map(one, range(pieces)):
            _check(st, "oracle_resample")
    return out


def resample_at(w, B: int, seed: int, idx, variant: int = MEGOPOLIS,
                stream_id: int = 0, psize_bytes: int = 0) -> np.ndarray:
    """Ancestors of the particles listed in idx, one by one."""
    lib = _load()
    w = _f32(w)
    n = w.shape[0]
    idx = np.asarray(idx, dtype=np.int64)
    out = np.empty(idx.shape[0], dtype=np.int32)
    one = np.empty(1, dtype=np.int32)
    for t, i in enumerate(idx.tolist()):
        st = lib.oracle_resample(_ptr(w), n, int(B), int(seed), int(stream_id),
                                 int(variant), int(psize_bytes), i, i + 1,
                                 _ptr(one))
        _check(st, "oracle_resample")
        out[t] = one[0]
    return out


def ancestor_counts(w, B: int, seed0: int, nseeds: int, variant: int = MEGOPOLIS,
                    stream_id: int = 0, psize_bytes: int = 0) -> np.ndarray:
    """counts[i, k]: over seeds seed0.., how often particle i ended at k."""
    lib = _load()
    w = _f32(w)
    n = w.shape[0]
    counts = np.zeros((n, n), dtype=np.uint64)
    st = lib.oracle_ancestor_counts(_ptr(w), n, int(B), int(seed0), int(nseeds),
                                    int(stream_id), int(variant),
                                    int(psize_bytes), _ptr(counts))
    _check(st, "oracle_ancestor_counts")
    return counts


# --------------------------------------------------------------------------
# Bound, gather, likelihood

B_MAX_DEFAULT = 1 << 24


def reduce(w):
    """(status, max w as float32, sum w in double)."""
    lib = _load()
    w = _f32(w)
    m = ctypes.c_float()
    s = ctypes.c_double()
    st = lib.oracle_reduce(_ptr(w), w.shape[0], ctypes.addressof(m),
                           ctypes.addressof(s))
    return st, np.float32(m.value), float(s.value)


def compute_B(w, eps: float, b_max: int = B_MAX_DEFAULT):
    """(status, B, q) with q the value before the ceiling (Eq. 3)."""
    lib = _load()
    w = _f32(w)
    B = ctypes.c_int32(-1)
    q = ctypes.c_double(float("nan"))
    st = lib.oracle_compute_B(_ptr(w), w.shape[0], float(eps), int(b_max),
                              ctypes.addressof(B), ctypes.addressof(q))
    return st, int(B.value), float(q.value)


def gather_soa(x_in, anc) -> np.ndarray:
    """x_out[d, i] = x_in[d, anc[i]] for a [dim, n] float32 array."""
    lib = _load()
    x_in = _f32(x_in)
    anc = np.ascontiguousarray(anc, dtype=np.int32)
    dim, n = x_in.shape
    out = np.empty_like(x_in)
    _check(lib.oracle_gather_soa(_ptr(x_in), _ptr(out), _ptr(anc), n, dim, n),
           "oracle_gather_soa")
    return out


def gather_aos4(x_in, anc) -> np.ndarray:
    """x_out[i, :] = x_in[anc[i], :] for an [n, 4] float32 array."""
    lib = _load()
    x_in = _f32(x_in)
    anc = np.ascontiguousarray(anc, dtype=np.int32)
    out = np.empty_like(x_in)
    _check(lib.oracle_gather_aos4(_ptr(x_in), _ptr(out), _ptr(anc), x_in.shape[0]),
           "oracle_gather_aos4")
    return out


def likelihood(x, y: float) -> np.ndarray:
    """w_i = exp(-(x_i - y)^2 / 2) in double, rounded to float32."""
    lib = _load()
    x = _f32(x)
    w = np.empty_like(x)
    lib.oracle_likelihood(_ptr(x), x.shape[0], ctypes.c_float(y), _ptr(w))
    return w


def sir_predict_update(x, v, drift: float, z: float):
    """Predict (Eq. 22) and weight (Eq. 23) of the SIR filter: (x_pred, w)."""
    lib = _load()
    x = _f32(x)
    v = _f32(v)
    xp = np.empty_like(x)
    w = np.empty_like(x)
    lib.oracle_sir_predict_update(_ptr(x), _ptr(v), x.shape[0], ctypes.c_float(drift),
                                  ctypes.c_float(z), _ptr(xp), _ptr(w))
    return xp, w


def mean(x) -> float:
    x = _f32(x)
    return float(_load().oracle_mean(_ptr(x), x.shape[0]))
