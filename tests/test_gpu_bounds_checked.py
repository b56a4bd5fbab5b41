"""The bounds-checked build of the single-resample library.

Compiled with -DMEGO_BOUNDS_CHECK, every weight and state index the chains
form is checked against n before it is used; a bad one is recorded in the
variant's fault word (value 2) and replaced by 0, so nothing is read out of
range.  Over ragged sizes, every variant, weight path and launch shape, no
index may be out of range (fault word 0), and the ancestors and gathered
state must still equal the oracle's.  The library is built here on demand
(nvcc, the same sm_103a flags) and called through its C ABI with ctypes.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
MEGOPOLIS, METROPOLIS, C1, C2 = 0, 1, 2, 3
PATH_GLOBAL, PATH_SMEM, PATH_TMA = 1, 2, 3


class LaunchCfg(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ppt", ctypes.c_int32),
                ("path", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


@pytest.fixture(scope="module")
def lib():
    from paper_2109_13504_gb300 import build
    lib = ctypes.CDLL(build.build_checked())
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.mego_resample_gather.argtypes = [vp, i32, i32, vp, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_int, ctypes.c_uint32, vp, vp, i32,
                                         ctypes.c_int64, ctypes.c_int, vp,
                                         ctypes.POINTER(LaunchCfg), vp]
    lib.mego_resample_gather.restype = ctypes.c_int
    lib.mego_device_fault.argtypes = [vp]
    lib.mego_device_fault.restype = ctypes.c_int
    return lib


def _fault(lib):
    h = ctypes.c_int32(-1)
    assert lib.mego_device_fault(ctypes.addressof(h)) == 0
    return h.value


def _run(lib, w_h, B, variant, cfg, psize=0, x_h=None):
    n = w_h.size
    w = torch.from_numpy(w_h).to(DEV)
    anc = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    x = x_out = None
    if x_h is not None:
        x = torch.from_numpy(x_h).to(DEV)
        x_out = torch.full_like(x, -1.0)
    c = LaunchCfg(*cfg, 0)
    st = lib.mego_resample_gather(w.data_ptr(), n, B, None, 5, 2, variant, psize,
                                  x.data_ptr() if x is not None else None,
                                  x_out.data_ptr() if x_out is not None else None,
                                  x_h.shape[0] if x_h is not None else 0,
                                  n if x_h is not None else 0, 0, anc.data_ptr(),
                                  ctypes.byref(c), None)
    torch.cuda.synchronize()
    return st, anc.cpu().numpy(), (x_out.cpu().numpy() if x_out is not None else None)


@pytest.mark.parametrize("variant", [MEGOPOLIS, METROPOLIS])
def test_no_index_out_of_range_and_oracle_equal(lib, variant):
    assert _fault(lib) == 0
    shapes = [(64, 1), (128, 2), (256, 4), (128, 6)]
    for n in (1, 31, 33, 100, 389, 4097, 70001):
        w_h = synthetic.gaussian_weights(n, 2.5, 60 + n)
        for B in (0, 1, 7, 33):
            ref = oracle.resample(w_h, B, 5, variant, stream_id=2)
            paths = [PATH_GLOBAL] + ([PATH_SMEM] if n <= 20000 else [])
            for path in paths:
                for threads, ppt in shapes:
                    if ppt == 6 and variant != MEGOPOLIS:
                        continue
                    st, got, _ = _run(lib, w_h, B, variant, (threads, ppt, path))
                    assert st == 0
                    assert np.array_equal(got, ref), (n, B, path, threads, ppt)
            if variant == MEGOPOLIS and n >= 64 * 6:
                for threads, ppt in ((128, 6), (256, 4)):
                    st, got, _ = _run(lib, w_h, B, variant, (threads, ppt, PATH_TMA))
                    assert st == 0 and np.array_equal(got, ref), (n, B, "tma", ppt)
            assert _fault(lib) == 0, (n, B)


@pytest.mark.parametrize("variant,psize", [(C1, 128), (C2, 512)])
def test_partition_variants_stay_in_range(lib, variant, psize):
    n = 8192
    w_h = synthetic.gaussian_weights(n, 3.0, 8)
    for B in (1, 33):
        ref = oracle.resample(w_h, B, 5, variant, stream_id=2, psize_bytes=psize)
        for ppt in (1, 2, 4):
            st, got, _ = _run(lib, w_h, B, variant, (256, ppt, PATH_GLOBAL), psize=psize)
            assert st == 0 and np.array_equal(got, ref), (B, ppt)
    assert _fault(lib) == 0


def test_gather_indices_stay_in_range(lib):
    n = 70001
    w_h = synthetic.gaussian_weights(n, 2.0, 9)
    x_h = synthetic.gaussian_state(n, 3, 10)
    ref = oracle.resample(w_h, 16, 5, MEGOPOLIS, stream_id=2)
    st, got, x_out = _run(lib, w_h, 16, MEGOPOLIS, (128, 6, PATH_GLOBAL), x_h=x_h)
    assert st == 0 and np.array_equal(got, ref)
    assert np.array_equal(x_out, oracle.gather_soa(x_h, ref))
    assert _fault(lib) == 0
