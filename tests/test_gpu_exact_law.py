"""The exact small-N law on the GPU: 250,000 independent four-particle
problems in one batched launch (same weights, stream id f for problem f).
Each particle's ancestor frequencies must follow e_i P^B, P the exact
one-step kernel of the discrete acceptance rule (brute force over all 2^23
values of u), chi-squared p > 0.01 -- for Megopolis and Metropolis."""
import ctypes
import sys
import os

import numpy as np
import pytest
import torch
from scipy import stats

pytestmark = pytest.mark.gpu

mego = pytest.importorskip("paper_2109_13504_gb300")
sys.path.insert(0, os.path.dirname(__file__))
from test_oracle_chain import _exact_marginals  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("variant", [mego.MEGOPOLIS, mego.METROPOLIS])
def test_batched_n4_follows_exact_law(variant):
    w_h = np.array([0.1, 1.0, 0.35, 2.5], dtype=np.float32)
    B, F = 3, 250_000
    w = torch.from_numpy(w_h).to(DEV)
    anc = torch.full((F, 4), -1, dtype=torch.int32, device=DEV)
    arr = (mego.Filter * F)()
    wp, ap = w.data_ptr(), anc.data_ptr()
    for f in range(F):
        arr[f] = mego.Filter(wp, ap + 16 * f, None, None, 0, 4, B, f, 0)
    lib = mego._load()
    nbytes = lib.mego_batch_plan_bytes(arr, F)
    plan = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
    h = mego.BatchHandle()
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.mego_batch_plan(arr, F, variant, mego.LAYOUT_SOA, 31, plan.data_ptr(), nbytes,
                               ctypes.byref(h), stream) == mego.MEGO_OK
    assert lib.mego_batch_resample(ctypes.byref(h), stream) == mego.MEGO_OK
    torch.cuda.synchronize()
    a = anc.cpu().numpy()
    assert a.min() >= 0 and a.max() < 4
    PB = _exact_marginals(w_h, B)
    chi2 = 0.0
    for i in range(4):
        counts = np.bincount(a[:, i], minlength=4).astype(np.float64)
        chi2 += float(((counts - F * PB[i]) ** 2 / (F * PB[i])).sum())
    p = stats.chi2.sf(chi2, df=12)
    assert p > 0.01, (chi2, p)
