"""mego_compute_B_noalloc: the bound for callers that cannot allocate device
memory (an application that owns all device memory through its own pool, or
a real-time loop that must not call the allocator while it runs).

It must give what mego_compute_B gives, call after call, although every call
reuses the same fixed scratch array inside the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

mego = pytest.importorskip("paper_2109_13504_gb300")

DEV = torch.device("cuda:0")


def _with_workspace(w):
    B, st, q = mego.mego_compute_B(w, 0.01)
    torch.cuda.synchronize()
    return int(B.item()), int(st.item()), float(q.item())


def _without_allocation(w, B_dev, status, q):
    # The outputs are preallocated by the test; the call itself allocates
    # nothing and goes straight through the C ABI.
    mego.mego_compute_B_noalloc(w, 0.01, B_dev, status, q)
    torch.cuda.synchronize()
    return int(B_dev.item()), int(status.item()), float(q.item())


def _same(a, b):
    # Both entry points run the same reduction grid and add the same
    # partials in the same order: B, status and q are identical, bit for bit.
    B1, s1, q1 = a
    B2, s2, q2 = b
    assert s1 == s2 == mego.MEGO_OK
    assert B1 == B2
    assert q1 == q2


def _matches_oracle(w_h, got):
    # The oracle's bound (Eq. 3, sum in double in index order) equals the
    # device's unless the value before the ceiling lies within 1e-9 of an
    # integer, where the two summation orders may round to either side.
    B, _, q = got
    st, B_ref, q_ref = oracle.compute_B(w_h, 0.01)
    assert st == oracle.OK
    assert abs(q - q_ref) <= 1e-9 * max(1.0, abs(q_ref))
    if B != B_ref:
        assert abs(q_ref - round(q_ref)) <= 1e-9 * max(1.0, abs(q_ref)) and abs(B - B_ref) <= 1


def test_noalloc_bound_matches_workspace_bound_two_calls_in_a_row():
    B_dev = torch.full((1,), -9, dtype=torch.int32, device=DEV)
    status = torch.full((1,), -9, dtype=torch.int32, device=DEV)
    q = torch.zeros(1, dtype=torch.float64, device=DEV)
    # Two calls in a row on different inputs (the second one larger, so it
    # fills all 1024 partials of the shared scratch where the first used
    # 16), then the first again; the largest case runs the widest grid.
    cases = [(1 << 16, 3.0, 1), ((1 << 21) + 77, 1.0, 2), (1 << 16, 3.0, 1),
             ((1 << 24) + 5, 4.0, 3)]
    for n, y, seed in cases:
        w_h = synthetic.gaussian_weights(n, y, seed)
        w = torch.from_numpy(w_h).to(DEV)
        got = _without_allocation(w, B_dev, status, q)
        _same(_with_workspace(w), got)
        _matches_oracle(w_h, got)


def test_noalloc_bound_reports_bad_weights_and_arguments():
    B_dev = torch.zeros(1, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    w = torch.from_numpy(synthetic.gaussian_weights(5000, 2.0, 3)).to(DEV)
    w[100] = float("nan")
    mego.mego_compute_B_noalloc(w, 0.01, B_dev, status)
    torch.cuda.synchronize()
    assert int(status.item()) == mego.MEGO_EWEIGHTS and int(B_dev.item()) == -1
    with pytest.raises(mego.MegoError):
        mego.mego_compute_B_noalloc(w, 0.0, B_dev, status)
