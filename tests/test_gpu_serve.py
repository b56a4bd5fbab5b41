"""The serving loop: requests of different sizes admitted under a device
memory budget, batched continuously, each result identical to the same
request resampled alone (same seed, stream id = request id, B from the
bound): bit-exact ancestors and gathered state."""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

mego = pytest.importorskip("paper_2109_13504_gb300")
DEV = torch.device("cuda:0")
SEED = 2024


def _alone(w_h, x_h, rid):
    w = torch.from_numpy(w_h).to(DEV)
    x = torch.from_numpy(x_h).to(DEV)
    B_dev, status, _ = mego.mego_compute_B(w, 0.01)
    anc = torch.empty(w_h.size, dtype=torch.int32, device=DEV)
    x_out = torch.empty_like(x)
    mego.mego_resample_gather(w, 0, B_dev, SEED, rid & 0xFFFFFFFF, mego.MEGOPOLIS, x_in=x,
                              x_out=x_out, layout=mego.LAYOUT_AOS4, anc=anc)
    torch.cuda.synchronize()
    return anc.cpu().numpy(), x_out.cpu().numpy(), int(B_dev.item())


def _requests(count, seed, lo=10.0, hi=15.0):
    t, sizes = synthetic.request_stream(count, 20000.0, lo, hi, seed)
    reqs = []
    for k, n in enumerate(sizes):
        w = torch.from_numpy(synthetic.gaussian_weights(int(n), 2.0, 300 + k))
        x = torch.from_numpy(np.ascontiguousarray(synthetic.gaussian_state(int(n), 4, 700 + k).T))
        reqs.append((1000 + k, w.pin_memory(), x.pin_memory(),
                     torch.full((int(n),), -1, dtype=torch.int32).pin_memory(),
                     torch.zeros((int(n), 4), dtype=torch.float32).pin_memory()))
    return t, reqs


def test_served_results_equal_alone_under_a_small_budget():
    t, reqs = _requests(120, 1)
    biggest = max(r[1].numel() for r in reqs)
    # Room for only a few requests at a time: admission has to wait for memory.
    server = mego.Server(arena_bytes=8 * 40 * biggest + (4 << 20), seed=SEED, max_batch=64)
    server.replay(reqs, t)
    done = server.poll()
    stats = server.stats()
    server.close()
    assert len(done) == len(reqs) and all(c[1] == mego.MEGO_OK for c in done)
    assert all(c[3] > 0 for c in done)
    assert stats["batches"] > 1 and stats["max_batch"] > 1      # batching happened
    assert stats["peak_arena_bytes"] <= 8 * 40 * biggest + (4 << 20)
    B_of = {c[0]: c[4] for c in done}
    for rid, w, x, anc, x_out in reqs:
        a_ref, x_ref, B_ref = _alone(w.numpy(), x.numpy(), rid)
        assert np.array_equal(anc.numpy(), a_ref), rid
        assert np.array_equal(x_out.numpy(), x_ref), rid
        assert B_of[rid] == B_ref, rid                # the completion reports the bound's B


def test_submit_poll_drain_and_rejections():
    t, reqs = _requests(10, 2, 8.0, 12.0)
    server = mego.Server(arena_bytes=64 << 20, seed=SEED, max_batch=4, streams=3)
    for r in reqs:
        server.submit(*r)
    server.drain(60.0)
    got = server.poll()
    assert sorted(c[0] for c in got) == sorted(r[0] for r in reqs)
    rid, w, x, anc, x_out = reqs[0]
    with pytest.raises(mego.MegoError):            # state required by this server
        server.submit(5, w, None, anc, None)
    huge = torch.zeros(1 << 22, dtype=torch.float32)
    with pytest.raises(mego.MegoError) as ei:     # can never fit the budget
        server.submit(6, huge, torch.zeros((1 << 22, 4), dtype=torch.float32))
    assert ei.value.status == mego.MEGO_ENOMEM
    server.close()
    for rid, w, x, anc, x_out in reqs:
        a_ref, x_ref, _ = _alone(w.numpy(), x.numpy(), rid)
        assert np.array_equal(anc.numpy(), a_ref) and np.array_equal(x_out.numpy(), x_ref)


@pytest.mark.parametrize("mode", ["copies", "weights_in_place", "pageable"])
def test_copied_buffers_match_direct_ones(mode):
    """By default inputs are uploaded and results written in place into
    page-locked buffers; host_copies = 1 copies both ways, 2 also reads the
    weights in place; pageable buffers are always copied.  All give the same
    results."""
    t, reqs = _requests(12, 3, 8.0, 14.0)
    if mode == "pageable":
        reqs = [(rid, w.clone(), x.clone(), anc.clone(), x_out.clone())
                for rid, w, x, anc, x_out in reqs]
        assert not reqs[0][1].is_pinned()
    server = mego.Server(arena_bytes=256 << 20, seed=SEED, max_batch=4, streams=2,
                         host_copies={"copies": 1, "weights_in_place": 2}.get(mode, 0))
    for r in reqs:
        server.submit(*r)
    server.drain(60.0)
    done = server.poll()
    server.close()
    assert len(done) == len(reqs) and all(c[1] == mego.MEGO_OK for c in done)
    for rid, w, x, anc, x_out in reqs:
        a_ref, x_ref, _ = _alone(w.numpy(), x.numpy(), rid)
        assert np.array_equal(anc.numpy(), a_ref), rid
        assert np.array_equal(x_out.numpy(), x_ref), rid
