"""The serving loop: requests of different sizes admitted under a device
memory budget, batched continuously, each result identical to the same
request resampled alone (same seed, stream id = request id, B from the
bound): bit-exact ancestors and gathered state."""
import numpy as np
import pytest
import torch

import oracle
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


def test_served_results_equal_the_oracle_up_to_2p20():
    """Requests shaped like the serving workload (N = floor(2^U[10,20]),
    Eq. 12 weights with y = 2, 4-dim AoS state), served in a mix under a
    budget that holds several at once: every ancestor and every gathered
    state row equals the CPU oracle's (Algorithm 5 with the request's id as
    stream id, then the gather), and each completion reports the oracle's B.
    The largest request is 2^20 particles."""
    t, reqs = _requests(14, 11, 10.0, 20.0)
    n = 1 << 20
    w = torch.from_numpy(synthetic.gaussian_weights(n, 2.0, 999)).pin_memory()
    x = torch.from_numpy(np.ascontiguousarray(synthetic.gaussian_state(n, 4, 998).T)).pin_memory()
    reqs.append((5000, w, x, torch.full((n,), -1, dtype=torch.int32).pin_memory(),
                 torch.zeros((n, 4), dtype=torch.float32).pin_memory()))
    t = list(t) + [float(t[-1])]
    server = mego.Server(arena_bytes=3 * 40 * n + (8 << 20), seed=SEED, max_batch=8)
    server.replay(reqs, t)
    done = {c[0]: c for c in server.poll()}
    server.close()
    assert len(done) == len(reqs)
    threads = oracle.host_threads()
    for rid, w, x, anc, x_out in reqs:
        c = done[rid]
        assert c[1] == mego.MEGO_OK, rid
        w_h = w.numpy()
        st, B_ref, q_ref = oracle.compute_B(w_h, 0.01)
        assert st == oracle.OK
        assert c[4] == B_ref or (abs(q_ref - round(q_ref)) <= 1e-9 * max(1.0, q_ref)
                                 and abs(c[4] - B_ref) <= 1), (rid, c[4], B_ref)
        ref = oracle.resample(w_h, c[4], SEED, oracle.MEGOPOLIS, stream_id=rid & 0xFFFFFFFF,
                              threads=threads)
        assert np.array_equal(anc.numpy(), ref), rid
        assert np.array_equal(x_out.numpy(), oracle.gather_aos4(x.numpy(), ref)), rid


def test_request_with_invalid_weights_completes_with_an_error():
    """A request whose weights the bound rejects (a NaN, or all zero)
    completes with MEGO_EWEIGHTS and B = -1; its output buffers are left as
    they were, and the requests batched with it are served normally."""
    t, reqs = _requests(6, 12, 8.0, 12.0)
    bad = []
    for k, fill in enumerate((float("nan"), 0.0)):
        rid, w, x, anc, x_out = reqs[2 * k + 1]
        if fill == fill:
            w.fill_(fill)
        else:
            w[w.numel() // 2] = fill
        bad.append(rid)
    server = mego.Server(arena_bytes=256 << 20, seed=SEED, max_batch=8)
    for r in reqs:
        server.submit(*r)
    server.drain(60.0)
    done = {c[0]: c for c in server.poll()}
    server.close()
    assert len(done) == len(reqs)
    for rid, w, x, anc, x_out in reqs:
        c = done[rid]
        if rid in bad:
            assert c[1] == mego.MEGO_EWEIGHTS and c[4] == -1, c
            assert (anc.numpy() == -1).all() and (x_out.numpy() == 0).all()
        else:
            assert c[1] == mego.MEGO_OK, c
            a_ref, x_ref, B_ref = _alone(w.numpy(), x.numpy(), rid)
            assert np.array_equal(anc.numpy(), a_ref) and np.array_equal(x_out.numpy(), x_ref)
