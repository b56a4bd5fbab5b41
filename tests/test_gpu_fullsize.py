"""The benchmark's own plan against the oracle, every particle.

The timed step of the benchmark resamples five N = 2^20 weight vectors
(x ~ N(0,1), w = exp(-(x - y)^2 / 2), y = 0..4, Eq. 12's shape) as one
batch: the batched bound (Eq. 3 at eps = 0.01) and one persistent Megopolis
launch (Algorithm 5), autotuned, captured in a CUDA graph and replayed on a
side stream.  This test builds that plan the same way and compares all
5 x 2^20 ancestors of the replay with the CPU oracle (and the bound with the
oracle's), for the default launch shape, the autotuned one and the graph
replay; the Metropolis batch (Algorithm 2) the benchmark times beside it is
checked the same way.  The oracle splits each vector over the host's cores.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

mego = pytest.importorskip("paper_2109_13504_gb300")

DEV = torch.device("cuda:0")
N = 1 << 20
YS = (0, 1, 2, 3, 4)
EPS = 0.01
SEED = 1
T = oracle.host_threads()


def _b_equal(B_gpu, B_cpu, q):
    return B_gpu == B_cpu or (abs(q - round(q)) <= 1e-9 * max(1.0, abs(q))
                              and abs(B_gpu - B_cpu) <= 1)


@pytest.fixture(scope="module")
def weights():
    ws_h = [synthetic.gaussian_weights(N, y, SEED + y) for y in YS]
    refs = [oracle.compute_B(w_h, EPS) for w_h in ws_h]
    return ws_h, refs


@pytest.mark.parametrize("variant", [mego.MEGOPOLIS, mego.METROPOLIS])
def test_bench_plan_every_particle(weights, variant):
    ws_h, refs = weights
    side = torch.cuda.Stream(DEV)
    w_dev = [torch.from_numpy(w_h).to(DEV) for w_h in ws_h]
    anc = [torch.full((N,), -1, dtype=torch.int32, device=DEV) for _ in YS]
    filters = [{"w": w_dev[t], "anc": anc[t], "B": -1, "stream_id": 0}
               for t in range(len(YS))]
    with torch.cuda.stream(side):
        b = mego.Batch(filters, variant=variant, seed=SEED, stream=side)
        b.bound(EPS, stream=side)
        b.resample(stream=side)
    side.synchronize()
    Bs = b.B.cpu().numpy().tolist()
    assert b.status.cpu().numpy().tolist() == [mego.MEGO_OK] * len(YS)
    expected = []
    for t, y in enumerate(YS):
        st, B_ref, q_ref = refs[t]
        assert st == oracle.OK
        assert _b_equal(Bs[t], B_ref, q_ref), (y, Bs[t], B_ref, q_ref)
        expected.append(oracle.resample(ws_h[t], Bs[t], SEED, variant, threads=T))
    shapes = [dict(b.shape)]
    for t in range(len(YS)):                  # default launch shape
        assert np.array_equal(anc[t].cpu().numpy(), expected[t]), ("default", YS[t])
    with torch.cuda.stream(side):
        b.autotune(reps=1, stream=side)
        b.capture(EPS, stream=side)
        for a in anc:
            a.fill_(-1)
        b.replay(stream=side)
        b.replay(stream=side)                 # the queue resets itself between replays
    side.synchronize()
    shapes.append(dict(b.shape))
    for t in range(len(YS)):                  # autotuned shape, graph replay
        assert np.array_equal(anc[t].cpu().numpy(), expected[t]), (shapes, YS[t])
    assert b.B.cpu().numpy().tolist() == Bs
    b.close()
