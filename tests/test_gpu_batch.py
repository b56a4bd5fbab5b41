"""Batched resampling (many filters, one persistent launch) against single
resamples and the oracle.  Each filter's ancestors must equal, bit for bit,
those of mego_resample_gather with the same seed, stream id and B -- alone or
in the batch -- and the per-filter bound must equal the oracle's (near-integer
rule as in test_gpu_parity)."""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

mego = pytest.importorskip("paper_2109_13504_gb300")
DEV = torch.device("cuda:0")
SEED = 77


def _b_equal(B_gpu, B_cpu, q):
    return B_gpu == B_cpu or (abs(q - round(q)) <= 1e-9 * max(1.0, abs(q))
                              and abs(B_gpu - B_cpu) <= 1)


def _make(count, seed, lo=5.0, hi=14.0, sizes=None):
    ns, ys = synthetic.filter_sizes(count, lo, hi, seed)
    if sizes is not None:
        ns = np.array(sizes, dtype=np.int64)
        ys = ys[: len(ns)]
    ws = [synthetic.gaussian_weights(int(n), float(y), 1000 + f) for f, (n, y) in enumerate(zip(ns, ys))]
    return ws


@pytest.mark.parametrize("variant", [mego.MEGOPOLIS, mego.METROPOLIS])
def test_batch_matches_single_resamples_and_oracle(variant):
    ws = _make(40, 3, sizes=[1, 2, 31, 32, 33, 100, 127, 128, 129, 4097] + [0] * 0) + _make(30, 4)
    filters = []
    for f, w_h in enumerate(ws):
        w = torch.from_numpy(w_h).to(DEV)
        fixed = (f % 3 == 0)
        filters.append({"w": w, "anc": torch.full((w_h.size,), -3, dtype=torch.int32, device=DEV),
                        "B": (f % 17) if fixed else -1, "stream_id": 500 + f})
    batch = mego.Batch(filters, variant=variant, seed=SEED)
    batch.bound(0.01)
    batch.resample()
    torch.cuda.synchronize()
    Bb = batch.B.cpu().numpy()
    st = batch.status.cpu().numpy()
    q = batch.q.cpu().numpy()
    for f, (d, w_h) in enumerate(zip(filters, ws)):
        assert st[f] == mego.MEGO_OK
        s_ref, B_ref, q_ref = oracle.compute_B(w_h, 0.01)
        assert _b_equal(int(Bb[f]), B_ref, q_ref), (f, Bb[f], B_ref)
        B = d["B"] if d["B"] >= 0 else int(Bb[f])
        got = d["anc"].cpu().numpy()
        alone = mego.mego_resample_gather(d["w"], B, None, SEED, d["stream_id"], variant,
                                          anc=torch.empty_like(d["anc"]))[0].cpu().numpy()
        assert np.array_equal(got, alone), f
        if w_h.size <= 5000:
            assert np.array_equal(got, oracle.resample(w_h, B, SEED, variant,
                                                       stream_id=d["stream_id"])), f


def test_batch_graph_replay_and_shapes_and_autotune():
    ws = _make(64, 9, 6.0, 13.0)
    filters = [{"w": torch.from_numpy(w_h).to(DEV),
                "anc": torch.empty(w_h.size, dtype=torch.int32, device=DEV),
                "B": -1, "stream_id": f} for f, w_h in enumerate(ws)]
    batch = mego.Batch(filters, seed=5)
    batch.bound(0.01)
    batch.resample()
    torch.cuda.synchronize()
    ref = [d["anc"].clone() for d in filters]
    assert batch.shape["ppt"] == 4        # small filters: items of 4, four chains per thread
    for threads, ppt in [(64, 1), (128, 2), (256, 4), (64, 6), (128, 6)]:
        batch.set_shape(threads, ppt)
        for d in filters:
            d["anc"].fill_(-1)
        batch.resample()
        torch.cuda.synchronize()
        assert all(torch.equal(a, d["anc"]) for a, d in zip(ref, filters))
    with pytest.raises(mego.MegoError):      # six per thread needs CTAs of <= 128
        batch.set_shape(256, 6)
    ms = batch.autotune(reps=2)
    assert ms > 0 and batch.shape["threads"] in (64, 128, 256)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        batch.capture(0.01, stream=side)
        for _ in range(3):                 # the work queue resets itself between launches
            for d in filters:
                d["anc"].fill_(-1)
            before = mego.launch_count()
            batch.replay(stream=side)
            assert mego.launch_count() - before == 3     # bound (2) + resample (1)
            side.synchronize()
            assert all(torch.equal(a, d["anc"]) for a, d in zip(ref, filters))
    batch.close()


@pytest.mark.parametrize("layout", [mego.LAYOUT_SOA, mego.LAYOUT_AOS4])
def test_batch_gather(layout):
    ws = _make(12, 11, 7.0, 12.0)
    filters = []
    for f, w_h in enumerate(ws):
        n = w_h.size
        if layout == mego.LAYOUT_SOA:
            x = torch.from_numpy(synthetic.gaussian_state(n, 3, f)).to(DEV)
        else:
            x = torch.from_numpy(np.ascontiguousarray(synthetic.gaussian_state(n, 4, f).T)).to(DEV)
        filters.append({"w": torch.from_numpy(w_h).to(DEV), "x_in": x,
                        "x_out": torch.empty_like(x),
                        "anc": torch.empty(n, dtype=torch.int32, device=DEV),
                        "B": 20 + f, "stream_id": 7 * f})
    batch = mego.Batch(filters, layout=layout, seed=SEED)
    batch.resample()
    torch.cuda.synchronize()
    for f, d in enumerate(filters):
        ref = oracle.resample(ws[f], d["B"], SEED, mego.MEGOPOLIS, stream_id=d["stream_id"])
        assert np.array_equal(d["anc"].cpu().numpy(), ref)
        xi = d["x_in"].cpu().numpy()
        want = oracle.gather_soa(xi, ref) if layout == mego.LAYOUT_SOA else oracle.gather_aos4(xi, ref)
        assert np.array_equal(d["x_out"].cpu().numpy(), want)


def test_batch_bad_filter_is_isolated():
    ws = _make(6, 2, 8.0, 10.0)
    ws[2] = ws[2].copy()
    ws[2][5] = np.nan
    filters = [{"w": torch.from_numpy(w_h).to(DEV),
                "anc": torch.full((w_h.size,), -9, dtype=torch.int32, device=DEV),
                "B": -1, "stream_id": f} for f, w_h in enumerate(ws)]
    batch = mego.Batch(filters, seed=1)
    batch.bound(0.01)
    batch.resample()
    torch.cuda.synchronize()
    st = batch.status.cpu().numpy()
    assert st[2] == mego.MEGO_EWEIGHTS and int(batch.B[2].item()) == -1
    assert (filters[2]["anc"].cpu().numpy() == -9).all()
    for f in (0, 1, 3, 4, 5):
        assert st[f] == mego.MEGO_OK and (filters[f]["anc"].cpu().numpy() >= 0).all()


def test_host_weights_and_host_ancestors_in_place():
    """Filters whose weights sit in page-locked host memory (w_host: the bound
    reads them over the CPU-GPU link and writes the device copy w) and whose
    ancestors go straight to page-locked host memory give the same B, the
    same device copy and the same ancestors as the all-device batch."""
    ws = _make(12, 9, sizes=[1, 33, 4096, 4097, 70000, 1 << 20]) + _make(6, 10)
    dev_f, host_f = [], []
    for f, w_h in enumerate(ws):
        n = w_h.size
        dev_f.append({"w": torch.from_numpy(w_h).to(DEV),
                      "anc": torch.empty(n, dtype=torch.int32, device=DEV),
                      "B": 9 if f == 2 else -1, "stream_id": 40 + f})
        host_f.append({"w": torch.full((n,), float("nan"), dtype=torch.float32, device=DEV),
                       "w_host": torch.from_numpy(w_h).pin_memory(),
                       "anc": torch.full((n,), -5, dtype=torch.int32).pin_memory(),
                       "B": 9 if f == 2 else -1, "stream_id": 40 + f})
    ref = mego.Batch(dev_f, seed=SEED)
    ref.bound(0.01)
    ref.resample()
    got = mego.Batch(host_f, seed=SEED)
    for _ in range(2):                       # the plan replays the same way
        got.bound(0.01)
        got.resample()
        torch.cuda.synchronize()
        assert np.array_equal(got.B.cpu().numpy(), ref.B.cpu().numpy())
        for d, h in zip(dev_f, host_f):
            assert torch.equal(h["w"], d["w"])
            assert np.array_equal(h["anc"].numpy(), d["anc"].cpu().numpy())
        for h in host_f:
            h["anc"].fill_(-5)
            h["w"].fill_(float("nan"))
    with pytest.raises(TypeError):           # w_host must be page-locked
        mego.Batch([{"w": dev_f[0]["w"], "w_host": torch.from_numpy(ws[0]),
                     "anc": dev_f[0]["anc"]}], seed=SEED)


def test_large_filters_take_six_chains_per_thread():
    """A batch dominated by filters of >= 2^17 particles is planned with items
    of six segments and six chains per thread; every shape (including ones
    that leave part of an item's batch empty) gives the same ancestors."""
    ws = _make(3, 12, sizes=[1 << 18, (1 << 17) + 33, 5000])
    filters = [{"w": torch.from_numpy(w_h).to(DEV),
                "anc": torch.empty(w_h.size, dtype=torch.int32, device=DEV),
                "B": -1, "stream_id": 70 + f} for f, w_h in enumerate(ws)]
    batch = mego.Batch(filters, seed=SEED)
    assert batch.shape["ppt"] == 6 and batch.shape["threads"] == 128
    batch.bound(0.01)
    batch.resample()
    torch.cuda.synchronize()
    ref = [d["anc"].clone() for d in filters]
    Bb = batch.B.cpu().numpy()
    for f, d in enumerate(filters):
        alone = mego.mego_resample_gather(d["w"], int(Bb[f]), None, SEED, d["stream_id"],
                                          mego.MEGOPOLIS, anc=torch.empty_like(d["anc"]))[0]
        assert torch.equal(alone, ref[f]), f
    for threads, ppt in [(64, 6), (256, 4), (128, 2), (64, 1)]:
        batch.set_shape(threads, ppt)
        for d in filters:
            d["anc"].fill_(-1)
        batch.resample()
        torch.cuda.synchronize()
        assert all(torch.equal(a, d["anc"]) for a, d in zip(ref, filters)), (threads, ppt)


@pytest.mark.parametrize("heavy_at", [0, 3, 6])
def test_heaviest_filter_first_keeps_every_result(heavy_at):
    """The queue hands the most expensive filter's work items out first; with
    that filter first, in the middle or last in the plan (fixed B, so the
    plan already knows it, then again after a bound), every filter's
    ancestors still equal its single resample."""
    ws = _make(7, 21, sizes=[300, 4097, 1000, 20000, 64, 9000, 33])
    Bs = [5, 3, 7, 2, 9, 4, 6]
    Bs[heavy_at] = 200
    filters = [{"w": torch.from_numpy(w_h).to(DEV),
                "anc": torch.empty(w_h.size, dtype=torch.int32, device=DEV),
                "B": Bs[f], "stream_id": 90 + f} for f, w_h in enumerate(ws)]
    batch = mego.Batch(filters, seed=SEED)
    for with_bound in (False, True):
        for d in filters:
            d["anc"].fill_(-1)
        if with_bound:
            batch.bound(0.01)
        batch.resample()
        torch.cuda.synchronize()
        for f, d in enumerate(filters):
            alone = mego.mego_resample_gather(d["w"], Bs[f], None, SEED, d["stream_id"],
                                              mego.MEGOPOLIS,
                                              anc=torch.empty_like(d["anc"]))[0]
            assert torch.equal(alone, d["anc"]), (heavy_at, with_bound, f)


@pytest.mark.parametrize("variant", [mego.MEGOPOLIS, mego.METROPOLIS])
def test_shared_memory_phase_matches_the_oracle(variant):
    """Filters at or below the shared-memory threshold are resampled whole
    by one CTA each from shared memory (their weights staged by bulk copy,
    the ragged tail by plain loads), the rest by the warp-level queue.  Every
    threshold, the autotuned one and a graph replay give the oracle's
    ancestors, with fixed and bound-computed B."""
    sizes = [1, 3, 31, 33, 100, 1001, 4095, 4096, 4097, 5003, 16384, 20001, 49152, 70001]
    ws = [synthetic.gaussian_weights(n, (k % 5) * 0.9, 4000 + k) for k, n in enumerate(sizes)]
    filters = [{"w": torch.from_numpy(w_h).to(DEV),
                "anc": torch.full((w_h.size,), -1, dtype=torch.int32, device=DEV),
                "B": (7 + k) if k % 4 == 1 else -1, "stream_id": 90 + k}
               for k, w_h in enumerate(ws)]
    batch = mego.Batch(filters, variant=variant, seed=SEED)
    batch.bound(0.01)
    batch.resample()
    torch.cuda.synchronize()
    Bs = batch.B.cpu().numpy()
    refs = []
    for k, (d, w_h) in enumerate(zip(filters, ws)):
        B = d["B"] if d["B"] >= 0 else int(Bs[k])
        ref = oracle.resample(w_h, B, SEED, variant, stream_id=d["stream_id"])
        assert np.array_equal(d["anc"].cpu().numpy(), ref), ("global", k)
        refs.append(ref)

    def check(tag):
        for k, d in enumerate(filters):
            assert np.array_equal(d["anc"].cpu().numpy(), refs[k]), (tag, sizes[k])

    for thr in (4096, 16384, 49152):
        batch.set_smem(thr)
        assert batch.shape["smem_filters"] == sum(n <= thr for n in sizes)
        for d in filters:
            d["anc"].fill_(-1)
        batch.resample()
        torch.cuda.synchronize()
        check(thr)
    assert (batch.B.cpu().numpy() == Bs).all()          # a re-plan keeps the bound's B
    batch.set_smem(0)
    batch.set_smem(16384)
    batch.autotune(reps=1)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        batch.capture(0.01, stream=side)
        for _ in range(2):
            for d in filters:
                d["anc"].fill_(-1)
            batch.replay(stream=side)
        side.synchronize()
    check("autotuned %s" % batch.shape)
    with pytest.raises(mego.MegoError):                # a captured graph pins the plan
        batch.set_smem(4096)
    batch.close()
    with pytest.raises(mego.MegoError):                # beyond the shared memory per CTA
        mego.Batch(filters, variant=variant, seed=SEED).set_smem(1 << 20)


def test_shared_memory_phase_with_aos4_gather():
    sizes = [777, 4096, 9001, 30000]
    ws = [synthetic.gaussian_weights(n, 2.0, 50 + k) for k, n in enumerate(sizes)]
    filters = []
    for k, w_h in enumerate(ws):
        x = torch.from_numpy(np.ascontiguousarray(synthetic.gaussian_state(w_h.size, 4, k).T)).to(DEV)
        filters.append({"w": torch.from_numpy(w_h).to(DEV), "x_in": x,
                        "x_out": torch.empty_like(x), "B": 25 + k, "stream_id": 3 * k})
    batch = mego.Batch(filters, layout=mego.LAYOUT_AOS4, seed=SEED)
    batch.set_smem(16384)
    assert batch.shape["smem_filters"] == 3
    batch.resample()
    torch.cuda.synchronize()
    for k, d in enumerate(filters):
        ref = oracle.resample(ws[k], d["B"], SEED, mego.MEGOPOLIS, stream_id=d["stream_id"])
        assert np.array_equal(d["x_out"].cpu().numpy(),
                              oracle.gather_aos4(d["x_in"].cpu().numpy(), ref)), sizes[k]
