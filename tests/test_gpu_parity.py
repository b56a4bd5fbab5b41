"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Ancestors and gathered state must be bit-exact (integer/index work and a
copy).  The bound B must be equal, except when the value before the ceiling
lies within 1e-9 (relative) of an integer, where the CPU and GPU sums may
round to different sides; then |B_gpu - B_cpu| <= 1.  The likelihood weight
(expf on the GPU, the oracle's exp in double rounded to float32) must agree
within |w_gpu - w_ref| <= (5 + 2|a|) 2^-23 w_ref + 2^-149, a = (x - y)^2 / 2:
the GPU's d = x - y and d d / 2 carry at most 3 binary32 roundings, which
exp turns into a relative error of 1.5 a 2^-23; expf adds at most 2 ulp and
the oracle's final rounding half an ulp; the last term covers subnormals.

Whole vectors are compared up to N = 2^20 (and at 2^22 and 2^24 for one
weight shape each, and at the 2^30 maximum with B = 3); the oracle splits
the particles over the host's cores
(its [i0, i1) entry, one contiguous range per task), which gives the same
array as its single-threaded run.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

mego = pytest.importorskip("paper_2109_13504_gb300")

DEV = torch.device("cuda:0")
VARIANTS = [mego.MEGOPOLIS, mego.METROPOLIS]


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _anc(w_h, B, seed, variant, cfg=None, sid=0, psize=0):
    w = _gpu(w_h)
    anc = torch.full((w_h.size,), -7, dtype=torch.int32, device=DEV)
    mego.mego_resample_gather(w, B, None, seed, sid, variant, psize, anc=anc, cfg=cfg)
    torch.cuda.synchronize()
    return anc.cpu().numpy()


def _b_equal(B_gpu, B_cpu, q):
    if B_gpu == B_cpu:
        return True
    near = abs(q - round(q)) <= 1e-9 * max(1.0, abs(q))
    return near and abs(B_gpu - B_cpu) <= 1


# ----------------------------------------------------------------------------
# Config: N = 4096, B = 32, seed 1, both variants, full bit-exact


@pytest.mark.parametrize("variant", VARIANTS)
def test_small_config_bit_exact(variant):
    w_h = synthetic.gaussian_weights(4096, 2.0, 1)
    ref = oracle.resample(w_h, 32, 1, variant)
    got = _anc(w_h, 32, 1, variant)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("path", [mego.PATH_GLOBAL, mego.PATH_SMEM])
@pytest.mark.parametrize("ppt", [1, 2, 4, 6, 8])
@pytest.mark.parametrize("threads", [64, 128, 256])
def test_launch_shape_invariance(variant, path, ppt, threads):
    n = 4096 + 1000 + 3
    w_h = synthetic.gaussian_weights(n, 3.0, 2)
    cfg = {"threads": threads, "ppt": ppt, "path": path}
    if ppt == 6 and (variant != mego.MEGOPOLIS or threads > 128):
        # six chains per thread: Megopolis only, in CTAs of at most 128 threads
        with pytest.raises(mego.MegoError) as ei:
            _anc(w_h, 45, 9, variant, cfg=cfg)
        assert ei.value.status == mego.MEGO_EINVAL
        return
    ref = oracle.resample(w_h, 45, 9, variant)
    got = _anc(w_h, 45, 9, variant, cfg=cfg)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 64, 100, 1000, 4097, 12345, 70001])
@pytest.mark.parametrize("B", [0, 1, 7, 33])
def test_ragged_sizes_bit_exact(variant, n, B):
    w_h = synthetic.gaussian_weights(n, 1.0, 3 + n)
    ref = oracle.resample(w_h, B, 5, variant)
    assert np.array_equal(_anc(w_h, B, 5, variant), ref)
    if n > 64:
        ref2 = oracle.resample(w_h, B, 5, variant, stream_id=3)
        assert np.array_equal(_anc(w_h, B, 5, variant, sid=3), ref2)


def test_equal_and_single_weight_cases():
    n = 5000
    w_h = np.full(n, 0.5, np.float32)
    for v in VARIANTS:
        assert np.array_equal(_anc(w_h, 9, 4, v), oracle.resample(w_h, 9, 4, v))
    w_h = np.zeros(n, np.float32)
    w_h[1234] = 1.0
    for v in VARIANTS:
        got = _anc(w_h, 2000, 4, v)
        assert got[1234] == 1234
        assert np.array_equal(got, oracle.resample(w_h, 2000, 4, v))


# ----------------------------------------------------------------------------
# Scaling sweep: N = 2^14..2^24, y = 0..4, 5 seeds, B from Eq. 3 at eps 0.01


def _sample_idx(n, rng, count=600):
    idx = set(range(min(n, 96)))
    idx.update(range(max(0, n - 96), n))
    idx.update(rng.integers(0, n, count).tolist())
    return np.array(sorted(idx), dtype=np.int64)


T = oracle.host_threads()


def _oracle_all(w_h, B, seed, variant, sid=0):
    return oracle.resample(w_h, B, seed, variant, stream_id=sid, threads=T)


@pytest.mark.parametrize("log2n", [14, 16, 18, 20, 22, 24])
def test_scaling_sweep(log2n):
    n = 1 << log2n
    rng = np.random.default_rng(log2n)
    ws = torch.empty(mego.workspace_bytes(n), dtype=torch.uint8, device=DEV)
    anc = torch.empty(n, dtype=torch.int32, device=DEV)
    for y in range(5):
        for dseed in range(1, 6):
            w_h = synthetic.gaussian_weights(n, y, dseed)
            w = _gpu(w_h)
            B_dev, status, q_dev = mego.mego_compute_B(w, 0.01, ws=ws)
            st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
            assert st == oracle.OK
            assert mego.mego_sync_status(status) == mego.MEGO_OK
            B_gpu = int(B_dev.item())
            assert _b_equal(B_gpu, B_cpu, q_cpu), (n, y, dseed, B_gpu, B_cpu, q_cpu)
            assert abs(float(q_dev.item()) - q_cpu) <= 1e-9 * max(1.0, q_cpu)
            # Every particle up to 2^20 (the benchmark's size); above it a
            # sample here, and whole vectors in test_whole_vector_above_2p20.
            full = n <= (1 << 20)
            idx = None if full else _sample_idx(n, rng)
            for v in VARIANTS:
                anc.fill_(-1)
                mego.mego_resample_gather(w, 0, B_dev, 100 + dseed, 0, v, anc=anc)
                got = anc.cpu().numpy()
                if full:
                    ref = _oracle_all(w_h, B_gpu, 100 + dseed, v)
                    assert np.array_equal(got, ref), (n, y, dseed, v)
                else:
                    ref = oracle.resample_at(w_h, B_gpu, 100 + dseed, idx, v)
                    assert np.array_equal(got[idx], ref), (n, y, dseed, v)
                    assert got.min() >= 0 and got.max() < n


@pytest.mark.parametrize("log2n,y", [(22, 4), (24, 2)])
def test_whole_vector_above_2p20(log2n, y):
    """Every particle at N = 2^22 with the most skewed weights (y = 4,
    B = 355) and at N = 2^24 with y = 2 (B = 16), both variants, B from the
    device bound."""
    n = 1 << log2n
    w_h = synthetic.gaussian_weights(n, y, 1)
    w = _gpu(w_h)
    B_dev, status, q_dev = mego.mego_compute_B(w, 0.01)
    st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
    assert mego.mego_sync_status(status) == mego.MEGO_OK
    B = int(B_dev.item())
    assert _b_equal(B, B_cpu, q_cpu)
    anc = torch.empty(n, dtype=torch.int32, device=DEV)
    for v in VARIANTS:
        anc.fill_(-1)
        mego.mego_resample_gather(w, 0, B_dev, 31, 0, v, anc=anc)
        got = anc.cpu().numpy()
        assert np.array_equal(got, _oracle_all(w_h, B, 31, v)), (n, y, v)
    del w, anc
    torch.cuda.empty_cache()


def test_maximum_size_whole_vector():
    """N = MEGO_N_MAX = 2^30 (4 GiB of weights), B = 3, both variants,
    every particle (the oracle on all host cores takes a few seconds)."""
    n = mego.N_MAX
    try:
        w = torch.empty(n, dtype=torch.float32, device=DEV)
        anc = torch.empty(n, dtype=torch.int32, device=DEV)
    except RuntimeError:
        pytest.skip("not enough device memory for N_MAX")
    w_h = synthetic.uniform_weights(n, 77)
    w.copy_(torch.from_numpy(w_h))
    for v in VARIANTS:
        anc.fill_(-1)
        mego.mego_resample_gather(w, 3, None, 11, 0, v, anc=anc)
        got = anc.cpu().numpy()
        assert np.array_equal(got, _oracle_all(w_h, 3, 11, v)), v
        del got
    del w, anc
    torch.cuda.empty_cache()


# ----------------------------------------------------------------------------
# Gather, device-side bound, likelihood


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", [777, 4096, 100003])
def test_gather_soa_and_aos4(variant, n):
    w_h = synthetic.gaussian_weights(n, 2.0, 4)
    x_h = synthetic.gaussian_state(n, 6, 5)
    ref = oracle.resample(w_h, 16, 3, variant)
    w = _gpu(w_h)
    # SoA with a row stride larger than n
    ld = n + 13
    x_pad = np.zeros((6, ld), np.float32)
    x_pad[:, :n] = x_h
    x_in = _gpu(x_pad)
    x_out = torch.full_like(x_in, -1.0)
    anc = torch.empty(n, dtype=torch.int32, device=DEV)
    mego.mego_resample_gather(w, 16, None, 3, 0, variant, x_in=x_in, x_out=x_out, anc=anc)
    out = x_out.cpu().numpy()
    assert np.array_equal(anc.cpu().numpy(), ref)
    assert np.array_equal(out[:, :n], oracle.gather_soa(x_h, ref))
    assert (out[:, n:] == -1.0).all()          # padding untouched
    # AoS4, ancestors not requested
    a_h = np.ascontiguousarray(x_h[:4].T)
    a_in = _gpu(a_h)
    a_out = torch.empty_like(a_in)
    mego.mego_resample_gather(w, 16, None, 3, 0, variant, x_in=a_in, x_out=a_out,
                              layout=mego.LAYOUT_AOS4)
    assert np.array_equal(a_out.cpu().numpy(), oracle.gather_aos4(a_h, ref))


def test_bound_workspace_reuse_garbage_and_graph_replay():
    """The bound writes one partial per CTA into the caller's workspace and
    folds them in a second launch.  A workspace full of arbitrary bytes,
    calls of different grid sizes on the same workspace, and replays of a
    captured graph whose input changes between replays must all give the
    oracle's B."""
    ws = torch.randint(0, 256, (mego.workspace_bytes(1 << 24),), dtype=torch.uint8,
                       device=DEV)
    cases = [((1 << 22) + 3, 2.0, 1), (5000, 4.0, 2), (1, 0.0, 3), ((1 << 22) + 3, 3.0, 4),
             (70_000, 1.0, 5)]
    for n, y, seed in cases:
        w_h = synthetic.gaussian_weights(n, y, seed)
        B_dev, status, q_dev = mego.mego_compute_B(_gpu(w_h), 0.01, ws=ws)
        st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
        assert mego.mego_sync_status(status) == mego.MEGO_OK
        assert _b_equal(int(B_dev.item()), B_cpu, q_cpu), (n, y)
        assert abs(float(q_dev.item()) - q_cpu) <= 1e-9 * max(1.0, q_cpu)
    n = 300_001
    w = torch.empty(n, dtype=torch.float32, device=DEV)
    B_dev = torch.empty(1, dtype=torch.int32, device=DEV)
    status = torch.empty(1, dtype=torch.int32, device=DEV)
    q_dev = torch.empty(1, dtype=torch.float64, device=DEV)
    side = torch.cuda.Stream(DEV)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        mego.mego_compute_B(w, 0.01, B_dev=B_dev, status=status, q=q_dev, ws=ws, stream=side)
    for y in (0.0, 4.0, 2.0, 2.0):
        w_h = synthetic.gaussian_weights(n, y, 7 + int(y))
        w.copy_(torch.from_numpy(w_h))
        g.replay()
        torch.cuda.synchronize()
        st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
        assert int(status.item()) == mego.MEGO_OK
        assert _b_equal(int(B_dev.item()), B_cpu, q_cpu), y


def test_device_bound_path_equals_host_path():
    n = 1 << 18
    w_h = synthetic.gaussian_weights(n, 3.0, 9)
    w = _gpu(w_h)
    B_dev, status, _ = mego.mego_compute_B(w, 0.01)
    a1 = torch.empty(n, dtype=torch.int32, device=DEV)
    mego.mego_resample_gather(w, 0, B_dev, 5, 0, mego.MEGOPOLIS, anc=a1)
    B = int(B_dev.item())
    a2 = mego.mego_resample(w, B, 5)
    assert torch.equal(a1, a2)
    assert torch.equal(mego.resample(w, None, 0.01, 5), a2)


@pytest.mark.parametrize("n", [(1 << 20), (1 << 20) + 5])
def test_likelihood_weights_and_fused_step(n):
    """The fused step at its full size: likelihood of state row 0 against
    y = 2, the bound, Megopolis and the gather of all six state rows, every
    particle compared."""
    x_h = synthetic.gaussian_state(n, 6, 12)
    x = _gpu(x_h)
    w, B_dev, status, q = mego.mego_likelihood_B(x[0], 2.0, 0.01)
    x_out = torch.full_like(x, -3.0)
    anc = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    mego.mego_resample_gather(w, 0, B_dev, 21, 0, mego.MEGOPOLIS, x_in=x, x_out=x_out,
                              anc=anc)
    assert mego.mego_sync_status(status) == mego.MEGO_OK
    w_gpu = w.cpu().numpy()
    ref = oracle.likelihood(x_h[0], 2.0).astype(np.float64)
    a = 0.5 * (x_h[0].astype(np.float64) - 2.0) ** 2
    tol = (5.0 + 2.0 * a) * 2.0 ** -23 * ref + 2.0 ** -149
    assert (np.abs(w_gpu.astype(np.float64) - ref) <= tol).all()
    # The bound and the ancestors are then exact functions of the GPU weights.
    st, B_cpu, q_cpu = oracle.compute_B(w_gpu, 0.01)
    assert _b_equal(int(B_dev.item()), B_cpu, q_cpu)
    B = int(B_dev.item())
    got = anc.cpu().numpy()
    ref_anc = _oracle_all(w_gpu, B, 21, mego.MEGOPOLIS)
    assert np.array_equal(got, ref_anc)
    assert np.array_equal(x_out.cpu().numpy(), oracle.gather_soa(x_h, ref_anc))


# ----------------------------------------------------------------------------
# Errors and status


def test_invalid_weights_report_status_and_write_nothing():
    n = 3000
    for bad in (np.nan, np.inf, -1.0):
        w_h = synthetic.gaussian_weights(n, 1.0, 2)
        w_h[17] = bad
        w = _gpu(w_h)
        B_dev, status, _ = mego.mego_compute_B(w, 0.01)
        anc = torch.full((n,), -5, dtype=torch.int32, device=DEV)
        mego.mego_resample_gather(w, 0, B_dev, 1, 0, mego.MEGOPOLIS, anc=anc)
        assert mego.mego_sync_status(status) == mego.MEGO_EWEIGHTS
        assert int(B_dev.item()) == -1
        assert (anc.cpu().numpy() == -5).all()
    w = torch.zeros(n, dtype=torch.float32, device=DEV)
    B_dev, status, _ = mego.mego_compute_B(w, 0.01)
    assert mego.mego_sync_status(status) == mego.MEGO_EWEIGHTS
    # a bound above its cap
    w_h = np.zeros(1 << 16, np.float32)
    w_h[0] = 1.0
    B_dev, status, _ = mego.mego_compute_B(_gpu(w_h), 0.01, b_max=100)
    assert mego.mego_sync_status(status) == mego.MEGO_EWEIGHTS


def test_argument_errors():
    w = torch.ones(100, dtype=torch.float32, device=DEV)
    anc = torch.empty(100, dtype=torch.int32, device=DEV)
    with pytest.raises(mego.MegoError):
        mego.mego_resample(w, -1, 1, anc=anc)
    with pytest.raises(mego.MegoError):
        mego.mego_resample_gather(w, 4, None, 1, 0, mego.METROPOLIS_C1, psize_bytes=12,
                                  anc=anc)   # 3 weights per partition does not divide 100
    with pytest.raises(mego.MegoError):
        mego.mego_resample_gather(w, 4, None, 1, 0, mego.MEGOPOLIS, anc=anc,
                                  cfg={"threads": 48})
    with pytest.raises(mego.MegoError):
        mego.mego_compute_B(w, 0.0)
    with pytest.raises(mego.MegoError):
        mego.mego_compute_B(w, 0.01, ws=torch.empty(16, dtype=torch.uint8, device=DEV))
    big = torch.ones(100_000, dtype=torch.float32, device=DEV)
    with pytest.raises(mego.MegoError):      # 400 KB does not fit shared memory
        mego.mego_resample_gather(big, 4, None, 1, 0, mego.MEGOPOLIS,
                                  anc=torch.empty(100_000, dtype=torch.int32, device=DEV),
                                  cfg={"path": mego.PATH_SMEM})


def test_sync_status_deadline():
    # A long resample and a zero deadline: the wait gives up, the stream
    # keeps running, and a later wait succeeds.
    n = 1 << 22
    w = torch.rand(n, dtype=torch.float32, device=DEV)
    anc = torch.empty(n, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    torch.cuda.synchronize()
    mego.mego_resample_gather(w, 4000, None, 1, 0, mego.METROPOLIS, anc=anc)
    with pytest.raises(mego.MegoError) as ei:
        mego.mego_sync_status(status, timeout_s=0.0)
    assert ei.value.status == mego.MEGO_ETIMEOUT
    assert mego.mego_sync_status(status, timeout_s=60.0) == mego.MEGO_OK


# ----------------------------------------------------------------------------
# End-to-end on host buffers, and Metropolis-C1/C2


def test_host_buffer_call_matches_device_call():
    n = 100_000
    w_h = synthetic.gaussian_weights(n, 2.0, 6)
    h_w = torch.from_numpy(w_h).pin_memory()
    h_anc = torch.empty(n, dtype=torch.int32).pin_memory()
    d_w = torch.empty(n, dtype=torch.float32, device=DEV)
    d_anc = torch.empty(n, dtype=torch.int32, device=DEV)
    d_sc = torch.empty(32, dtype=torch.uint8, device=DEV)
    ws = torch.empty(mego.workspace_bytes(n), dtype=torch.uint8, device=DEV)
    B = mego.mego_resample_host(h_w, -1, 0.01, 3, 0, mego.MEGOPOLIS, h_anc, d_w, d_anc, d_sc,
                                ws)
    st, B_cpu, q = oracle.compute_B(w_h, 0.01)
    assert _b_equal(B, B_cpu, q)
    assert np.array_equal(h_anc.numpy(), oracle.resample(w_h, B, 3, mego.MEGOPOLIS))
    B2 = mego.mego_resample_host(h_w, 7, 0.01, 3, 0, mego.METROPOLIS, h_anc, d_w, d_anc, d_sc,
                                 ws)
    assert B2 == 7
    assert np.array_equal(h_anc.numpy(), oracle.resample(w_h, 7, 3, mego.METROPOLIS))


@pytest.mark.parametrize("variant", [mego.METROPOLIS_C1, mego.METROPOLIS_C2])
@pytest.mark.parametrize("psize", [128, 512, 2048])
@pytest.mark.parametrize("ppt", [1, 2, 4, 8])
def test_partition_variants_bit_exact(variant, psize, ppt):
    n = 1 << 13
    w_h = synthetic.gaussian_weights(n, 2.0, 7)
    ref = oracle.resample(w_h, 37, 8, variant, psize_bytes=psize)
    got = _anc(w_h, 37, 8, variant, cfg={"ppt": ppt}, psize=psize)
    assert np.array_equal(got, ref)


def test_autotune_picks_a_shape_and_keeps_results_exact():
    n = 50_000
    w_h = synthetic.gaussian_weights(n, 3.0, 13)
    w = _gpu(w_h)
    cfg, ms = mego.mego_autotune(w, 60, mego.MEGOPOLIS)
    assert cfg["threads"] in (64, 128, 256) and cfg["ppt"] in (1, 2, 4, 6, 8)
    assert cfg["path"] in (mego.PATH_GLOBAL, mego.PATH_SMEM, mego.PATH_TMA) and ms > 0
    got = _anc(w_h, 60, 5, mego.MEGOPOLIS)            # no cfg: the tuned shape
    assert np.array_equal(got, oracle.resample(w_h, 60, 5, mego.MEGOPOLIS))
    for ppt in (1, 2, 4, 6, 8):
        got = _anc(w_h, 60, 5, mego.MEGOPOLIS, cfg={"ppt": ppt, "threads": 128})
        assert np.array_equal(got, oracle.resample(w_h, 60, 5, mego.MEGOPOLIS))


@pytest.mark.parametrize("ppt,threads", [(6, 128), (6, 64), (4, 256), (4, 128)])
@pytest.mark.parametrize("n", [64 * 6 + 5, 4096 * 3 + 17, 70001, 1 << 20])
def test_tma_window_path_bit_exact(ppt, threads, n):
    """The TMA window path (each warp's five windows of a group fetched by
    1-D tensor copies into shared memory; groups whose windows run past n
    load directly) gives the oracle's ancestors, with the tail group, B = 0,
    and ragged n; no window copy misses its wait."""
    w_h = synthetic.gaussian_weights(n, 3.0, 21)
    cfg = {"ppt": ppt, "threads": threads, "path": mego.PATH_TMA}
    for B in (0, 1, 7, 33, 61):
        got = _anc(w_h, B, 19, mego.MEGOPOLIS, cfg=cfg)
        assert np.array_equal(got, _oracle_all(w_h, B, 19, mego.MEGOPOLIS)), (n, B)
    assert mego.mego_device_fault() == 0


def test_tma_window_path_arguments():
    w = torch.ones(4096, dtype=torch.float32, device=DEV)
    anc = torch.empty(4096, dtype=torch.int32, device=DEV)
    for variant, ppt in ((mego.METROPOLIS, 6), (mego.MEGOPOLIS, 2)):
        with pytest.raises(mego.MegoError) as ei:
            mego.mego_resample_gather(w, 4, None, 1, 0, variant, anc=anc,
                                      cfg={"ppt": ppt, "path": mego.PATH_TMA})
        assert ei.value.status == mego.MEGO_EINVAL
    with pytest.raises(mego.MegoError):          # fewer than 64 x ppt weights
        mego.mego_resample_gather(w[:300], 4, None, 1, 0, mego.MEGOPOLIS, anc=anc[:300],
                                  cfg={"ppt": 6, "path": mego.PATH_TMA})
    with pytest.raises(mego.MegoError):          # a window copy needs 16-byte alignment
        mego.mego_resample_gather(w[1:], 4, None, 1, 0, mego.MEGOPOLIS, anc=anc[1:],
                                  cfg={"ppt": 6, "path": mego.PATH_TMA})


def test_no_device_faults_after_the_shared_memory_path():
    n = 9000
    w_h = synthetic.gaussian_weights(n, 2.0, 3)
    for v in VARIANTS:
        _anc(w_h, 10, 1, v, cfg={"path": mego.PATH_SMEM})
    assert mego.mego_device_fault() == 0


def test_shared_memory_staging_wait_runs_out_and_reports():
    # A zero poll budget makes the staging wait give up at once: the CTAs
    # record fault 1 and write nothing (each still waits for its own bulk
    # copy to land before it leaves).  The next call with the default budget
    # is exact and reports no fault.
    n = 9000                       # 36000 bytes: the bulk-copy branch
    w_h = synthetic.gaussian_weights(n, 2.0, 3)
    w = _gpu(w_h)
    assert mego.mego_device_fault() == 0
    for v in VARIANTS:
        anc = torch.full((n,), -7, dtype=torch.int32, device=DEV)
        mego.mego_set_stage_poll_budget(0)
        try:
            mego.mego_resample_gather(w, 10, None, 1, 0, v, anc=anc,
                                      cfg={"path": mego.PATH_SMEM})
            torch.cuda.synchronize()
        finally:
            mego.mego_set_stage_poll_budget(-1)
        assert mego.mego_device_fault() == 1
        assert (anc.cpu().numpy() == -7).all()
        assert np.array_equal(_anc(w_h, 10, 1, v, cfg={"path": mego.PATH_SMEM}),
                              oracle.resample(w_h, 10, 1, v))
        assert mego.mego_device_fault() == 0
    with pytest.raises(mego.MegoError):
        mego.mego_set_stage_poll_budget(1 << 40)


@pytest.mark.parametrize("alpha", [0.5, 2.0, 3.0, 10.0, 50.0])
def test_gamma_weights_bit_exact(alpha):
    """The paper's second weight generator (Eq. 13, Appendix A): gamma
    weights with rate 1, both variants, B from the bound."""
    for n in (40_000, 1 << 18):
        w_h = synthetic.gamma_weights(n, alpha, 3)
        w = _gpu(w_h)
        B_dev, status, _ = mego.mego_compute_B(w, 0.01)
        st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
        assert _b_equal(int(B_dev.item()), B_cpu, q_cpu)
        B = int(B_dev.item())
        for v in VARIANTS:
            anc = torch.empty(n, dtype=torch.int32, device=DEV)
            mego.mego_resample_gather(w, 0, B_dev, 17, 0, v, anc=anc)
            got = anc.cpu().numpy()
            assert np.array_equal(got, _oracle_all(w_h, B, 17, v)), (alpha, n, v)


def test_huge_weights_are_reported_not_mistaken():
    """Finite weights so large that a 4096-weight chunk's sum leaves the
    binary32 range cannot give B on the device: the bound reports
    MEGO_EWEIGHTS (and the resample writes nothing) instead of a wrong B;
    large weights below that limit still match the oracle."""
    n = 3 * 4096 + 5
    w_h = np.full(n, 1e36, dtype=np.float32)
    B_dev, status, _ = mego.mego_compute_B(_gpu(w_h), 0.01)
    assert int(status.item()) == mego.MEGO_EWEIGHTS and int(B_dev.item()) == -1
    w_h = (synthetic.gaussian_weights(n, 2.0, 5) * np.float32(1e30)).astype(np.float32)
    B_dev, status, q_dev = mego.mego_compute_B(_gpu(w_h), 0.01)
    st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
    assert int(status.item()) == mego.MEGO_OK and _b_equal(int(B_dev.item()), B_cpu, q_cpu)
    assert abs(float(q_dev.item()) - q_cpu) <= 1e-9 * max(1.0, q_cpu)


def _mixed_tiny_weights(n, seed):
    """Weights with signed zeros and subnormals among ordinary ones: R6's test
    fl(u w_k) <= w_j must then run without flush-to-zero on both sides (a
    subnormal product or weight flushed to 0 changes the comparison)."""
    rng = np.random.default_rng(seed)
    w = synthetic.gaussian_weights(n, 2.0, seed).copy()
    kind = rng.integers(0, 10, n)
    sub = rng.integers(1, 1 << 23, n, dtype=np.uint32).view(np.float32)
    w[kind < 3] = sub[kind < 3]                       # 30 % subnormal
    w[kind == 3] = np.float32(-0.0)
    w[kind == 4] = np.float32(0.0)
    w[kind == 5] *= np.float32(2.0 ** -120)           # tiny normal: products go subnormal
    return w


@pytest.mark.parametrize("variant", VARIANTS)
def test_subnormal_and_signed_zero_weights_bit_exact(variant):
    n = 2 * 4096 + 77
    w_h = _mixed_tiny_weights(n, 21)
    assert np.any(np.signbit(w_h) & (w_h == 0)) and np.any((w_h > 0) & (w_h < 2.0 ** -126))
    st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
    B_dev, status, q_dev = mego.mego_compute_B(_gpu(w_h), 0.01)
    assert st == oracle.OK and int(status.item()) == mego.MEGO_OK
    assert _b_equal(int(B_dev.item()), B_cpu, q_cpu)
    assert abs(float(q_dev.item()) - q_cpu) <= 1e-9 * max(1.0, q_cpu)
    for B in (40, B_cpu):
        ref = oracle.resample(w_h, B, 3, variant)
        paths = [mego.PATH_GLOBAL, mego.PATH_SMEM] + \
            ([mego.PATH_TMA] if variant == mego.MEGOPOLIS else [])
        for path in paths:
            cfg = {"path": path, "ppt": 4, "threads": 128}
            assert np.array_equal(_anc(w_h, B, 3, variant, cfg=cfg), ref), (B, path)
    # An all-subnormal vector: valid weights, and every product u w_k is subnormal.
    w_h = np.random.default_rng(5).integers(1, 1 << 23, n, dtype=np.uint32).view(np.float32)
    st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
    B_dev, status, _ = mego.mego_compute_B(_gpu(w_h), 0.01)
    assert st == oracle.OK and int(status.item()) == mego.MEGO_OK
    assert _b_equal(int(B_dev.item()), B_cpu, q_cpu)
    assert np.array_equal(_anc(w_h, B_cpu, 4, variant), oracle.resample(w_h, B_cpu, 4, variant))


@pytest.mark.parametrize("variant,psize", [(mego.METROPOLIS_C1, 128), (mego.METROPOLIS_C2, 512)])
def test_subnormal_weights_partition_variants_bit_exact(variant, psize):
    n = 8192
    w_h = _mixed_tiny_weights(n, 22)
    for B in (1, 33):
        ref = oracle.resample(w_h, B, 6, variant, psize_bytes=psize)
        assert np.array_equal(_anc(w_h, B, 6, variant, psize=psize), ref), B


def test_subnormal_weights_in_a_batch():
    sizes = (3000, 8192 + 5)
    ws_h = [_mixed_tiny_weights(m, 30 + k) for k, m in enumerate(sizes)]
    ancs = [torch.full((m,), -1, dtype=torch.int32, device=DEV) for m in sizes]
    b = mego.Batch([{"w": _gpu(w_h), "anc": a, "B": -1, "stream_id": k}
                    for k, (w_h, a) in enumerate(zip(ws_h, ancs))], seed=8)
    b.bound(0.01)
    b.resample()
    torch.cuda.synchronize()
    Bs = b.B.cpu().numpy().tolist()
    for k, (w_h, a) in enumerate(zip(ws_h, ancs)):
        st, B_cpu, q_cpu = oracle.compute_B(w_h, 0.01)
        assert st == oracle.OK and _b_equal(Bs[k], B_cpu, q_cpu)
        ref = oracle.resample(w_h, Bs[k], 8, mego.MEGOPOLIS, stream_id=k)
        assert np.array_equal(a.cpu().numpy(), ref), k
    b.close()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,B", [(5, mego.B_MAX), (1000, 100003), (4096 + 33, 30031)])
def test_long_chains_up_to_the_B_cap(variant, n, B):
    """Chains of up to MEGO_B_MAX iterations: the offset counter, the group
    counter of the u draws and the table refills run through their whole
    range; compared with the oracle on every particle."""
    w_h = synthetic.gaussian_weights(n, 3.0, n)
    ref = oracle.resample(w_h, B, 12, variant, threads=oracle.host_threads())
    assert np.array_equal(_anc(w_h, B, 12, variant), ref)


@pytest.mark.parametrize("variant", VARIANTS + [mego.METROPOLIS_C1, mego.METROPOLIS_C2])
def test_extreme_seeds_and_stream_ids(variant):
    """The key is (lo32(seed), hi32(seed)) and the stream id is a counter
    word: seeds and stream ids at the ends of their ranges give the oracle's
    ancestors too."""
    n = 4096
    w_h = synthetic.gaussian_weights(n, 2.5, 77)
    psize = 256 if variant in (mego.METROPOLIS_C1, mego.METROPOLIS_C2) else 0
    for seed in (0, 1, 0xFFFFFFFF, 1 << 32, 0x8000000000000000, 0xFFFFFFFFFFFFFFFF):
        for sid in (0, 0x7FFFFFFF, 0xFFFFFFFF):
            ref = oracle.resample(w_h, 21, seed, variant, stream_id=sid, psize_bytes=psize)
            got = _anc(w_h, 21, seed, variant, sid=sid, psize=psize)
            assert np.array_equal(got, ref), (hex(seed), hex(sid))
