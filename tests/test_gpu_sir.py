"""The SIR filter stages on the GPU against the oracle: predict bit-exact
(binary32, same operation order), weights within 2 ulp (expf), then one full
filter step (predict, Megopolis with the gather, mean) exact from the GPU
weights; and an end-to-end run whose error stays bounded."""
import math

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

mego = pytest.importorskip("paper_2109_13504_gb300")
DEV = torch.device("cuda:0")


def test_predict_update_and_one_filter_step():
    n = (1 << 16) + 3
    x_h = synthetic.sir_initial_particles(n, 1) * np.float32(6.0)
    v_h = synthetic.sir_process_noise(n, 1, 2)[0]
    drift = float(np.float32(8 * math.cos(1.2 * 3)))
    z = 7.25
    x, v = torch.from_numpy(x_h).to(DEV), torch.from_numpy(v_h).to(DEV)
    xp, w = mego.mego_sir_predict_update(x, v, drift, z)
    xp_ref, w_ref = oracle.sir_predict_update(x_h, v_h, drift, z)
    xp_h, w_h = xp.cpu().numpy(), w.cpu().numpy()
    assert np.array_equal(xp_h, xp_ref)
    ulp = np.spacing(np.maximum(w_ref, np.float32(1e-38)))
    assert (np.abs(w_h.astype(np.float64) - w_ref) <= 2 * ulp + 2.0 ** -149).all()
    # resample with the gather of the 1-dim state, then the estimate
    x_new = torch.empty((1, n), dtype=torch.float32, device=DEV)
    anc = torch.empty(n, dtype=torch.int32, device=DEV)
    mego.mego_resample_gather(w, 32, None, 9, 3, mego.MEGOPOLIS, x_in=xp.view(1, n),
                              x_out=x_new, anc=anc)
    est = mego.mego_mean(x_new.view(-1))
    a_ref = oracle.resample(w_h, 32, 9, mego.MEGOPOLIS, stream_id=3)
    assert np.array_equal(anc.cpu().numpy(), a_ref)
    assert np.array_equal(x_new.cpu().numpy()[0], xp_h[a_ref])
    m_ref = oracle.mean(xp_h[a_ref])
    assert abs(float(est.item()) - m_ref) <= 1e-12 * max(1.0, abs(m_ref))


def test_filter_tracks_the_truth():
    n, T = 1 << 16, 60
    xt, zt = synthetic.sir_truth(T, 11)
    sq = []
    for run in range(2):
        x = torch.from_numpy(synthetic.sir_initial_particles(n, 20 + run)).to(DEV)
        noise = synthetic.sir_process_noise(n, T, 30 + run, device=DEV)
        xs = torch.empty((1, n), dtype=torch.float32, device=DEV)
        est = torch.empty(T + 1, dtype=torch.float64, device=DEV)
        for t in range(1, T + 1):
            xp, w = mego.mego_sir_predict_update(x, noise[t - 1], 8 * math.cos(1.2 * t), zt[t])
            mego.mego_resample_gather(w, 32, None, 100 + run, t, mego.MEGOPOLIS,
                                      x_in=xp.view(1, n), x_out=xs)
            mego.mego_mean(xs.view(-1), out=est[t:t + 1])
            x = xs.view(-1).clone()
        sq.append((est.cpu().numpy()[1:] - xt[1:]) ** 2)
    rmse = float(np.mean(np.sqrt(np.mean(sq, axis=0))))
    # The model's posterior is bimodal (z sees x^2), so the error stays a few units;
    # a broken filter drifts to tens.
    assert rmse < 8.0, rmse
