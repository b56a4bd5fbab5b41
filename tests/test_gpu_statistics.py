"""Resampling quality of the CUDA path against the paper's printed tables:
MSE/N of offspring counts (Section 5.1) for Megopolis and Metropolis
(Tables 3-4) at N = 2^15..2^20 and for Metropolis-C1/C2 (Tables 5-6), K runs
per weight sequence, within 4 standard errors plus a small model margin.
Also Megopolis' smaller variance than Metropolis (Section 6.1) and the
offspring bound B + 1 with 32 | N."""
import json
import os

import numpy as np
import pytest
import torch

import synthetic
from oracle.stats import offspring_stats

pytestmark = pytest.mark.gpu

mego = pytest.importorskip("paper_2109_13504_gb300")
DEV = torch.device("cuda:0")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_mse_tables.json")


@pytest.fixture(scope="module")
def paper():
    with open(GOLDEN) as f:
        return json.load(f)


def _mse_runs(n, y, variant, K, wseeds, psize=0):
    vals, maxoff = [], 0
    for ws in wseeds:
        w_h = synthetic.gaussian_weights(n, y, ws)
        w = torch.from_numpy(w_h).to(DEV)
        B_dev, _, _ = mego.mego_compute_B(w, 0.01)
        B = int(B_dev.item())
        anc = torch.empty(n, dtype=torch.int32, device=DEV)
        for k in range(K):
            mego.mego_resample_gather(w, B, None, 7000 + k, ws, variant, psize, anc=anc)
            s = offspring_stats(w_h, [anc.cpu().numpy()])
            vals.append(s["mse_per_n"])
            maxoff = max(maxoff, s["max_offspring"])
    return np.asarray(vals), B, maxoff


@pytest.mark.parametrize("log2n,K", [(15, 96), (18, 32), (20, 12)])
def test_megopolis_and_metropolis_mse_match_tables(paper, log2n, K):
    n = 1 << log2n
    for y in range(5):
        got = {}
        for variant, name in ((mego.MEGOPOLIS, "megopolis"), (mego.METROPOLIS, "metropolis")):
            vals, B, maxoff = _mse_runs(n, y, variant, K, (1, 2))
            want = paper[name]["all"][str(n)]["mse_per_n"][y]
            se = vals.std(ddof=1) / np.sqrt(vals.size)
            assert abs(vals.mean() - want) <= 4 * se + 0.004, (name, n, y, vals.mean(), want, se)
            got[name] = vals.mean()
            if variant == mego.MEGOPOLIS:
                assert maxoff <= B + 1
        assert got["megopolis"] < got["metropolis"]      # lower variance (Section 6.1)


@pytest.mark.parametrize("variant,name", [(mego.METROPOLIS_C1, "c1"), (mego.METROPOLIS_C2, "c2")])
@pytest.mark.parametrize("psize", [128, 256, 512, 1024, 2048])
def test_partition_variants_mse_match_tables(paper, variant, name, psize):
    n = 1 << 15
    for y in range(5):
        vals, _, _ = _mse_runs(n, y, variant, 24, (1, 2), psize)
        want = paper[name][str(psize)][str(n)]["mse_per_n"][y]
        se = vals.std(ddof=1) / np.sqrt(vals.size)
        assert abs(vals.mean() - want) <= 4 * se + 0.01 * want, (name, psize, y, vals.mean(), want)
