"""The precision form's error statement: mu, sigma, sigma_Nmax and SNR of the
GPU on FP16 / BF16 storage (per-row scale) against the FP64 oracle on the same
rows before quantisation, with Eq. 5 (sigma_Nmax at Nmax = 256).  Unlike the
parity tests, which compare on the dequantised values, this measures what
the storage costs; the bounds hold the measured figures with margin."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
WIDTHS = list(range(1, 17)) + list(range(24, 257, 8))
THR = 7.0

# the storage's relative step is 2^-11 (FP16) or 2^-8 (BF16) of values near the
# per-row maximum (scale = max|x| / 16384); boxcar sums average part of it away
BOUNDS = {
    "f16": {"mean_abs_err": 2e-5, "sd_rel_err": 1e-5, "sd_nmax_rel_err": 5e-6,
            "snr_err_max_candidates": 2e-3},
    "bf16": {"mean_abs_err": 3e-3, "sd_rel_err": 5e-4, "sd_nmax_rel_err": 5e-5,
             "snr_err_max_candidates": 2e-2},
}


@pytest.fixture(scope="module")
def spd():
    import paper_1611_09704_gb300 as m
    m.build()
    m.load()
    return m


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_quantisation_error_against_fp64(spd, dt):
    sp, rows = synth.precision_plane(64, 524288, device=DEV, seed=1611_7, train_frac=0.25)
    ref = oracle.Plane(synth.to_host_numpy(sp.data))
    q = synth.quantise_rows(sp, dt)
    mean, sd, sdn, tab = oracle.msd_and_sigma(ref, WIDTHS, oracle.SIGMA_LINEAR, 0, 256)
    best, _ = oracle.boxcar_snr(ref, mean, sd, tab, WIDTHS)
    m = spd.msd(q.data, 0, 256, scale=q.scale)
    snr, _ = spd.boxcar_snr(q.data, m, WIDTHS, spd.SIGMA_LINEAR, 0, scale=q.scale)
    torch.cuda.synchronize()
    g = spd.msd_to_numpy(m)[0]
    s = snr.cpu().numpy().astype(np.float64)
    cand = best >= THR
    rel = np.abs(s - best) / np.maximum(np.abs(best), 1.0)
    report = {"mean_abs_err": abs(float(g["mean"]) - float(mean[0])),
              "sd_rel_err": abs(float(g["sd"]) / float(sd[0]) - 1),
              "sd_nmax_rel_err": abs(float(g["sd_nmax"]) / float(sdn[0]) - 1),
              "snr_err_max_candidates": float(rel[cand].max())}
    print(dt, report, "snr_err_max_all", float(rel.max()), "candidates", int(cand.sum()))
    assert cand.sum() > 0
    for k, bound in BOUNDS[dt].items():
        assert report[k] < bound, (k, report[k], bound)
