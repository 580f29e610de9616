"""Comparison rules between the CUDA path and the FP64 oracle.

Tolerances (the single-pulse search's stated bar):
  - SNR:   |snr_gpu - snr_oracle| <= 1e-4 * max(|snr_oracle|, 1)
  - width: equal, or a tie -- the oracle's SNR at the GPU's width is within
           1e-5 * max(|best_oracle|, 1) of the oracle's best
  - candidate sets: identical except samples whose oracle SNR lies within 1e-3
           of the threshold
  - MSD:   |mu_gpu - mu| <= 2e-7 |mu| + 1e-6 sigma, |sigma_gpu/sigma - 1| <= 2e-6
           (an FP32 accumulation held to a budget that keeps the SNR error of the
           widest boxcar, sqrt(w) * d_mu / sigma, inside the SNR tolerance)
"""
from __future__ import annotations

import numpy as np

import oracle

SNR_RTOL = 1e-4
TIE_RTOL = 1e-5
BAND = 1e-3


def check_msd(gpu_msd, mean, sd):
    g = np.atleast_1d(gpu_msd)
    assert g.shape[0] == np.atleast_1d(mean).shape[0]
    mu, s = np.atleast_1d(mean), np.atleast_1d(sd)
    dmu = np.abs(g["mean"] - mu)
    assert np.all(dmu <= 2e-7 * np.abs(mu) + 1e-6 * s), (g["mean"], mu, dmu.max())
    assert np.all(np.abs(g["sd"] / s - 1.0) <= 2e-6), (g["sd"], s)
    assert np.all(g["status"] == 0)


def check_plane(snr_g, w_g, best_o, win_o, plane, mean, sigma_of, rows=None, scope=0):
    """snr_g/w_g: GPU planes [rows, n_samp]; best_o/win_o: oracle planes.
    sigma_of(entry, width) -> sigma_w used to evaluate ties."""
    snr_g = np.asarray(snr_g, dtype=np.float64)
    w_g = np.asarray(w_g)
    tol = SNR_RTOL * np.maximum(np.abs(best_o), 1.0)
    bad = np.abs(snr_g - best_o) > tol
    assert not bad.any(), (
        f"{bad.sum()} SNR mismatches, worst {np.abs(snr_g - best_o).max():.3e}; first at "
        f"{np.argwhere(bad)[:5].tolist()}: gpu {snr_g[bad][:5]} oracle {best_o[bad][:5]}")
    r0 = rows[0] if rows else 0
    mism = np.argwhere(w_g != win_o)
    for (r, i) in mism:
        wg = int(w_g[r, i])
        e = (r0 + r) if scope == 1 else 0
        s_at = oracle.snr_at(plane, r0 + r, i, wg, float(np.atleast_1d(mean)[e]), sigma_of(e, wg))
        assert s_at >= best_o[r, i] - TIE_RTOL * max(abs(best_o[r, i]), 1.0), (
            f"width mismatch at row {r0 + r} sample {i}: gpu {wg} (oracle SNR {s_at}) vs "
            f"oracle {win_o[r, i]} (SNR {best_o[r, i]})")
    return len(mism)


def check_candidates(recs, count, capacity, best_o, thr, row0=0, win_o=None, plane=None,
                     mean=None, sigma_of=None, scope=0, rows=None):
    """GPU records vs the oracle's (best, width) planes over rows [row0, ...)."""
    assert recs.shape[0] == min(count, capacity)
    n_rows, n_samp = best_o.shape
    key = recs["dm"].astype(np.int64) * n_samp + recs["sample"]
    assert np.unique(key).size == key.size, "duplicate candidates"
    assert np.all((recs["dm"] >= row0) & (recs["dm"] < row0 + n_rows))
    assert np.all((recs["sample"] >= 0) & (recs["sample"] < n_samp))
    o_mask = best_o >= thr
    if count <= capacity:
        g_mask = np.zeros_like(o_mask)
        g_mask[recs["dm"] - row0, recs["sample"]] = True
        diff = g_mask ^ o_mask
        band = np.abs(best_o - thr) <= BAND
        assert not (diff & ~band).any(), (
            f"{(diff & ~band).sum()} candidates differ outside the threshold band: "
            f"{np.argwhere(diff & ~band)[:5].tolist()}")
    else:
        # overflow: every written record is a true candidate (or in the band)
        ok = (best_o[recs["dm"] - row0, recs["sample"]] >= thr - BAND)
        assert ok.all()
    b = best_o[recs["dm"] - row0, recs["sample"]]
    assert np.all(np.abs(recs["snr"] - b) <= SNR_RTOL * np.maximum(np.abs(b), 1.0))
    if win_o is not None:
        wo = win_o[recs["dm"] - row0, recs["sample"]]
        for k in np.nonzero(recs["width"] != wo)[0]:
            r, i, wg = int(recs["dm"][k]), int(recs["sample"][k]), int(recs["width"][k])
            e = r if scope == 1 else 0
            s_at = oracle.snr_at(plane, r, i, wg, float(np.atleast_1d(mean)[e]), sigma_of(e, wg))
            assert s_at >= b[k] - TIE_RTOL * max(abs(b[k]), 1.0)
