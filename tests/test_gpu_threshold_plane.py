"""spd_threshold_plane (Sec. 2.4 on the plane) against the oracle's statement
of it, applied to the same SNR plane, and against the candidate list."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def spd():
    import paper_1611_09704_gb300 as m
    m.build()
    m.load()
    return m


@pytest.mark.parametrize("n_samp,stride", [(4096, 4096), (3001, 3008), (777, 781)])
def test_threshold_plane_matches_oracle_and_list(spd, n_samp, stride):
    sp = synth.plain_tophat(9, n_samp, device=DEV, seed=81)
    widths = list(range(1, 33))
    thr = 4.0
    m = spd.msd(sp.data)
    snr = torch.full((9, stride), float("nan"), device=DEV)
    wid = torch.zeros((9, stride), dtype=torch.int16, device=DEV)
    spd.boxcar_snr(sp.data, m, widths, snr_out=snr[:, :n_samp], width_out=wid[:, :n_samp])
    s0 = snr[:, :n_samp].cpu().numpy().copy()
    w0 = spd.widths_to_numpy(wid[:, :n_samp])
    out, res = spd.threshold_candidates(snr, wid, thr, 1 << 16, n_samp=n_samp)
    cnt, st = spd.read_result(res)
    recs = spd.candidates_to_numpy(out, cnt)
    spd.threshold_plane(snr, wid, thr, n_samp=n_samp)
    torch.cuda.synchronize()
    s1 = snr.cpu().numpy()
    w1 = spd.widths_to_numpy(wid)
    eb, ew = oracle.threshold_plane(s0, w0, thr)
    assert np.array_equal(s1[:, :n_samp].astype(np.float64), eb)
    assert np.array_equal(w1[:, :n_samp], ew)
    assert np.isnan(s1[:, n_samp:]).all()          # columns past n_samp untouched
    kept = np.argwhere(s1[:, :n_samp] != 0)
    assert st == 0 and cnt == len(kept) > 0
    got = np.sort(recs, order=["dm", "sample"])
    assert np.array_equal(np.stack([got["dm"], got["sample"]], 1), kept)


def test_threshold_plane_bad_args(spd):
    snr = torch.zeros((2, 10), device=DEV)
    with pytest.raises(spd.SpdError):
        spd.threshold_plane(snr, None, float("nan"))
    spd.threshold_plane(snr[:, :0], None, 1.0, n_samp=0)   # empty: nothing to do
