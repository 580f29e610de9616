"""Decimated search (spd_search_decimated) against the oracle, level by level:
each level's records (told apart by their native width) against the oracle's
search of the decimated series with that level's own MSD."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def spd():
    import paper_1611_09704_gb300 as m
    m.build()
    m.load()
    return m


def _oracle_plane(x, scale=None):
    dt = {torch.float32: "f32", torch.float16: "f16", torch.bfloat16: "bf16"}[x.dtype]
    return oracle.Plane(synth.to_host_numpy(x), dtype=dt,
                        scale=None if scale is None else scale.cpu().numpy())


LEVELS = [(0, list(range(1, 33))), (1, list(range(17, 33))), (2, list(range(17, 33))),
          (4, [9, 12, 16, 24, 32])]


@pytest.mark.parametrize("dtype,n_samp", [("f32", 40000), ("f32", 33333), ("f16", 40000),
                                          ("bf16", 36000)])
def test_decimated_matches_oracle(spd, dtype, n_samp):
    sp = synth.ska_like(10, n_samp, n_pulses=12, mean=0.0, sd=1.0, drift_amp=0.0,
                        fwhm_range=(1.0, 400.0), device=DEV, seed=91)
    x, scale = sp.data, None
    if dtype != "f32":
        q = synth.quantise_rows(sp, dtype)
        x, scale = q.data, q.scale
    thr, cap = 6.0, 1 << 20
    out, res, msd = spd.search_decimated(x, LEVELS, thr, cap, scale=scale)
    count, status = spd.read_result(res)
    assert status == 0 and 0 < count < cap
    recs = spd.candidates_to_numpy(out, count)
    gm = spd.msd_to_numpy(msd)
    op = _oracle_plane(x, scale)
    lo = 0
    for k, (level, widths) in enumerate(LEVELS):
        hi = widths[-1] << level
        sel = recs[(recs["width"] > lo) & (recs["width"] <= hi)]
        lo = hi
        m = 1 << level
        assert np.all(sel["sample"] % m == 0) and np.all(sel["width"] % m == 0)
        xl = oracle.decimate(op, level).astype(np.float32)
        cands, best, win, (mean, sd, _, _) = oracle.search(
            xl, widths, thr, start_w1=(level == 0 or widths[0] == 1))
        P.check_msd(gm[k:k + 1], mean, sd)
        lv = sel.copy()
        lv["sample"] //= m
        lv["width"] //= m
        P.check_candidates(lv, len(lv), cap, best, thr, win_o=win,
                           plane=oracle.Plane(xl), mean=mean,
                           sigma_of=lambda e, w, sd=sd: math.sqrt(w) * float(sd[0]))
        assert len(cands) == 0 or len(lv) > 0


def test_decimated_level0_only_equals_search(spd):
    sp = synth.plain_tophat(8, 20000, device=DEV, seed=92)
    widths = list(range(1, 33))
    out, res, _ = spd.search_decimated(sp.data, [(0, widths)], 6.0, 1 << 16)
    c1, s1 = spd.read_result(res)
    o2, r2, _ = spd.search(sp.data, widths, 6.0, 1 << 16)
    c2, s2 = spd.read_result(r2)
    a = np.sort(spd.candidates_to_numpy(out, c1), order=["dm", "sample"])
    b = np.sort(spd.candidates_to_numpy(o2, c2), order=["dm", "sample"])
    assert (c1, s1) == (c2, s2) and np.array_equal(a, b)


def test_decimated_short_plane_and_bad_levels(spd):
    x = torch.randn((3, 20), device=DEV)
    # level 5 has no complete group of 32 samples: it contributes nothing
    out, res, msd = spd.search_decimated(x, [(0, [1, 2]), (5, [1])], 3.0, 1024)
    c, st = spd.read_result(res)
    assert np.all(spd.candidates_to_numpy(out, c)["width"] <= 2)
    with pytest.raises(spd.SpdError):
        spd.search_decimated(x, [(0, [1, 2, 4]), (1, [2])], 3.0, 1024)
