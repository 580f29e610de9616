"""De-dispersion (spd_dedisperse, the producer of the DM x time plane the
detector searches) against the FP64 oracle, and the coupled path: DM trials
written straight into a streaming search's chunk view and searched in place,
whose candidates must meet the stated rule against the oracle's
de-dispersion followed by the oracle's replay of the same chunk schedule."""
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


@pytest.mark.parametrize("in_dt,out_dt,n_chan,n_samp", [
    ("f32", "f32", 64, 9000),
    ("f32", "f16", 33, 5001),     # ragged sizes, FP16 output
    ("f16", "f32", 48, 7000),     # FP16 channels with per-channel scale
    ("bf16", "bf16", 16, 3000),
    ("f32", "f32", 300, 6000),    # three chunks of channel delays, ragged
])
def test_dedisperse_matches_oracle(spd, in_dt, out_dt, n_chan, n_samp):
    # 11 trials: one partial block of DM trials; 300 channels: 40 trials
    n_trials = 40 if n_chan > 128 else 11
    fb = synth.filterbank(n_chan, n_samp, dms=np.linspace(0, 25, n_trials),
                          pulses=((3, 500, 4, 2.0), (9, 900, 16, 1.0)), device=DEV, seed=7)
    x, scale, dt = fb.data, None, "f32"
    if in_dt != "f32":
        q = synth.quantise_rows(synth.SynthPlane(fb.data, n_samp), in_dt)
        x, scale, dt = q.data, q.scale, in_dt
    delays = torch.from_numpy(fb.delays).to(DEV)
    odt = {"f32": spd.F32, "f16": spd.F16, "bf16": spd.BF16}[out_dt]
    out = spd.dedisperse(spd.Plane(x, scale=scale), delays, fb.n_out, out_dtype=odt)
    got = out.float().cpu().numpy().astype(np.float64)
    op = oracle.Plane(synth.to_host_numpy(x), dtype=dt,
                      scale=None if scale is None else scale.cpu().numpy())
    want = oracle.dedisperse(op, fb.delays, fb.n_out)
    mag = oracle.dedisperse(oracle.Plane(np.abs(op.values()).astype(np.float32)), fb.delays,
                            fb.n_out)
    # FP32 channel sum: a few ulp of the running magnitude per channel; the
    # output type's own rounding on top
    out_rel = {"f32": 0.0, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}[out_dt]
    tol = 2e-7 * n_chan * mag + out_rel * np.abs(want) + 1e-30
    assert np.all(np.abs(got - want) <= tol), np.abs(got - want).max()


def test_wide_delay_spread_matches_oracle(spd):
    """DM trials far apart (spreads of thousands of samples inside one block
    of trials): those channels are summed from global memory, the others
    from the staged window; the same sums either way."""
    dms = np.concatenate([np.linspace(0, 800, 9), np.linspace(2, 6, 9)])
    fb = synth.filterbank(24, 21000, dms=dms, pulses=((4, 600, 8, 2.0),), device=DEV, seed=12)
    assert int(fb.delays.max()) - int(fb.delays.min()) > 1536
    out = spd.dedisperse(fb.data, torch.from_numpy(fb.delays).to(DEV), fb.n_out)
    got = out.cpu().numpy().astype(np.float64)
    op = oracle.Plane(synth.to_host_numpy(fb.data))
    want = oracle.dedisperse(op, fb.delays, fb.n_out)
    mag = oracle.dedisperse(oracle.Plane(np.abs(op.values()).astype(np.float32)), fb.delays,
                            fb.n_out)
    assert np.all(np.abs(got - want) <= 2e-7 * 24 * mag + 1e-30)


def test_out_of_range_delay_sets_status(spd):
    fb = synth.filterbank(8, 2000, dms=np.linspace(0, 10, 4), pulses=(), device=DEV, seed=8)
    bad = fb.delays.copy()
    bad[2, 5] = 2000 - fb.n_out + 1          # one sample past the row for the last output
    res = torch.zeros(16, dtype=torch.uint8, device=DEV)
    out = spd.dedisperse(fb.data, torch.from_numpy(bad).to(DEV), fb.n_out, status=res)
    count, status = spd.read_result(res)
    assert status == 1                        # SPD_ERR_INVALID_ARG
    o = out.cpu().numpy()
    assert np.isnan(o[2]).all() and np.isfinite(np.delete(o, 2, axis=0)).all()


def test_coupled_stream_matches_oracle(spd):
    """A beam's filterbank arrives in time chunks; each chunk's DM trials are
    de-dispersed straight into the push workspace's chunk view and searched
    in place.  Oracle: de-dispersion of the whole filterbank, the plane
    rounded to FP32, then the replay of the same chunk schedule."""
    n_chan, dms = 32, np.linspace(0, 60, 24)
    pulses = ((4, 2500, 8, 0.9), (17, 9000, 24, 0.5), (21, 15000, 3, 1.6))
    delays_np = synth.dispersion_delays(n_chan, dms)
    maxd = int(delays_np.max())
    lengths = [4096, 3000, 777, 8192, 5000]
    total = sum(lengths)
    fb = synth.filterbank(n_chan, total + maxd, dms=dms, pulses=pulses, device=DEV, seed=9)
    assert fb.n_out == total
    delays = torch.from_numpy(fb.delays).to(DEV)
    widths = list(range(1, 17)) + list(range(24, 65, 8))
    thr, cap = 6.0, 1 << 14
    n_dm = len(dms)
    bs = spd.binding.BeamStream(n_dm, torch.float32, widths, thr, 0, device=DEV)
    ws = torch.empty(bs.workspace_bytes(max(lengths)), dtype=torch.uint8, device=DEV)
    out = torch.empty((cap, 4), dtype=torch.int32, device=DEV)
    res = torch.empty(16, dtype=torch.uint8, device=DEV)
    calls, t = [], 0
    for L in lengths:
        view = bs.chunk_view(L, ws)
        spd.dedisperse(fb.data[:, t:t + L + maxd], delays, L, out=view)
        bs.push(spd.Plane(view), out, cap, res, ws)
        cnt, st = spd.read_result(res)
        calls.append((cnt, st, spd.candidates_to_numpy(out, cnt)))
        t += L
    bs.flush(out, cap, res, ws)
    cnt, st = spd.read_result(res)
    calls.append((cnt, st, spd.candidates_to_numpy(out, cnt)))

    plane = oracle.dedisperse(synth.to_host_numpy(fb.data), fb.delays, total).astype(np.float32)
    bounds = np.cumsum([0] + lengths)
    chunks = [np.ascontiguousarray(plane[:, a:b]) for a, b in zip(bounds[:-1], bounds[1:])]
    rep = oracle.stream_replay(chunks, widths, thr, 0, detail=True)
    assert len(calls) == len(rep)
    for k, ((cnt, st, recs), r) in enumerate(zip(calls, rep)):
        assert st == 0, (k, st)
        lo, hi = r["lo"], r["hi"]
        if hi <= lo:
            assert cnt == 0
            continue
        assert np.all((recs["sample"] >= lo) & (recs["sample"] < hi))
        shifted = recs.copy()
        shifted["sample"] -= lo
        sd = float(np.atleast_1d(r["sd"])[0])
        P.check_candidates(shifted, cnt, cap, r["best"], thr, win_o=r["win"], plane=r["sub"],
                           mean=r["mean"], sigma_of=lambda e, w: math.sqrt(w) * sd)
    found = np.concatenate([c[2] for c in calls])
    for (k, t0, w, amp) in pulses:          # each dispersed pulse found at its trial
        assert np.any((found["dm"] == k) & (np.abs(found["sample"] - t0) <= w))


def test_full_size_sampled_trials_match_oracle(spd):
    """The bench's workload (256 channels 1200-1500 MHz at 64 us, 256 trials
    at DM 0..100, 2^18 output samples) in its launch configuration: every
    output of 8 trials spread over the range against the oracle's
    de-dispersion of those trials."""
    n_chan, n_dm, n_out = 256, 256, 1 << 18
    dms = np.linspace(0.0, 100.0, n_dm)
    delays_np = synth.dispersion_delays(n_chan, dms)
    fb = synth.filterbank(n_chan, n_out + int(delays_np.max()), dms=dms,
                          pulses=((100, 5000, 8, 0.5),), device=DEV, seed=1611_8)
    assert fb.n_out == n_out
    out = spd.dedisperse(fb.data, torch.from_numpy(fb.delays).to(DEV), n_out)
    sel = np.arange(0, n_dm, 37)
    got = out[torch.from_numpy(sel).to(DEV)].cpu().numpy().astype(np.float64)
    x = synth.to_host_numpy(fb.data)
    want = oracle.dedisperse(x, np.ascontiguousarray(fb.delays[sel]), n_out)
    mag = oracle.dedisperse(np.abs(x).astype(np.float32), np.ascontiguousarray(fb.delays[sel]),
                            n_out)
    assert np.all(np.abs(got - want) <= 2e-7 * n_chan * mag + 1e-30), np.abs(got - want).max()
