"""Parity at full size, in the launch configuration the benchmark times.

The SKA-like 4096 x 524288 FP32 plane goes through the sharded search path of
bench.py (one shard), its FP16 precision form (Eq. 5) through spd_search, and
the four batched ranges through one captured batched launch.  The oracle
cannot search these planes whole, so the tests check:
- the MSD over the whole plane (FP64 two-pass), and for Eq. 5 sigma_Nmax from
  FP64 cumulative sums;
- sampled outputs, one by one: the SNR and width of candidate records, and
  the candidate/non-candidate decision at random positions of sampled rows,
  from direct FP64 boxcar sums (Algorithm 1 at one start)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SKA_WIDTHS = list(range(1, 17)) + list(range(24, 257, 8))
CAND = np.dtype([("dm", "<i4"), ("sample", "<i4"), ("snr", "<f4"), ("width", "<i4")])


@pytest.fixture(scope="module")
def spd():
    import paper_1611_09704_gb300 as m
    m.build()
    m.load()
    return m


def _best_at(op, r, i, widths, mean, sd, sigma_of=None):
    """Algorithm 1 at one start, from direct sums: (best SNR, its width);
    sigma_of(w) gives sigma_w (default Eq. 4)."""
    sig = sigma_of or (lambda w: math.sqrt(w) * sd)
    best, win = oracle.snr_at(op, r, i, 1, mean, sig(1)), 1
    for w in widths:
        if w == 1:
            continue
        s = oracle.snr_at(op, r, i, w, mean, sig(w))
        if s != s:          # past the row end
            break
        if s > best:
            best, win = s, w
    return best, win


def _check_rows(op, recs_dev, rows, dm_offset, widths, mean, sd, thr, rng, n_cand=120,
                n_pos=200, sigma_of=None):
    """Sampled candidates and sampled positions of the given rows."""
    n_samp = op.n_samp
    checked = 0
    for r in rows:
        sel = recs_dev[recs_dev[:, 0] == dm_offset + r]
        recs = sel.cpu().numpy().copy().view(CAND).reshape(-1)
        samples = set(recs["sample"].tolist())
        assert len(samples) == len(recs), "duplicate candidates"
        for k in rng.choice(len(recs), size=min(n_cand, len(recs)), replace=False):
            rec = recs[k]
            b, w = _best_at(op, r, int(rec["sample"]), widths, mean, sd, sigma_of)
            assert b >= thr - P.BAND
            assert abs(float(rec["snr"]) - b) <= P.SNR_RTOL * max(abs(b), 1.0), (r, rec, b)
            if int(rec["width"]) != w:   # a tie within the stated tolerance
                wg = int(rec["width"])
                sw = oracle.snr_at(op, r, int(rec["sample"]), wg, mean,
                                   sigma_of(wg) if sigma_of else math.sqrt(wg) * sd)
                assert sw >= b - P.TIE_RTOL * max(abs(b), 1.0), (r, rec, b, w)
            checked += 1
        for i in rng.integers(0, n_samp, size=n_pos):
            b, _ = _best_at(op, r, int(i), widths, mean, sd, sigma_of)
            if b >= thr + P.BAND:
                assert int(i) in samples, (r, i, b)
            elif b < thr - P.BAND:
                assert int(i) not in samples, (r, i, b)
            checked += 1
    return checked


def test_ska_like_full_size_sharded_path(spd):
    from paper_1611_09704_gb300.sharding import ShardedSearch
    n_dm, n_samp, thr = 4096, 524288, 7.0
    x = synth.ska_like(n_dm, n_samp, device=DEV, seed=1611_1).data   # bench.py's plane
    cap = int(n_dm * n_samp * 0.45) + 1024
    ss = ShardedSearch(x, SKA_WIDTHS, thr, cap)
    ss.run()
    count, status = spd.read_result(ss.result)
    assert status == 0 and 0 < count <= cap
    gm = spd.msd_to_numpy(ss.msd)
    op = oracle.Plane(synth.to_host_numpy(x))
    mean, sd = oracle.plane_msd(op)
    P.check_msd(gm, mean, sd)
    rng = np.random.default_rng(2024)
    rows = rng.choice(n_dm, size=6, replace=False)
    n = _check_rows(op, ss.out[:count], rows, 0, SKA_WIDTHS, float(mean[0]), float(sd[0]),
                    thr, rng)
    assert n > 1000


def _sd_nmax_fp64(op, nmax, shift):
    """sigma_Nmax by its definition (population sd of the nmax-sample boxcar
    series over full windows, pooled over the plane), in FP64 from per-row
    cumulative sums of the dequantised values, 256 rows at a time.  The sums
    are taken about `shift` (near nmax x mean), so the one-pass moments lose
    nothing to cancellation."""
    s1 = s2 = 0.0
    count = 0
    for r0 in range(0, op.n_dm, 256):
        sub = oracle.Plane(op.data[r0:r0 + 256], dtype=op.dtype, n_samp=op.n_samp,
                           scale=None if op.scale is None else op.scale[r0:r0 + 256])
        c = np.cumsum(sub.values(), axis=1)
        b = c[:, nmax - 1:].copy()
        b[:, 1:] -= c[:, :-nmax]
        b -= shift
        s1 += b.sum()
        s2 += np.dot(b.ravel(), b.ravel())
        count += b.size
    m = s1 / count
    return math.sqrt(s2 / count - m * m)


def test_precision_form_full_size_eq5(spd):
    n_dm, n_samp, thr = 4096, 524288, 7.0
    sp, _ = synth.precision_plane(n_dm, n_samp, device=DEV)      # bench.py's recipe
    q = synth.quantise_rows(sp, "f16")
    del sp
    torch.cuda.empty_cache()
    cap = int(n_dm * n_samp * 0.45) + 1024
    out, res, msd = spd.search(q.data, SKA_WIDTHS, thr, cap, spd.SIGMA_LINEAR, 0, 256,
                               scale=q.scale)
    count, status = spd.read_result(res)
    assert status == 0 and 0 < count <= cap
    g = spd.msd_to_numpy(msd)
    op = oracle.Plane(synth.to_host_numpy(q.data), dtype="f16", scale=q.scale.cpu().numpy())
    mean, sd = oracle.plane_msd(op)
    P.check_msd(g, mean, sd)
    sdn = _sd_nmax_fp64(op, 256, 256 * float(mean[0]))
    assert float(g["sd_nmax"][0]) == pytest.approx(sdn, rel=1e-5)
    tab = oracle.sigma_table(oracle.SIGMA_LINEAR, float(sd[0]), SKA_WIDTHS, sdn, 256)
    sig = dict(zip(SKA_WIDTHS, tab))
    rng = np.random.default_rng(2026)
    recs_dev = out[:count]
    hit = torch.unique(recs_dev[:, 0]).cpu().numpy()
    rows = list(rng.choice(hit, size=min(3, len(hit)), replace=False)) + \
        list(rng.choice(n_dm, size=2, replace=False))
    n = _check_rows(op, recs_dev, rows, 0, SKA_WIDTHS, float(mean[0]), float(sd[0]), thr, rng,
                    n_cand=80, n_pos=120, sigma_of=lambda w: sig[w])
    assert n > 300


def test_batched_full_size_one_graph_launch(spd):
    specs, planes, off = [], [], 0
    for sp, dec, widths in synth.batched_ranges(1.0, device=DEV):
        specs.append(spd.RangeSpec(sp.data, widths, 7.0, dm_offset=off, decimation=dec))
        planes.append((sp.data, widths, off))
        off += sp.n_dm
    cap = 1 << 24
    bs = spd.BatchedSearch(specs, cap, tuning={"ctas_per_sm": 0, "group_scale": 1}, graph=True)
    bs.run()
    count, status = spd.read_result(bs.result)
    assert status == 0 and 0 < count < cap
    gm = spd.msd_to_numpy(bs.msd)
    rng = np.random.default_rng(2025)
    recs_dev = bs.out[:count]
    for k, (x, widths, dm_off) in enumerate(planes):
        op = oracle.Plane(synth.to_host_numpy(x))
        mean, sd = oracle.plane_msd(op)
        P.check_msd(gm[k:k + 1], mean, sd)
        # rows with a candidate, and random rows
        dms = recs_dev[(recs_dev[:, 0] >= dm_off) & (recs_dev[:, 0] < dm_off + x.shape[0]), 0]
        hit = (torch.unique(dms) - dm_off).cpu().numpy()
        rows = list(rng.choice(hit, size=min(2, len(hit)), replace=False)) + \
            list(rng.choice(x.shape[0], size=1))
        _check_rows(op, recs_dev, rows, dm_off, widths, float(mean[0]), float(sd[0]), 7.0, rng,
                    n_cand=60, n_pos=80)
        del op
