"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded
synthetic planes: MSD (step a), per-sample best SNR and width (steps b, c),
candidate lists (step d), the fused search, and the edge cases."""
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


def _oracle_plane(x, n_samp, scale=None, offset=None):
    """Host copy of a device plane as the oracle's Plane."""
    dt = {torch.float32: "f32", torch.float16: "f16", torch.bfloat16: "bf16"}[x.dtype]
    return oracle.Plane(synth.to_host_numpy(x), dtype=dt, n_samp=n_samp,
                        scale=None if scale is None else scale.cpu().numpy(),
                        offset=None if offset is None else offset.cpu().numpy())


def _full_case(spd, x, n_samp, widths, thr, scope=0, scale=None, offset=None, capacity=None,
               mode=0, nmax=0):
    """Run every GPU call on x and compare each with the oracle."""
    op = _oracle_plane(x, n_samp, scale, offset)
    mean, sd, sdn, tab = oracle.msd_and_sigma(op, widths, mode, scope, nmax)
    kw = dict(n_samp=n_samp, scale=scale, offset=offset)
    nm = int(nmax or widths[-1]) if mode else 0

    m = spd.msd(x, scope, nm, **kw)
    torch.cuda.synchronize()
    gm = spd.msd_to_numpy(m)
    P.check_msd(gm, mean, sd)
    if mode:
        assert np.all(gm["nmax"] == nm)
        assert np.allclose(gm["sd_nmax"], sdn, rtol=1e-5), (gm["sd_nmax"], sdn)

    best_o, win_o = oracle.boxcar_snr(op, mean, sd, tab, widths, scope)
    snr_g, w_g = spd.boxcar_snr(x, m, widths, mode, scope, **kw)
    torch.cuda.synchronize()

    def sigma_of(e, w):
        return float(oracle.sigma_table(mode, float(np.atleast_1d(sd)[e]), [w],
                                        float(np.atleast_1d(sdn)[e]), nm)[0])

    P.check_plane(snr_g.cpu().numpy(), spd.widths_to_numpy(w_g), best_o, win_o, op, mean,
                  sigma_of, scope=scope)

    n_o = int((best_o >= thr).sum())
    cap = capacity if capacity is not None else max(n_o + 64, 16)
    out, res, _ = spd.search(x, widths, thr, cap, mode, scope, nm, **kw)
    count, status = spd.read_result(res)
    assert status == 0
    recs = spd.candidates_to_numpy(out, count)
    P.check_candidates(recs, count, cap, best_o, thr, win_o=win_o, plane=op, mean=mean,
                       sigma_of=sigma_of, scope=scope)

    # thresholding the plane output (spd_threshold_candidates) meets the same
    # bar against the oracle as the fused search
    out2, res2 = spd.threshold_candidates(snr_g, w_g, thr, cap, n_samp=n_samp)
    c2, s2 = spd.read_result(res2)
    assert s2 == 0
    r2 = spd.candidates_to_numpy(out2, c2)
    P.check_candidates(r2, c2, cap, best_o, thr, win_o=win_o, plane=op, mean=mean,
                       sigma_of=sigma_of, scope=scope)
    return count, best_o


def test_plain_fp32_config(spd):
    """64 DM x 65536 samples, N(0,1), five top-hats, widths 1..32, threshold 6."""
    sp = synth.plain_tophat(64, 65536, device=DEV, seed=1611_0)
    count, best_o = _full_case(spd, sp.data, sp.n_samp, list(range(1, 33)), 6.0)
    for p in sp.pulses:
        assert best_o[p.dm, p.sample] >= 6.0


@pytest.mark.parametrize("n_dm,n_samp,stride", [(5, 10001, 10016), (3, 4097, 4097),
                                                (2, 4095, 4100), (7, 13, 16), (3, 1, 1),
                                                (1, 8191, 8192)])
def test_ragged_shapes(spd, n_dm, n_samp, stride):
    sp = synth.plain_tophat(n_dm, n_samp, widths=(3,) if n_samp > 200 else (), device=DEV,
                            seed=n_samp, stride=stride)
    _full_case(spd, sp.data, n_samp, list(range(1, 33)), 3.0)


@pytest.mark.parametrize("widths", [
    [1], [7], [2, 3, 5, 9, 17, 40, 100], list(range(1, 17)) + list(range(24, 257, 8)),
    [1, 2, 4, 8, 16, 32, 64, 128], list(range(4, 200, 4)), [16, 32, 48, 64, 80],
    list(range(1, 301)), [1, 64, 1024, 4096], list(range(100, 165))])
def test_width_programs(spd, widths):
    """Width lists exercising fine steps, coarse steps of 4/8/16, irregular gaps,
    more than 64 widths (several groups) and the widest halo."""
    sp = synth.ska_like(4, 12000, n_pulses=6, device=DEV, seed=len(widths) + widths[-1],
                        drift_period=4096)
    _full_case(spd, sp.data, sp.n_samp, widths, 7.0)


def test_wide_pulses_at_the_row_end(spd):
    """Top-hats whose windows end a few samples before the row end, found by
    the coarse groups of the 46-width list: the groups' start sums must not
    come from a wider group whose windows met the row end."""
    n_samp = 12000
    sp = synth.ska_like(4, n_samp, n_pulses=0, mean=0.0, sd=1.0, drift_amp=0.0, device=DEV,
                        seed=77)
    for r, w in enumerate((40, 100, 184, 56)):
        synth.inject_tophat(sp.data, r, n_samp - w - 3 * r - 2, w, 15.0 / math.sqrt(w))
    widths = list(range(1, 17)) + list(range(24, 257, 8))
    count, best_o = _full_case(spd, sp.data, n_samp, widths, 7.0)
    for r, w in enumerate((40, 100, 184, 56)):
        assert best_o[r, n_samp - w - 3 * r - 2] >= 7.0


@pytest.mark.parametrize("widths", [list(range(1, 4097)), list(range(8, 4097, 8))])
def test_maximum_width_lists(spd, widths):
    """The API's limits: all 4096 widths (the largest group scale, 64 groups,
    plane output packed over 64 blocks of widths) and 512 coarse widths up to
    SPD_MAX_WIDTH, on rows a little longer than the widest window."""
    sp = synth.ska_like(2, 9000, n_pulses=3, device=DEV, seed=4096 + len(widths),
                        fwhm_range=(1.0, 1500.0))
    _full_case(spd, sp.data, sp.n_samp, widths, 7.0)


def test_ska_like_small(spd):
    """The SKA-like recipe (drift + Gaussian pulses) at reduced size, config widths."""
    widths = list(range(1, 17)) + list(range(24, 257, 8))
    sp = synth.ska_like(16, 65536 + 333, n_pulses=20, device=DEV, seed=1611_1)
    count, _ = _full_case(spd, sp.data, sp.n_samp, widths, 7.0)
    assert count > 0


def test_per_row_scope(spd):
    sp = synth.ska_like(6, 20000, n_pulses=4, device=DEV, seed=9)
    _full_case(spd, sp.data, sp.n_samp, list(range(1, 65)), 6.0, scope=1)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_half_storage_with_scale_offset(spd, dt):
    sp = synth.ska_like(6, 30000, n_pulses=5, device=DEV, seed=21)
    q = synth.quantise_rows(sp, dt)
    off = torch.linspace(-3, 3, q.n_dm, device=DEV, dtype=torch.float32)
    _full_case(spd, q.data, q.n_samp, list(range(1, 17)) + list(range(24, 129, 8)), 7.0,
               scale=q.scale, offset=off)
    _full_case(spd, q.data, q.n_samp, list(range(1, 33)), 7.0, scale=q.scale)


def test_integer_ties(spd):
    """Small integer data gives exact SNR ties between widths; any tied width
    passes, the SNR must match."""
    g = torch.Generator(device=DEV).manual_seed(4)
    x = torch.randint(-2, 3, (4, 3000), generator=g, device=DEV).to(torch.float32)
    _full_case(spd, x, 3000, list(range(1, 9)), 2.5)


def test_overflow_keeps_exact_count(spd):
    sp = synth.ska_like(4, 30000, n_pulses=2, device=DEV, seed=5, drift_period=8192)
    count, _ = _full_case(spd, sp.data, sp.n_samp, list(range(1, 65)), 3.0, capacity=100)
    assert count > 100


def test_degenerate_sigma(spd):
    x = torch.full((3, 5000), 2.5, device=DEV)
    m = spd.msd(x)
    out, res, msd = spd.search(x, [1, 2, 4], 6.0, 10)
    count, status = spd.read_result(res)
    assert count == 0 and status == 5
    assert spd.msd_to_numpy(msd)["status"][0] == 5
    assert spd.msd_to_numpy(m)["status"][0] == 5
    snr, w = spd.boxcar_snr(x, m, [1, 2, 4])
    assert torch.isnan(snr).all() and (w == 0).all()


def test_empty_planes(spd):
    for shape in [(0, 100), (4, 0)]:
        x = torch.empty(shape, device=DEV)
        out, res, _ = spd.search(x, [1, 2], 6.0, 4)
        assert spd.read_result(res) == (0, 0)


def test_repeat_calls_are_deterministic(spd):
    sp = synth.ska_like(8, 40000, n_pulses=10, device=DEV, seed=77)
    w = list(range(1, 17)) + list(range(24, 257, 8))
    o1, r1, m1 = spd.search(sp.data, w, 7.0, 200000)
    o2, r2, m2 = spd.search(sp.data, w, 7.0, 200000)
    c1, c2 = spd.read_result(r1)[0], spd.read_result(r2)[0]
    assert c1 == c2
    assert torch.equal(m1, m2)
    a = np.sort(spd.candidates_to_numpy(o1, c1), order=["dm", "sample"])
    b = np.sort(spd.candidates_to_numpy(o2, c2), order=["dm", "sample"])
    assert np.array_equal(a, b)


def test_boxcar_sums_closed_forms(spd):
    n = 3000
    c = torch.full((2, n), 3.0, device=DEV)
    for w in (1, 7, 64, 999):
        s = spd.boxcar_sums(c, w).cpu().numpy()
        assert np.array_equal(s[:, : n - w + 1], np.full((2, n - w + 1), 3.0 * w))
        assert np.isnan(s[:, n - w + 1:]).all()
    ramp = (5.0 + 2.0 * torch.arange(n, device=DEV, dtype=torch.float32)).reshape(1, -1)
    for w in (1, 3, 50):
        i = np.arange(n - w + 1)
        want = w * 5.0 + 2.0 * (w * i + w * (w - 1) / 2)
        assert np.array_equal(spd.boxcar_sums(ramp, w).cpu().numpy()[0, : n - w + 1], want)
    x = torch.randn(3, 5000, device=DEV)
    for w in (1, 5, 256):
        g = spd.boxcar_sums(x, w).cpu().numpy()
        o = oracle.boxcar_sums(x.cpu().numpy(), w)
        ok = np.isfinite(o)
        assert np.array_equal(np.isnan(g), ~ok)
        assert np.allclose(g[ok], o[ok], rtol=1e-5, atol=1e-5 * math.sqrt(w))


def test_figure1_tophat_response(spd):
    """A top-hat of width W on zero-mean unit noise is found at its leading
    sample with width W (Figure 1)."""
    for W in (1, 4, 13, 32):
        x = torch.zeros((1, 4096), device=DEV)
        x[0, ::2] = 1.0
        x[0, 1::2] = -1.0      # mean 0, sd 1
        x[0, 1000:1000 + W] += 25.0 / math.sqrt(W)
        m = spd.msd(x)
        snr, w = spd.boxcar_snr(x, m, list(range(1, 65)))
        assert int(spd.widths_to_numpy(w)[0, 1000]) in (W, W + 1, W - 1 if W > 1 else 1)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("scope", [0, 1])
def test_eq5_linear_sigma(spd, mode, scope):
    """Eq. 5 (as printed, and read as a linear excess) with sigma_Nmax measured
    on the GPU, on data with signal-dominated rows (a pulse train)."""
    sp = synth.ska_like(6, 30000, n_pulses=4, device=DEV, seed=40 + mode)
    synth.inject_pulse_train(sp.data, row=2, t0=1000, n_pulses=60, width=8, period=32,
                             amp=6.0 * 12.0, n_samp=sp.n_samp)
    widths = list(range(1, 17)) + list(range(24, 129, 8))
    _full_case(spd, sp.data, sp.n_samp, widths, 5.0, scope=scope, mode=mode, nmax=128)


@pytest.mark.parametrize("nmax", [2, 17, 256])
def test_sigma_nmax_against_oracle(spd, nmax):
    sp = synth.ska_like(5, 20001, n_pulses=3, device=DEV, seed=nmax)
    op = _oracle_plane(sp.data, sp.n_samp)
    for scope in (0, 1):
        want = oracle.plane_sd_nmax(op, nmax, scope)
        got = spd.msd_to_numpy(spd.msd(sp.data, scope, nmax))
        assert np.allclose(got["sd_nmax"], want, rtol=1e-5), (got["sd_nmax"], want)


@pytest.mark.parametrize("n_dm,n_samp,stride,nmax,dt,scope", [
    (3, 70001, None, 48, "f32", 0),      # several partials per row; Nmax = 16 k, not 64 k
    (3, 70001, None, 1000, "f32", 1),    # Nmax not a multiple of 16; per-row scope
    (2, 50001, 50017, 300, "f32", 0),    # odd stride (scalar staging), NaN past the row end
    (2, 40000, None, 4096, "bf16", 0),   # the widest window (shared memory above 48 KB)
    (3, 33000, None, 2000, "f16", 1),    # FP16 with per-row scale and offset
])
def test_sigma_nmax_windows(spd, n_dm, n_samp, stride, nmax, dt, scope):
    """MSD and sigma_Nmax against the oracle (two-pass; direct window sums) for
    the window shapes and storage forms the tiled kernels treat apart."""
    x = synth.noise_plane(n_dm, n_samp, 100.0, 12.0, device=DEV, seed=nmax + n_samp,
                          stride=stride)
    scale = offset = None
    if dt != "f32":
        scale = (x[:, :n_samp].abs().amax(dim=1) / 16384.0).contiguous()
        offset = torch.linspace(-2.0, 2.0, n_dm, device=DEV, dtype=torch.float32)
        td = torch.float16 if dt == "f16" else torch.bfloat16
        x = (x / scale.unsqueeze(1)).to(td)
    op = _oracle_plane(x, n_samp, scale, offset)
    mean, sd = oracle.plane_msd(op, scope)
    want = oracle.plane_sd_nmax(op, nmax, scope)
    got = spd.msd_to_numpy(spd.msd(x, scope, nmax, n_samp=n_samp, scale=scale, offset=offset))
    P.check_msd(got, mean, sd)
    assert np.all(got["nmax"] == nmax)
    assert np.allclose(got["sd_nmax"], want, rtol=1e-5), (got["sd_nmax"], want)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_precision_form_eq5(spd, dt):
    """The precision form: FP16 / BF16 storage with per-row scale, 5% of rows
    signal-dominated, Eq. 5 with sigma_Nmax at Nmax = 256."""
    sp = synth.ska_like(20, 40000, n_pulses=6, device=DEV, seed=77)
    synth.inject_pulse_train(sp.data, row=3, t0=2000, n_pulses=125, width=8, period=32,
                             amp=200 * 12.0 / math.sqrt(1000), n_samp=sp.n_samp)
    q = synth.quantise_rows(sp, dt)
    widths = list(range(1, 17)) + list(range(24, 257, 8))
    _full_case(spd, q.data, q.n_samp, widths, 7.0, scale=q.scale, mode=2, nmax=256)
