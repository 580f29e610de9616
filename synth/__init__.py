"""Seeded synthetic DM x time planes for the single-pulse search.

This module only draws random numbers and lays out test signals; it holds
none of the detection arithmetic (no mean/sd estimation, no boxcar, no SNR).
Both the CUDA path's tests and the oracle's tests take their inputs from here.

The paper's SKA-like data (about 6000 DM trials at 64 us sampling, Sec. 3) is
not available, so these planes stand in for de-dispersed data:

- :func:`plain_tophat` -- i.i.d. N(mu, sd) noise with top-hat pulses of given
  widths (the plain FP32 case: 64 x 65536, widths {1,3,8,17,30}).
- :func:`ska_like` -- N(100, 12^2) noise, a slow per-row sinusoidal baseline
  drift of +-2 sd with period 2^16 samples, and Gaussian-profile pulses with
  FWHM 1..200 samples and matched-filter SNR 6..50 spread over 5..20 adjacent
  DM trials (4096 x 524288 at full size).
- :func:`quantise_rows` -- FP16 / BF16 storage with an FP32 per-row scale.

All generators run on the requested torch device with a seeded
``torch.Generator``; the same tensor, copied to the host, feeds the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

SAMPLE_TIME_S = 64e-6  # sampling time of the SKA-like data (Sec. 3)


@dataclass
class Pulse:
    dm: int            # first DM row the pulse touches
    sample: int        # leading sample of the top-hat, or centre of the Gaussian
    width: float       # top-hat width in samples, or Gaussian FWHM
    snr: float         # intended matched-filter SNR
    n_dm: int = 1      # rows spanned
    kind: str = "tophat"


@dataclass
class SynthPlane:
    data: torch.Tensor                 # [n_dm, stride] float32 (or fp16/bf16)
    n_samp: int
    pulses: list = field(default_factory=list)
    scale: torch.Tensor | None = None  # per-row FP32 scale (quantised planes)
    offset: torch.Tensor | None = None
    seed: int = 0
    recipe: str = ""

    @property
    def n_dm(self) -> int:
        return self.data.shape[0]


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _uniform(g, lo, hi, device):
    return float(lo + (hi - lo) * torch.rand((), generator=g, device=device).item())


def _randint(g, lo, hi_incl, device):
    return int(torch.randint(lo, hi_incl + 1, (), generator=g, device=device).item())


def noise_plane(n_dm, n_samp, mean=0.0, sd=1.0, *, device="cpu", seed=0,
                stride=None, row_block=256) -> torch.Tensor:
    """i.i.d. Gaussian noise [n_dm, stride]; columns >= n_samp are set to NaN
    so that any read past the row end shows up in the results."""
    stride = n_samp if stride is None else stride
    g = _gen(device, seed)
    out = torch.empty((n_dm, stride), dtype=torch.float32, device=device)
    for r0 in range(0, n_dm, row_block):
        r1 = min(n_dm, r0 + row_block)
        out[r0:r1, :n_samp].normal_(mean, sd, generator=g)
    if stride > n_samp:
        out[:, n_samp:] = float("nan")
    return out


def inject_tophat(plane: torch.Tensor, dm: int, t0: int, width: int, amp: float,
                  n_samp: int | None = None):
    n_samp = plane.shape[1] if n_samp is None else n_samp
    t1 = min(n_samp, t0 + width)
    plane[dm, t0:t1] += amp


def inject_pulse_train(plane: torch.Tensor, row: int, t0: int, n_pulses: int, width: int,
                       period: int, amp: float, n_samp: int | None = None):
    """A train of n_pulses top-hats of `width` samples every `period` samples
    starting at t0 on one row (signal-dominated rows of the precision form)."""
    n_samp = plane.shape[1] if n_samp is None else n_samp
    for k in range(n_pulses):
        a = t0 + k * period
        if a >= n_samp:
            break
        plane[row, a:min(n_samp, a + width)] += amp


def _gauss_profile(fwhm: float, device):
    s = fwhm / 2.3548
    half = int(math.ceil(4.0 * s)) + 1
    t = torch.arange(-half, half + 1, dtype=torch.float64, device=device)
    return t, torch.exp(-0.5 * (t / s) ** 2)


def plain_tophat(n_dm=64, n_samp=65536, *, widths=(1, 3, 8, 17, 30), snr_range=(8.0, 30.0),
                 mean=0.0, sd=1.0, device="cpu", seed=1611_0, stride=None) -> SynthPlane:
    """N(mean, sd^2) noise with one top-hat pulse per listed width.  Amplitude
    a = SNR * sd / sqrt(W) gives boxcar SNR ~ U(snr_range) at the matching width.
    Pulses sit on distinct rows when n_dm allows, else > 64 samples apart."""
    data = noise_plane(n_dm, n_samp, mean, sd, device=device, seed=seed, stride=stride)
    g = _gen("cpu", seed + 7)
    rows = torch.randperm(n_dm, generator=g)[: len(widths)].tolist()
    pulses = []
    used = []
    for k, w in enumerate(widths):
        dm = rows[k % len(rows)]
        snr = _uniform(g, *snr_range, "cpu")
        for _ in range(1000):
            t0 = _randint(g, 64, max(64, n_samp - w - 64), "cpu")
            if all(d != dm or abs(t0 - t) > 64 + w + ww for d, t, ww in used):
                break
        used.append((dm, t0, w))
        amp = snr * sd / math.sqrt(w)
        inject_tophat(data, dm, t0, w, amp, n_samp)
        pulses.append(Pulse(dm, t0, w, snr))
    return SynthPlane(data, n_samp, pulses, seed=seed,
                      recipe=f"N({mean},{sd}^2) + top-hats {tuple(widths)} SNR U{snr_range}")


def ska_like(n_dm=4096, n_samp=524288, *, n_pulses=200, mean=100.0, sd=12.0,
             drift_amp=24.0, drift_period=65536, fwhm_range=(1.0, 200.0),
             snr_range=(6.0, 50.0), adj_range=(5, 20), device="cpu", seed=1611_1,
             stride=None, row_block=256) -> SynthPlane:
    """SKA-like chunk: noise N(mean, sd^2) + drift_amp * sin(2 pi t / period + phi_row)
    with phi_row ~ U(0, 2 pi), plus Gaussian pulses.  A pulse of FWHM f has
    profile g(t) = exp(-t^2 / 2 s^2), s = f / 2.3548, and amplitude
    a = SNR * sd / sqrt(sum g^2); it spans n_adj ~ U{5..20} adjacent rows with
    the SNR tapering linearly to 50% at the edges and a per-row arrival shift
    of U[-2, 2] samples."""
    stride = n_samp if stride is None else stride
    data = noise_plane(n_dm, n_samp, mean, sd, device=device, seed=seed, stride=stride,
                       row_block=row_block)
    gp = _gen("cpu", seed + 11)
    phi = torch.rand(n_dm, generator=gp, dtype=torch.float64) * (2 * math.pi)
    t = torch.arange(n_samp, dtype=torch.float64, device=device) * (2 * math.pi / drift_period)
    for r0 in range(0, n_dm, row_block):
        r1 = min(n_dm, r0 + row_block)
        ph = phi[r0:r1].to(device).unsqueeze(1)
        data[r0:r1, :n_samp] += (drift_amp * torch.sin(t.unsqueeze(0) + ph)).to(torch.float32)
    pulses = []
    for _ in range(n_pulses):
        fwhm = _uniform(gp, *fwhm_range, "cpu")
        snr = _uniform(gp, *snr_range, "cpu")
        n_adj = _randint(gp, adj_range[0], adj_range[1], "cpu")
        dm0 = _randint(gp, 0, max(0, n_dm - n_adj), "cpu")
        tc = _randint(gp, 512, max(512, n_samp - 512), "cpu")
        tt, prof = _gauss_profile(fwhm, device)
        amp0 = snr * sd / float(torch.sqrt((prof * prof).sum()))
        centre = (n_adj - 1) / 2.0
        for j in range(min(n_adj, n_dm - dm0)):
            taper = 1.0 - 0.5 * abs(j - centre) / max(centre, 1e-9) if n_adj > 1 else 1.0
            shift = _randint(gp, -2, 2, "cpu")
            idx = tt.long() + tc + shift
            keep = (idx >= 0) & (idx < n_samp)
            data[dm0 + j, idx[keep]] += (amp0 * taper * prof[keep]).to(torch.float32)
        pulses.append(Pulse(dm0, tc, fwhm, snr, n_adj, "gauss"))
    if stride > n_samp:
        data[:, n_samp:] = float("nan")
    return SynthPlane(data, n_samp, pulses, seed=seed,
                      recipe=(f"N({mean},{sd}^2) + {drift_amp}*sin(2pi t/{drift_period}+phi) + "
                              f"{n_pulses} Gaussian pulses FWHM U{fwhm_range} SNR U{snr_range} "
                              f"over U{adj_range} rows"))


def precision_plane(n_dm=4096, n_samp=524288, *, device="cpu", seed=1611_2,
                    train_frac=0.05, train_seed=1611_3) -> tuple:
    """The precision form's FP32 signal before storage: the SKA-like recipe plus,
    on a seeded train_frac of the rows, a 4000-sample pulse train (125 width-8
    top-hats every 32 samples from sample 100000, total matched SNR 200 at
    sd 12).  Returns (SynthPlane, train rows)."""
    sp = ska_like(n_dm, n_samp, device=device, seed=seed)
    n_train = max(1, int(round(train_frac * n_dm)))
    g = torch.Generator().manual_seed(train_seed)
    rows = torch.randperm(n_dm, generator=g)[:n_train].tolist()
    for r in rows:
        inject_pulse_train(sp.data, r, min(100000, max(0, n_samp - 4000)), 125, 8, 32,
                           200 * 12.0 / math.sqrt(1000), n_samp)
    return sp, rows


def quantise_rows(sp: SynthPlane, dtype: str, q_max: float = 16384.0) -> SynthPlane:
    """Store a float32 plane as FP16 or BF16 with an FP32 per-row scale
    scale_r = max|x_r| / q_max (offset 0); the stored value is round(x / scale)."""
    n = sp.n_samp
    x = sp.data[:, :n].to(torch.float32)
    amax = x.abs().amax(dim=1).clamp_min(1e-30)
    scale = (amax / q_max).to(torch.float32)
    td = torch.float16 if dtype == "f16" else torch.bfloat16
    q = torch.zeros(sp.data.shape, dtype=td, device=sp.data.device)
    q[:, :n] = (x / scale.unsqueeze(1)).to(td)
    return SynthPlane(q, n, sp.pulses, scale=scale.contiguous(), offset=None,
                      seed=sp.seed, recipe=sp.recipe + f"; stored {dtype} with per-row scale")


def snr_plane(n_dm, n_samp, *, stride=None, device="cpu", seed=0, levels=10, nan_frac=0.01,
              max_width=512):
    """A seeded stand-in for a per-sample best-SNR plane and its width plane:
    SNRs drawn from the integers 0..levels-1 (exact in FP32, so equal peaks
    occur), a nan_frac of them NaN, widths uniform in 1..max_width (int16
    holding uint16).  Columns >= n_samp of a wider stride are NaN / 0."""
    stride = n_samp if stride is None else stride
    g = _gen(device, seed)
    snr = torch.full((n_dm, stride), float("nan"), dtype=torch.float32, device=device)
    v = torch.randint(0, levels, (n_dm, n_samp), generator=g, device=device).to(torch.float32)
    nan = torch.rand((n_dm, n_samp), generator=g, device=device) < nan_frac
    snr[:, :n_samp] = torch.where(nan, torch.full_like(v, float("nan")), v)
    width = torch.zeros((n_dm, stride), dtype=torch.int16, device=device)
    width[:, :n_samp] = torch.randint(1, max_width + 1, (n_dm, n_samp), generator=g,
                                      device=device).to(torch.int16)
    return snr, width


def to_host_numpy(t: torch.Tensor) -> np.ndarray:
    """Host copy for the oracle: float32 as is, fp16/bf16 as raw uint16 bits."""
    t = t.detach().cpu().contiguous()
    if t.dtype == torch.float32:
        return t.numpy()
    return t.view(torch.int16).numpy().view(np.uint16)


# Decimations and shapes of the batched form: four DM ranges searched at time
# decimation 1/2/4/8 with widths 1..64 / 1..128 / 1..256 / 1..512 (decimated
# samples).
BATCHED_RANGES = [(2048, 524288, 1, 64), (1536, 262144, 2, 128), (1024, 131072, 4, 256),
                  (512, 65536, 8, 512)]


def batched_ranges(scale: float = 1.0, *, device="cpu", seed=1611_4, pulses_per_range=50):
    """The batched form's ranges as SynthPlanes: N(0, 1) noise with Gaussian
    pulses as in the SKA-like recipe (no drift); `scale` shrinks the DM count
    of each range (tests).  Returns [(SynthPlane, decimation, widths)]."""
    out = []
    for k, (n_dm, n_samp, dec, wmax) in enumerate(BATCHED_RANGES):
        nd = max(1, int(round(n_dm * scale)))
        sp = ska_like(nd, n_samp, n_pulses=max(1, int(pulses_per_range * scale)), mean=0.0,
                      sd=1.0, drift_amp=0.0, fwhm_range=(1.0, min(200.0, wmax)), device=device,
                      seed=seed + k)
        out.append((sp, dec, list(range(1, wmax + 1))))
    return out


# Serving form: beams of 2048 DM trials delivered in chunks of U{8192..65536}
# samples, N(0, 1) noise, top-hat pulses arriving as a Poisson process in data
# time.
@dataclass
class ServingBeam:
    beam: int
    chunks: list              # torch tensors [n_dm, L_k] (storage dtype)
    lengths: list
    pulses: list


def serving_beams(n_beams=16, n_dm=2048, chunks_per_beam=4, *, length_range=(8192, 65536),
                  rate_hz=0.5, snr_range=(6.0, 40.0), width_range=(1, 128), adj_range=(1, 8),
                  dtype="f16", sample_time=SAMPLE_TIME_S, device="cpu", seed=1611_5,
                  pin_memory=False) -> list:
    """Per beam: chunk lengths L ~ U{length_range}; N(0, 1) noise; pulses at
    Poisson times (rate_hz per second of data at `sample_time` sampling) with
    SNR ~ U(snr_range), top-hat width W ~ U{width_range}, amplitude SNR / sqrt(W),
    over n_adj ~ U{adj_range} adjacent DM rows; a pulse may straddle chunks.
    Chunks are stored as `dtype` ("f16", "bf16" or "f32"), copied to
    page-locked host memory when pin_memory is set."""
    td = {"f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}[dtype]
    out = []
    for b in range(n_beams):
        g = _gen("cpu", seed * 1000 + b)
        lengths = [_randint(g, length_range[0], length_range[1], "cpu")
                   for _ in range(chunks_per_beam)]
        total = sum(lengths)
        t_data = total * sample_time
        n_p = int(torch.poisson(torch.tensor([rate_hz * t_data], dtype=torch.float64),
                                generator=g).item())
        pulses = []
        for _ in range(n_p):
            t0 = _randint(g, 0, total - 1, "cpu")
            w = _randint(g, width_range[0], width_range[1], "cpu")
            snr = _uniform(g, *snr_range, "cpu")
            n_adj = _randint(g, adj_range[0], adj_range[1], "cpu")
            dm0 = _randint(g, 0, max(0, n_dm - n_adj), "cpu")
            pulses.append(Pulse(dm0, t0, w, snr, n_adj))
        chunks = []
        a = 0
        for k, L in enumerate(lengths):
            x = noise_plane(n_dm, L, device=device, seed=seed * 1000 + b * 64 + k + 1)
            for p in pulses:
                lo, hi = max(p.sample, a), min(p.sample + int(p.width), a + L)
                if lo < hi:
                    x[p.dm:p.dm + p.n_dm, lo - a:hi - a] += p.snr / math.sqrt(p.width)
            x = x.to(td)
            if pin_memory:
                x = x.cpu().pin_memory()
            chunks.append(x)
            a += L
        out.append(ServingBeam(b, chunks, lengths, pulses))
    return out


# Filterbanks for the de-dispersion producer: channel rows of noise with
# pulses dispersed as a cold plasma does (delay proportional to DM / f^2).
K_DM_S = 4.148808e3   # dispersion constant, s MHz^2 pc^-1 cm^3


def dispersion_delays(n_chan: int, dms, f_lo_mhz: float = 1200.0, f_hi_mhz: float = 1500.0,
                      t_samp: float = SAMPLE_TIME_S) -> np.ndarray:
    """Integer delays [n_dm, n_chan] (samples) of each channel relative to the
    highest frequency, channels ordered from f_hi down to f_lo."""
    f = np.linspace(f_hi_mhz, f_lo_mhz, n_chan)
    dms = np.asarray(dms, dtype=np.float64).reshape(-1, 1)
    dt = K_DM_S * dms * (f.reshape(1, -1) ** -2 - f_hi_mhz ** -2) / t_samp
    return np.rint(dt).astype(np.int32)


@dataclass
class Filterbank:
    data: torch.Tensor        # [n_chan, n_samp] float32
    delays: np.ndarray        # [n_dm, n_chan] int32
    n_out: int                # de-dispersed samples per DM trial
    pulses: list              # (dm trial, start sample in the DM x time plane, width, amp)


def filterbank(n_chan=64, n_samp=20000, dms=None, *, pulses=((5, 3000, 8, 2.0),),
               sd=1.0, device="cpu", seed=1611_7) -> Filterbank:
    """N(0, sd^2) channel noise with top-hat pulses, each dispersed exactly
    along one DM trial's delays: pulse (k, t0, w, amp) adds amp to channel c
    at samples t0 + delays[k, c] .. + w - 1, so the de-dispersed trial k holds
    a top-hat of height n_chan * amp at t0 .. t0 + w - 1."""
    if dms is None:
        dms = np.linspace(0.0, 40.0, 16)
    delays = dispersion_delays(n_chan, dms)
    n_out = n_samp - int(delays.max())
    if n_out <= 0:
        raise ValueError("filterbank shorter than the largest delay")
    g = _gen(device, seed)
    data = torch.empty((n_chan, n_samp), dtype=torch.float32, device=device)
    data.normal_(0.0, sd, generator=g)
    for (k, t0, w, amp) in pulses:
        for c in range(n_chan):
            a = int(t0 + delays[k, c])
            data[c, a:min(n_samp, a + w)] += amp
    return Filterbank(data, delays, n_out, list(pulses))
