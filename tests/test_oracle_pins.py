"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Nothing here compares the oracle with itself: every check is a closed form,
a hand-evaluated table (tests/golden/), an invariant, a library routine, or a
brute-force enumeration written independently of the oracle's loops.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# ------------------------------------------------------------ Sec. 2.1, Eq. 1/2

def test_chan_stream_hand_values():
    """Eq. 1 with the square restored reproduces hand-evaluated (T, S)."""
    for xs, T, S in _rows("chan_small.txt"):
        x = np.array([float(v) for v in xs.split(",")])
        t, s = oracle.chan_stream(x)
        assert t == pytest.approx(float(T), rel=0, abs=1e-12)
        assert s == pytest.approx(float(S), rel=1e-14, abs=1e-12)


def test_chan_first_step_closed_form():
    """j = 2: S must be (x2 - x1)^2 / 2, the population S of two samples."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, b = rng.normal(size=2) * 10
        _, s = oracle.chan_stream([a, b])
        assert s == pytest.approx((b - a) ** 2 / 2, rel=1e-13, abs=1e-13)


def test_eq1_as_printed_is_not_the_variance():
    """The printed update (no square) disagrees with the definition, which is
    why the oracle reads Eq. 1 with the square (planted on the CPU)."""
    x = np.array([1.0, 2.0, 4.0])
    t, s = 0.0, 0.0
    for j, xj in enumerate(x, start=1):
        t += xj
        if j > 1:
            s += (j * xj - t) / (j * (j - 1))
    assert abs(s - 42 / 9) > 1.0
    _, s_ok = oracle.chan_stream(x)
    assert s_ok == pytest.approx(42 / 9, rel=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 4097])
def test_chan_stream_equals_twopass(n):
    rng = np.random.default_rng(n)
    x = rng.normal(100.0, 12.0, size=n)
    t, s = oracle.chan_stream(x)
    mu, sd = oracle.twopass(x)
    assert t / n == pytest.approx(np.mean(x), rel=1e-13)
    assert mu == pytest.approx(np.mean(x), rel=1e-13)
    assert math.sqrt(s / n) == pytest.approx(np.std(x), rel=1e-11, abs=1e-12)
    assert sd == pytest.approx(np.std(x), rel=1e-12, abs=1e-13)


def test_chan_merge_any_split_and_tree():
    """Eq. 2: every split point and a random merge tree give the stream result."""
    rng = np.random.default_rng(11)
    x = rng.normal(-3.0, 2.5, size=257)
    T0, S0 = oracle.chan_stream(x)
    for cut in [1, 2, 100, 128, 256]:
        Ta, Sa = oracle.chan_stream(x[:cut])
        Tb, Sb = oracle.chan_stream(x[cut:])
        T, S = oracle.chan_merge(cut, Ta, Sa, x.size - cut, Tb, Sb)
        assert T == pytest.approx(T0, rel=1e-13, abs=1e-12)
        assert S == pytest.approx(S0, rel=1e-12)
    # random binary tree over random-size pieces
    cuts = np.sort(rng.choice(np.arange(1, x.size), size=20, replace=False))
    parts = [(p.size, *oracle.chan_stream(p)) for p in np.split(x, cuts)]
    while len(parts) > 1:
        k = int(rng.integers(0, len(parts) - 1))
        (m, Ta, Sa), (n, Tb, Sb) = parts[k], parts[k + 1]
        parts[k: k + 2] = [(m + n, *oracle.chan_merge(m, Ta, Sa, n, Tb, Sb))]
    n, T, S = parts[0]
    assert n == x.size
    assert T == pytest.approx(T0, rel=1e-13, abs=1e-12)
    assert S == pytest.approx(np.var(x) * x.size, rel=1e-12)


def test_chan_merge_empty_side():
    assert oracle.chan_merge(0, 0, 0, 3, 6.0, 2.0) == (6.0, 2.0)
    assert oracle.chan_merge(3, 6.0, 2.0, 0, 0, 0) == (6.0, 2.0)


def test_plane_msd_ramp_closed_form():
    """x = a + b i: mean a + b (n-1)/2, variance b^2 (n^2 - 1)/12."""
    n_dm, n = 3, 5000
    a, b = 7.0, 0.25
    row = a + b * np.arange(n)
    plane = np.tile(row, (n_dm, 1)).astype(np.float32)
    for fn in (lambda p: oracle.plane_msd(p, oracle.SCOPE_PER_ROW),
               lambda p: oracle.plane_msd_chan(p, 777, oracle.SCOPE_PER_ROW)):
        mean, sd = fn(plane)
        assert np.allclose(mean, a + b * (n - 1) / 2, rtol=1e-13)
        assert np.allclose(sd, math.sqrt(b * b * (n * n - 1) / 12), rtol=1e-12)


def test_plane_msd_constant_is_zero_sd():
    plane = np.full((4, 999), 3.5, dtype=np.float32)
    mean, sd = oracle.plane_msd(plane)
    assert mean[0] == 3.5 and sd[0] == 0.0
    mean, sd = oracle.plane_msd_chan(plane, 64)
    assert mean[0] == 3.5 and sd[0] == 0.0


@pytest.mark.parametrize("block", [1, 7, 256, 10 ** 6])
def test_plane_block_scheme_equals_definition(block):
    """The two-kernel block scheme of Sec. 2.1 equals numpy's mean / std."""
    rng = np.random.default_rng(block)
    plane = rng.normal(100.0, 12.0, size=(6, 3001)).astype(np.float32)
    ref = plane.astype(np.float64)
    for scope in (oracle.SCOPE_GLOBAL, oracle.SCOPE_PER_ROW):
        m1, s1 = oracle.plane_msd(plane, scope)
        m2, s2 = oracle.plane_msd_chan(plane, block, scope)
        if scope == oracle.SCOPE_GLOBAL:
            mr, sr = np.array([ref.mean()]), np.array([ref.std()])
        else:
            mr, sr = ref.mean(axis=1), ref.std(axis=1)
        assert np.allclose(m1, mr, rtol=1e-13) and np.allclose(m2, mr, rtol=1e-12)
        assert np.allclose(s1, sr, rtol=1e-12) and np.allclose(s2, sr, rtol=1e-10)


def test_ragged_stride_is_ignored():
    """Samples past n_samp (here NaN) never enter any oracle result."""
    rng = np.random.default_rng(3)
    full = rng.normal(size=(3, 130)).astype(np.float32)
    padded = np.full((3, 160), np.nan, dtype=np.float32)
    padded[:, :130] = full
    p = oracle.Plane(padded, n_samp=130)
    m, s = oracle.plane_msd(p)
    assert m[0] == pytest.approx(full.astype(np.float64).mean(), rel=1e-13)
    assert s[0] == pytest.approx(full.astype(np.float64).std(), rel=1e-12)
    b = oracle.boxcar_sums(p, 5)
    assert np.isfinite(b[:, :126]).all() and np.isnan(b[:, 126:]).all()


# --------------------------------------------------------- dequantisation

def test_half_and_bf16_decoding_match_library_conversions():
    import torch
    bits = np.arange(0, 65536, dtype=np.uint32).astype(np.uint16)
    bits = bits[(bits & 0x7C00) != 0x7C00]  # drop inf / nan patterns
    plane = bits.reshape(1, -1)
    got = oracle.Plane(plane, dtype="f16").values()[0]
    want = bits.view(np.float16).astype(np.float64)
    assert np.array_equal(got, want)
    b2 = np.arange(0, 65536, dtype=np.uint32).astype(np.uint16)
    b2 = b2[(b2 & 0x7F80) != 0x7F80]
    got = oracle.Plane(b2.reshape(1, -1), dtype="bf16").values()[0]
    want = torch.from_numpy(b2.view(np.int16)).view(torch.bfloat16).double().numpy()
    assert np.array_equal(got, want)


def test_scale_offset_is_fp32_fma():
    q = np.array([[1.0, 2.0, 3.0]], dtype=np.float16)
    sc = np.array([0.1], np.float32)
    off = np.array([5.0], np.float32)
    got = oracle.Plane(q.view(np.uint16), dtype="f16", scale=sc, offset=off).values()[0]
    # an FP32 fused multiply-add rounds once: emulate with float64 then round
    want = (np.float64(sc[0]) * q.astype(np.float64)[0] + np.float64(off[0])).astype(np.float32)
    assert np.array_equal(got, want.astype(np.float64))


# ------------------------------------------------------------ Sec. 2.2, Eq. 4/5

def test_sigma_table_hand_values():
    rows = _rows("eq5_sigma_table.txt")
    widths = [int(r[0]) for r in rows]
    cols = np.array([[float(v) for v in r[1:]] for r in rows])
    assert np.allclose(oracle.sigma_table(oracle.SIGMA_SQRTN, 1.0, widths), cols[:, 0],
                       rtol=1e-15)
    assert np.allclose(oracle.sigma_table(oracle.SIGMA_LINEAR, 1.0, widths, 10.0, 4),
                       cols[:, 1], rtol=1e-15)
    assert np.allclose(oracle.sigma_table(oracle.SIGMA_LINEAR_EXCESS, 1.0, widths, 10.0, 4),
                       cols[:, 2], rtol=1e-15)


def test_eq5_endpoints():
    """E reading: exact at N = 1 and N = Nmax.  L as printed: sigma at N = 1 and
    sigma_Nmax + sqrt(Nmax) sigma at N = Nmax."""
    sd, sdn, nmax = 1.7, 30.0, 256
    e = oracle.sigma_table(oracle.SIGMA_LINEAR_EXCESS, sd, [1, nmax], sdn, nmax)
    l_ = oracle.sigma_table(oracle.SIGMA_LINEAR, sd, [1, nmax], sdn, nmax)
    assert e[0] == pytest.approx(sd) and e[1] == pytest.approx(sdn)
    assert l_[0] == pytest.approx(sd) and l_[1] == pytest.approx(sdn + 16 * sd)


def test_sqrtN_on_gaussian_noise():
    """Eq. 3/4: the empirical sd of B_N on N(0, sd^2) noise is sqrt(N) sd within
    3 standard errors (about n/N independent windows)."""
    rng = np.random.default_rng(42)
    sd = 2.0
    plane = rng.normal(0.0, sd, size=(4, 50000)).astype(np.float32)
    for N in (1, 4, 16, 64):
        b = oracle.boxcar_sums(plane, N)
        emp = np.nanstd(b)
        n_eff = plane.size / N
        se = sd * math.sqrt(N) / math.sqrt(2 * n_eff)
        assert abs(emp - sd * math.sqrt(N)) < 3 * se + 1e-3 * sd


def test_sd_nmax_closed_forms():
    """Alternating +-1: B_Nmax is 0 for even Nmax (sd 0) and +-1 for odd (sd 1).
    Ramp b i: B_Nmax(i) = b Nmax i + const, sd = b Nmax sqrt((m^2 - 1)/12),
    m = n - Nmax + 1 windows."""
    alt = np.tile(np.array([1.0, -1.0], np.float32), (2, 50))
    assert oracle.plane_sd_nmax(alt, 4)[0] == pytest.approx(0.0, abs=1e-15)
    assert oracle.plane_sd_nmax(alt, 5)[0] == pytest.approx(1.0, rel=1e-14)
    n, nm, b = 300, 16, 0.5
    ramp = (b * np.arange(n, dtype=np.float64)).astype(np.float32).reshape(1, -1)
    m = n - nm + 1
    want = b * nm * math.sqrt((m * m - 1) / 12)
    assert oracle.plane_sd_nmax(ramp, nm)[0] == pytest.approx(want, rel=1e-12)


# ------------------------------------------------------------ Sec. 2.3, boxcars

def test_boxcar_sums_constant_ramp_spike():
    n = 200
    const = np.full((2, n), 3.0, np.float32)
    for w in (1, 2, 7, 64, 200):
        b = oracle.boxcar_sums(const, w)
        assert np.array_equal(b[:, : n - w + 1], np.full((2, n - w + 1), 3.0 * w))
        assert np.isnan(b[:, n - w + 1:]).all()
    a, s = 5.0, 2.0
    ramp = (a + s * np.arange(n)).astype(np.float32).reshape(1, -1)
    for w in (1, 3, 16, 50):
        i = np.arange(n - w + 1)
        want = w * a + s * (w * i + w * (w - 1) / 2)
        assert np.array_equal(oracle.boxcar_sums(ramp, w)[0, : n - w + 1], want)
    spike = np.zeros((1, n), np.float32)
    spike[0, 100] = 9.0
    for w in (1, 5, 33):
        b = oracle.boxcar_sums(spike, w)[0, : n - w + 1]
        i = np.arange(n - w + 1)
        want = np.where((i <= 100) & (100 <= i + w - 1), 9.0, 0.0)
        assert np.array_equal(b, want)


def _brute_force(x, mu, sigma_by_width, widths):
    """All (start, width) SNRs from numpy cumulative sums; the winner is the
    first maximum over [width 1, listed widths...] (np.argmax's first index),
    which is what a strict '>' scan in ascending width order selects."""
    n = x.size
    c = np.concatenate([[0.0], np.cumsum(x)])
    cols = [1] + list(widths)
    sig = [sigma_by_width[1]] + [sigma_by_width[w] for w in widths]
    snr = np.full((n, len(cols)), -np.inf)
    for k, (w, s) in enumerate(zip(cols, sig)):
        i = np.arange(0, n - w + 1)
        snr[i, k] = (c[i + w] - c[i] - w * mu) / s
    arg = np.argmax(snr, axis=1)
    return snr[np.arange(n), arg], np.array(cols)[arg]


@pytest.mark.parametrize("seed", range(12))
def test_algorithm1_against_brute_force(seed):
    """Tiny integer inputs with exact ties, random width subsets of 1..8."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 65))
    x = rng.integers(-3, 4, size=(2, n)).astype(np.float32)
    all_w = np.arange(1, 9)
    widths = np.sort(rng.choice(all_w, size=int(rng.integers(1, 9)), replace=False))
    mu, sd = 0.25, 1.5
    sig = {w: math.sqrt(w) * sd for w in range(1, 9)}
    tab = oracle.sigma_table(oracle.SIGMA_SQRTN, sd, widths)
    best, win = oracle.boxcar_snr(x, [mu], [sd], tab, widths)
    for r in range(2):
        bb, ww = _brute_force(x[r].astype(np.float64), mu, sig, widths)
        assert np.allclose(best[r], bb, rtol=1e-13, atol=1e-13)
        assert np.array_equal(win[r], ww)


@pytest.mark.parametrize("seed", range(6))
def test_listed_widths_only_against_brute_force(seed):
    """start_w1=False (decimated levels): the winner among the listed widths
    alone, -inf / width 0 where no listed width fits."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 40))
    x = rng.integers(-3, 4, size=(1, n)).astype(np.float32)
    widths = np.sort(rng.choice(np.arange(2, 9), size=int(rng.integers(1, 6)), replace=False))
    mu, sd = -0.5, 2.0
    tab = oracle.sigma_table(oracle.SIGMA_SQRTN, sd, widths)
    best, win = oracle.boxcar_snr(x, [mu], [sd], tab, widths, start_w1=False)
    c = np.concatenate([[0.0], np.cumsum(x[0].astype(np.float64))])
    for i in range(n):
        fits = [w for w in widths if i + w <= n]
        if not fits:
            assert best[0, i] == -np.inf and win[0, i] == 0
            continue
        snr = [(c[i + w] - c[i] - w * mu) / (math.sqrt(w) * sd) for w in fits]
        k = int(np.argmax(snr))
        assert best[0, i] == pytest.approx(snr[k], rel=1e-13, abs=1e-13)
        assert win[0, i] == fits[k]


def test_tie_rule_smallest_width_wins():
    """x = (1, 0, 0, ...) with sigma_w = 1 for all w: every width has SNR 1 at
    sample 0, and strict '>' keeps width 1."""
    x = np.zeros((1, 10), np.float32)
    x[0, 0] = 1.0
    widths = [1, 2, 3, 4]
    best, win = oracle.boxcar_snr(x, [0.0], [1.0], np.ones(4), widths)
    assert best[0, 0] == 1.0 and win[0, 0] == 1


def test_figure1_tophat_response():
    """Figure 1: a top-hat of width W, amplitude a (mu = 0, sigma = 1) gives
    SNR(N) = a min(N, W) / sqrt(N) at its leading sample; the best is N = W."""
    a, n = 3.0, 256
    widths = list(range(1, 65))
    for W in (1, 5, 16, 40):
        x = np.zeros((1, n), np.float32)
        x[0, 50:50 + W] = a
        tab = oracle.sigma_table(oracle.SIGMA_SQRTN, 1.0, widths)
        best, win = oracle.boxcar_snr(x, [0.0], [1.0], tab, widths)
        assert win[0, 50] == W
        assert best[0, 50] == pytest.approx(a * math.sqrt(W), rel=1e-14)
        for N in (1, 3, 64):
            b = oracle.boxcar_sums(x, N)[0, 50]
            assert b / math.sqrt(N) == pytest.approx(a * min(N, W) / math.sqrt(N))


def test_row_end_truncates_width_set():
    """At the last samples only widths w <= n_samp - i are evaluated."""
    x = np.zeros((1, 8), np.float32)
    x[0, 6:] = 5.0
    widths = [1, 2, 4]
    tab = oracle.sigma_table(oracle.SIGMA_SQRTN, 1.0, widths)
    best, win = oracle.boxcar_snr(x, [0.0], [1.0], tab, widths)
    assert win[0, 7] == 1 and best[0, 7] == 5.0
    assert win[0, 6] == 2 and best[0, 6] == pytest.approx(10 / math.sqrt(2))
    assert win[0, 4] == 4 and best[0, 4] == pytest.approx(10 / 2)


# ------------------------------------------------------------ Sec. 2.4

def test_threshold_inclusive():
    thr = 6.0
    best = np.array([[thr, np.nextafter(thr, -np.inf), thr + 1, -thr]])
    width = np.array([[1, 2, 3, 4]], np.int32)
    c = oracle.threshold(best, width, thr, row0=5)
    assert list(c["sample"]) == [0, 2] and list(c["dm"]) == [5, 5]
    assert list(c["width"]) == [1, 3]


def test_search_finds_injected_tophats():
    """Statistical check, not parity: the plain FP32 case's pulses are found
    at their leading sample with SNR near the target and the matching width."""
    import synth
    sp = synth.plain_tophat(16, 8192, device="cpu", seed=77)
    x = synth.to_host_numpy(sp.data)
    cands, best, win, _ = oracle.search(x, list(range(1, 33)), 6.0)
    for p in sp.pulses:
        sel = cands[(cands["dm"] == p.dm) & (abs(cands["sample"] - p.sample) <= 2)]
        assert sel.size > 0
        top = sel[np.argmax(sel["snr"])]
        assert abs(top["snr"] - p.snr) < 4.0
        assert abs(int(top["width"]) - p.width) <= max(2, p.width // 3)


@pytest.mark.parametrize("seed", range(8))
def test_search_end_to_end_against_brute_force(seed):
    """The four steps composed, on tiny planes, against an independent numpy
    statement of each: mean and population sd (np.mean / np.std over the
    scope), sigma_Nmax as np.std of every full Nmax-sample window sum pooled
    over the scope, sigma_w of Eq. 4 or Eq. 5 (both readings), Algorithm 1 by
    brute force, and the inclusive threshold."""
    rng = np.random.default_rng(700 + seed)
    n_dm, n = int(rng.integers(1, 4)), int(rng.integers(12, 80))
    x = (rng.normal(0.0, 1.0, size=(n_dm, n)) + rng.normal(0.0, 0.3, size=(n_dm, 1))
         ).astype(np.float32)
    x[:, int(rng.integers(0, n - 4)):][:, :4] += 3.0          # a small pulse
    mode = seed % 3
    scope = (seed // 3) % 2
    widths = np.sort(rng.choice(np.arange(2, 11), size=int(rng.integers(1, 6)),
                                replace=False)).astype(np.int32)
    thr = 2.0
    cands, best, win, (mean, sd, sdn, _) = oracle.search(x, widths, thr, mode, scope)

    x64 = x.astype(np.float64)
    groups = [x64] if scope == oracle.SCOPE_GLOBAL else [x64[r:r + 1] for r in range(n_dm)]
    nmax = int(widths[-1])
    want_b, want_w = np.zeros((n_dm, n)), np.zeros((n_dm, n), np.int64)
    for e, g in enumerate(groups):
        mu, s = float(np.mean(g)), float(np.std(g))
        assert mean[e] == pytest.approx(mu, abs=1e-12) and sd[e] == pytest.approx(s, rel=1e-12)
        if mode:
            win_sums = np.lib.stride_tricks.sliding_window_view(g, nmax, axis=1).sum(axis=2)
            sn = float(np.std(win_sums))
            assert sdn[e] == pytest.approx(sn, rel=1e-10)
        sig = {}
        for w in [1] + list(widths):
            if mode == 0:
                sig[w] = math.sqrt(w) * s
            elif mode == 1:
                sig[w] = math.sqrt(w) * s + (w - 1) * sn / (nmax - 1)
            else:
                sig[w] = math.sqrt(w) * s + (w - 1) * (sn - math.sqrt(nmax) * s) / (nmax - 1)
        rows = range(n_dm) if scope == oracle.SCOPE_GLOBAL else [e]
        for r in rows:
            want_b[r], want_w[r] = _brute_force(x64[r], mu, sig, widths)
    assert np.allclose(best, want_b, rtol=1e-10, atol=1e-12)
    assert np.array_equal(win, want_w)
    keep = np.argwhere(want_b >= thr)
    assert [(int(c["dm"]), int(c["sample"])) for c in cands] == [(int(r), int(i)) for r, i in keep]
    assert np.array_equal(cands["width"], want_w[want_b >= thr])


def _components(best, width, thr, gap):
    """Clusters as connected components of the graph that links any two
    candidates of a row at most `gap` samples apart (union-find over every
    pair): a statement independent of the oracle's sequential scan."""
    out = []
    for r in range(best.shape[0]):
        idx = [i for i in range(best.shape[1]) if best[r, i] >= thr]
        parent = {i: i for i in idx}

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a
        for a in idx:
            for b in idx:
                if a < b and b - a <= gap:
                    parent[find(b)] = find(a)
        comps = {}
        for i in idx:
            comps.setdefault(find(i), []).append(i)
        for m in comps.values():
            vals = [best[r, i] for i in m]
            k = int(np.argmax(vals))           # the first of equal maxima
            out.append((r, m[0], m[-1], m[k], vals[k], int(width[r, m[k]]), len(m)))
    return sorted(out)


@pytest.mark.parametrize("seed", range(10))
def test_cluster_rows_against_components(seed):
    rng = np.random.default_rng(900 + seed)
    n_dm, n = int(rng.integers(1, 4)), int(rng.integers(1, 90))
    best = rng.integers(0, 10, size=(n_dm, n)).astype(np.float64)
    best[rng.random((n_dm, n)) < 0.05] = np.nan
    width = rng.integers(1, 300, size=(n_dm, n))
    thr, gap = float(rng.integers(4, 9)), int(rng.integers(1, 6))
    c = oracle.cluster_rows(best, width, thr, gap)
    got = sorted((int(x["dm"]), int(x["first"]), int(x["last"]), int(x["peak_sample"]),
                  float(x["peak_snr"]), int(x["peak_width"]), int(x["members"])) for x in c)
    assert got == _components(best, width, thr, gap)
    # the members are exactly the candidates
    assert int(c["members"].sum()) == int(np.sum(best >= thr))


def test_cluster_rows_closed_forms():
    """Isolated spikes further apart than the gap: one cluster each; a
    contiguous run: one cluster spanning it, peaked at its first maximum; a
    gap of exactly max_gap joins, max_gap + 1 splits; row0 offsets dm."""
    best = np.zeros((2, 40))
    best[0, [3, 10, 20]] = 7.0
    best[1, 5:12] = [6, 8, 9, 9, 7, 6, 6]
    w = np.arange(80).reshape(2, 40)
    c = oracle.cluster_rows(best, w, 6.0, 4, row0=100)
    assert list(c["dm"]) == [100, 100, 100, 101]
    assert list(c["first"]) == [3, 10, 20, 5] and list(c["last"]) == [3, 10, 20, 11]
    assert list(c["members"]) == [1, 1, 1, 7]
    assert c["peak_sample"][3] == 7 and c["peak_snr"][3] == 9 and c["peak_width"][3] == 47
    x = np.zeros((1, 20))
    x[0, [2, 5, 9]] = 8.0                       # gaps of 3 and 4
    assert len(oracle.cluster_rows(x, np.ones((1, 20)), 8.0, 3)) == 2
    assert len(oracle.cluster_rows(x, np.ones((1, 20)), 8.0, 4)) == 1
    assert len(oracle.cluster_rows(np.full((1, 5), np.nan), np.ones((1, 5)), 0.0, 1)) == 0


def test_snr_at_matches_closed_form():
    """One-pair SNR: a ramp's window sum is closed-form; past the row end NaN."""
    n, a, b = 50, 2.0, 0.5
    ramp = (a + b * np.arange(n)).astype(np.float32).reshape(1, -1)
    i, w, mu, sw = 7, 9, 1.25, 3.0
    want = (w * a + b * (w * i + w * (w - 1) / 2) - w * mu) / sw
    assert oracle.snr_at(ramp, 0, i, w, mu, sw) == pytest.approx(want, rel=1e-15)
    assert math.isnan(oracle.snr_at(ramp, 0, 45, 9, mu, sw))


# ------------------------------------------------------------ streaming reading

def _stream_brute(chunks, widths, thr, per_row):
    """Independent statement of the streaming reading, by enumeration: every
    start i is scored by the first push whose data end e_k satisfies
    i + wmax <= e_k (else at the end, e = n, with the row-end truncation),
    with the population mean / sd (numpy) of all samples before e."""
    x = np.concatenate([np.asarray(c, np.float64) for c in chunks], axis=1)
    n_dm, n = x.shape
    wmax = max(widths)
    ends = np.cumsum([c.shape[1] for c in chunks])
    rows = []
    for i in range(n):
        e = next((int(t) for t in ends if i + wmax <= t), n)
        for d in range(n_dm):
            seen = x[d, :e] if per_row else x[:, :e]
            mu, sd = seen.mean(), seen.std()
            best, win = (x[d, i] - mu) / sd, 1
            for w in widths:
                if i + w > e:
                    break
                s = (x[d, i:i + w].sum() - w * mu) / (math.sqrt(w) * sd)
                if s > best:
                    best, win = s, w
            if best >= thr:
                rows.append((d, i, best, win))
    return sorted(rows)


@pytest.mark.parametrize("per_row", [False, True])
def test_stream_replay_brute_force(per_row):
    rng = np.random.default_rng(5)
    x = rng.normal(0.0, 1.0, (3, 90)).astype(np.float32)
    x[1, 40:46] += 2.5
    x[2, 86:90] += 3.0                      # pulse in the tail: found by the flush
    chunks = [x[:, :7], x[:, 7:8], x[:, 8:40], x[:, 40:41], x[:, 41:90]]
    widths, thr = [1, 2, 3, 5, 8], 2.0
    got = np.concatenate(oracle.stream_replay(chunks, widths, thr, scope=int(per_row)))
    got.sort(order=["dm", "sample"])
    want = _stream_brute(chunks, widths, thr, per_row)
    assert len(got) == len(want) > 0
    for g, (d, i, s, w) in zip(got, sorted(want)):
        assert (g["dm"], g["sample"], g["width"]) == (d, i, w)
        assert g["snr"] == pytest.approx(s, rel=1e-12, abs=1e-12)


def test_stream_replay_single_chunk_is_one_shot():
    """One chunk then the flush covers every start once with the MSD of the
    whole plane: the same list as the one-shot search."""
    import synth
    sp = synth.plain_tophat(8, 3000, device="cpu", seed=9)
    x = synth.to_host_numpy(sp.data)
    w = list(range(1, 33))
    one, *_ = oracle.search(x, w, 6.0)
    rep = oracle.stream_replay([x], w, 6.0)
    assert len(rep) == 2
    allc = np.concatenate(rep)
    allc.sort(order=["dm", "sample"])
    assert np.array_equal(one, allc)


def test_threshold_plane_cases_and_list_agreement():
    """Sec. 2.4 on the plane: kept iff >= f_T (exactly f_T kept, the float
    below it and NaN zeroed); the kept entries are the candidate list."""
    thr = 6.5
    best = np.array([[thr, np.nextafter(thr, -np.inf), np.nan, 9.0, -7.0, 0.0]])
    width = np.array([[3, 4, 5, 6, 7, 8]], np.int32)
    b, w = oracle.threshold_plane(best, width, thr)
    assert b.tolist() == [[thr, 0.0, 0.0, 9.0, 0.0, 0.0]]
    assert w.tolist() == [[3, 0, 0, 6, 0, 0]]
    rng = np.random.default_rng(4)
    best = rng.normal(0, 3, (7, 300))
    width = rng.integers(1, 64, best.shape).astype(np.int32)
    b, w = oracle.threshold_plane(best, width, 4.0)
    c = oracle.threshold(best, width, 4.0)
    nz = np.argwhere(b != 0)
    assert [tuple(x) for x in nz] == list(zip(c["dm"], c["sample"]))
    assert np.array_equal(b[b != 0], c["snr"]) and np.array_equal(w[b != 0], c["width"])


# ------------------------------------------------------- decimation in time

def test_decimate_ramp_closed_form():
    n, a, b = 40, 3.0, 0.5
    x = (a + b * np.arange(n)).astype(np.float32).reshape(1, -1)
    for level in range(4):
        m = 1 << level
        j = np.arange(n >> level)
        want = m * a + b * (m * m * j + m * (m - 1) / 2)
        assert np.array_equal(oracle.decimate(x, level)[0], want)


def test_decimated_boxcar_is_the_plain_boxcar_at_aligned_starts():
    """B^l_w(j) on the decimated series = B_{w 2^l}(j 2^l) on the native one
    (integer data: every sum exact)."""
    rng = np.random.default_rng(8)
    x = rng.integers(-50, 50, (3, 203)).astype(np.float32)
    for level in (1, 2, 3):
        xl = oracle.decimate(x, level).astype(np.float32)
        for w in (1, 3, 5):
            bl = oracle.boxcar_sums(xl, w)
            bn = oracle.boxcar_sums(x, w << level)
            n = xl.shape[1] - w + 1
            assert np.array_equal(bl[:, :n], bn[:, :(n << level):(1 << level)])


def test_search_decimated_level0_is_the_plain_search():
    import synth
    sp = synth.plain_tophat(6, 5000, device="cpu", seed=12)
    x = synth.to_host_numpy(sp.data)
    widths = list(range(1, 33))
    one, *_ = oracle.search(x, widths, 6.0)
    got, msds = oracle.search_decimated(x, [(0, widths)], 6.0)
    assert np.array_equal(got["dm"], one["dm"]) and np.array_equal(got["sample"], one["sample"])
    assert np.array_equal(got["width"], one["width"]) and np.array_equal(got["snr"], one["snr"])


def test_search_decimated_noise_scaling_and_aligned_tophat():
    """On N(0,1) noise the level-l sd is sqrt(2^l) (3 standard errors); a
    top-hat of 2^l w samples starting at a multiple of 2^l is found at level l
    with width 2^l w and an SNR near its plain matched SNR."""
    rng = np.random.default_rng(9)
    x = rng.normal(0, 1, (4, 1 << 16)).astype(np.float32)
    level, w = 3, 8               # native width 64
    t0, snr = 8 * 1000, 25.0
    x[2, t0:t0 + (w << level)] += snr / np.sqrt(w << level)
    got, msds = oracle.search_decimated(x, [(0, list(range(1, 17))), (level, [4, 8, 16])], 7.0)
    n_l = x.size >> level
    assert abs(msds[1][1] / np.sqrt(1 << level) - 1) < 3 / np.sqrt(2 * n_l)
    hit = got[(got["dm"] == 2) & (got["level"] == level)]
    top = hit[np.argmax(hit["snr"])]
    assert top["sample"] == t0 and top["width"] == w << level
    assert abs(top["snr"] - snr) < 4.0


def test_cluster_rows_signed_zeros():
    """-0.0 and +0.0 are equal: the earlier stays the peak whichever comes first."""
    best = np.array([[-1.0, -0.0, 0.0, -1.0, 0.0, -0.0]])
    width = np.arange(1, 7).reshape(1, 6)
    c = oracle.cluster_rows(best, width, 0.0, 1)
    assert list(c["first"]) == [1, 4] and list(c["peak_sample"]) == [1, 4]
    assert list(c["peak_width"]) == [2, 5]


# ------------------------------------------------------------ de-dispersion

def test_dedisperse_impulse_response():
    """One unit sample in channel c0 at time T shows up in DM trial d exactly
    at t = T - delay[d, c0] (and nowhere else)."""
    rng = np.random.default_rng(3)
    n_chan, n_samp, n_out = 5, 60, 45
    delays = rng.integers(0, n_samp - n_out + 1, size=(4, n_chan)).astype(np.int32)
    x = np.zeros((n_chan, n_samp), dtype=np.float32)
    c0, T = 2, 30
    x[c0, T] = 1.0
    out = oracle.dedisperse(x, delays, n_out)
    for d in range(4):
        want = np.zeros(n_out)
        t = T - delays[d, c0]
        if 0 <= t < n_out:
            want[t] = 1.0
        assert np.array_equal(out[d], want)


def test_dedisperse_zero_delays_sum_channels():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((7, 40)).astype(np.float32)
    out = oracle.dedisperse(x, np.zeros((2, 7), np.int32), 40)
    assert np.allclose(out[0], x.astype(np.float64).sum(axis=0), rtol=0, atol=1e-12)
    assert np.array_equal(out[0], out[1])


def test_dedisperse_against_fancy_indexing():
    """An independent statement of the definition by numpy gathers."""
    rng = np.random.default_rng(5)
    n_chan, n_samp, n_out, n_dm = 6, 80, 50, 9
    x = rng.standard_normal((n_chan, n_samp)).astype(np.float32)
    delays = rng.integers(0, n_samp - n_out + 1, size=(n_dm, n_chan)).astype(np.int32)
    t = np.arange(n_out)
    want = np.stack([x[np.arange(n_chan)[:, None], t[None, :] + delays[d][:, None]]
                     .astype(np.float64).sum(axis=0) for d in range(n_dm)])
    assert np.allclose(oracle.dedisperse(x, delays, n_out), want, rtol=0, atol=1e-12)


def test_dedisperse_restores_a_dispersed_pulse():
    """A noise-free top-hat dispersed along trial k: trial k holds n_chan * amp
    over the pulse's samples; other trials hold less at every sample."""
    fb = synth.filterbank(16, 4000, dms=np.linspace(0, 30, 8), pulses=((5, 700, 6, 1.5),),
                          sd=0.0)
    out = oracle.dedisperse(synth.to_host_numpy(fb.data), fb.delays, fb.n_out)
    want = np.zeros(fb.n_out)
    want[700:706] = 16 * 1.5
    assert np.allclose(out[5], want)
    assert np.all(np.delete(out, 5, axis=0).max(axis=1) < 16 * 1.5)


def test_dedisperse_rejects_out_of_range_delays():
    x = np.zeros((3, 20), dtype=np.float32)
    with pytest.raises(ValueError):
        oracle.dedisperse(x, np.array([[0, 6, 0]], np.int32), 15)
    with pytest.raises(ValueError):
        oracle.dedisperse(x, np.array([[0, -1, 0]], np.int32), 10)
