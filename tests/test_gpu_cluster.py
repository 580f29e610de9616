"""Per-DM clustering of the candidates (spd_cluster_rows) against the FP64
oracle's clustering of the same seeded SNR planes: index work, so every
field of every record must be equal."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FIELDS = ["dm", "first", "last", "peak_sample", "peak_width", "members"]


@pytest.fixture(scope="module")
def spd():
    import paper_1611_09704_gb300 as m
    m.build()
    m.load()
    return m


def _sorted(c):
    return np.sort(c, order=["dm", "first"])


def _compare(got, want):
    got, want = _sorted(got), _sorted(want)
    assert got.size == want.size
    for f in FIELDS:
        assert np.array_equal(got[f], want[f]), f
    assert np.array_equal(got["peak_snr"].astype(np.float32), want["peak_snr"].astype(np.float32))


@pytest.mark.parametrize("n_dm,n_samp,stride,thr,gap", [
    (5, 1000, None, 7.0, 1),       # adjacent samples only
    (3, 4099, 4112, 8.0, 7),       # ragged length, NaN padding past the row end
    (9, 777, None, 9.0, 300),      # gaps spanning 32- and 256-sample steps
    (2, 33, None, 0.0, 2),         # every non-NaN sample a candidate
    (17, 256, None, 9.0, 40),      # one load round per row, more rows than a CTA holds
])
def test_clusters_match_oracle(spd, n_dm, n_samp, stride, thr, gap):
    snr, width = synth.snr_plane(n_dm, n_samp, stride=stride, device=DEV, seed=n_samp + gap)
    out, res = spd.cluster_rows(snr, width, thr, gap, 1 << 16, n_samp=n_samp)
    count, status = spd.read_result(res)
    assert status == 0
    got = spd.clusters_to_numpy(out, count)
    s = synth.to_host_numpy(snr)[:, :n_samp]
    w = synth.to_host_numpy(width).view(np.uint16)[:, :n_samp]
    want = oracle.cluster_rows(s, w, thr, gap)
    assert count == want.size and count > 0
    _compare(got, want)


def test_capacity_keeps_the_exact_count(spd):
    snr, width = synth.snr_plane(4, 3000, device=DEV, seed=11)
    s = synth.to_host_numpy(snr)
    w = synth.to_host_numpy(width).view(np.uint16)
    want = oracle.cluster_rows(s, w, 8.0, 3)
    cap = want.size // 3
    out, res = spd.cluster_rows(snr, width, 8.0, 3, cap)
    count, status = spd.read_result(res)
    assert count == want.size and status == 0
    got = spd.clusters_to_numpy(out, count)
    assert got.size == cap
    keys = {tuple(int(r[f]) for f in FIELDS) for r in want}
    assert all(tuple(int(r[f]) for f in FIELDS) in keys for r in got)


def test_clusters_of_a_search_plane_hold_every_candidate(spd):
    """On the GPU's own SNR plane of a small SKA-like search: the members of
    all clusters are exactly the candidates spd_threshold_candidates lists,
    each candidate inside its row's cluster extent (properties, any size)."""
    widths = list(range(1, 17)) + list(range(24, 129, 8))
    sp = synth.ska_like(8, 40000, n_pulses=6, device=DEV, seed=12)
    m = spd.msd(sp.data)
    snr, w = spd.boxcar_snr(sp.data, m, widths)
    cand, cres = spd.threshold_candidates(snr, w, 7.0, 1 << 20)
    n_cand, _ = spd.read_result(cres)
    out, res = spd.cluster_rows(snr, w, 7.0, 16, 1 << 18)
    n_cl, st = spd.read_result(res)
    assert st == 0 and 0 < n_cl <= n_cand
    cl = spd.clusters_to_numpy(out, n_cl)
    assert int(cl["members"].sum()) == n_cand
    c = spd.candidates_to_numpy(cand, n_cand)
    for r in range(8):
        rc = np.sort(c[c["dm"] == r]["sample"])
        rl = _sorted(cl[cl["dm"] == r])
        inside = np.zeros(rc.size, bool)
        for k in rl:
            sel = (rc >= k["first"]) & (rc <= k["last"])
            assert int(sel.sum()) == int(k["members"])
            inside |= sel
        assert inside.all()


def test_empty_and_bad_arguments(spd):
    snr, width = synth.snr_plane(3, 100, device=DEV, seed=1)
    out, res = spd.cluster_rows(snr[:0], width[:0], 5.0, 2, 16)
    assert spd.read_result(res) == (0, 0)
    out, res = spd.cluster_rows(snr, width, 5.0, 2, 16, n_samp=0)
    assert spd.read_result(res) == (0, 0)
    with pytest.raises(spd.SpdError):
        spd.cluster_rows(snr, width, 5.0, 0, 16)
    with pytest.raises(spd.SpdError):
        spd.cluster_rows(snr, width, float("nan"), 2, 16)
    torch.cuda.synchronize()


def test_signed_zeros_keep_the_earliest_peak(spd):
    """-0.0 and +0.0 are equal SNRs: with a threshold of 0 the earlier of the
    two stays the cluster's peak (strict ">" keeps the first among equals)."""
    n = 64
    s = np.full((2, n), -1.0, dtype=np.float32)
    s[0, 10], s[0, 11] = -0.0, 0.0          # -0.0 first
    s[1, 20], s[1, 21] = 0.0, -0.0          # +0.0 first
    w = np.arange(1, 2 * n + 1, dtype=np.uint16).reshape(2, n)
    snr = torch.from_numpy(s).to(DEV)
    width = torch.from_numpy(w.view(np.int16)).to(DEV)
    out, res = spd.cluster_rows(snr, width, 0.0, 4, 64)
    count, status = spd.read_result(res)
    assert status == 0 and count == 2
    got = _sorted(spd.clusters_to_numpy(out, count))
    want = oracle.cluster_rows(s, w, 0.0, 4)
    assert list(want["peak_sample"]) == [10, 20]
    _compare(got, want)
