"""DM-row shards on one GPU (no collective: the gathered partials are the
shards' partials concatenated in shard order): the merged MSD and sigma_Nmax
against spd_msd and the oracle, merge-order invariance, and the union of the
shards' candidates against the one-shot search and the oracle."""
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


def _shards(spd, x, world, scale=None):
    """Shard r's rows of x, with the same rows of the per-row scale."""
    from paper_1611_09704_gb300.sharding import shard_rows
    out = []
    for r in range(world):
        r0, r1 = shard_rows(x.shape[0], world, r)
        out.append(((r0, r1), spd.Plane(x[r0:r1], scale=None if scale is None
                                        else scale[r0:r1])))
    return out


def _gathered(spd, shards):
    return torch.cat([spd.binding.msd_shard_partial(pl) for _, pl in shards])


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_sharded_msd_and_sd_nmax(spd, dtype):
    sp = synth.ska_like(13, 40000, n_pulses=6, device=DEV, seed=61)
    kw = {}
    x = sp.data
    if dtype == "f16":
        q = synth.quantise_rows(sp, "f16")
        x, kw = q.data, {"scale": q.scale}
    whole = spd.msd_to_numpy(spd.msd(x, 0, 64, **kw))[0]
    op = oracle.Plane(synth.to_host_numpy(x), dtype=dtype,
                      scale=None if not kw else kw["scale"].cpu().numpy())
    mean_o, sd_o = oracle.plane_msd(op)
    sdn_o = oracle.plane_sd_nmax(op, 64)
    for world in (1, 2, 3, 5):
        shards = _shards(spd, x, world, **kw)
        parts = _gathered(spd, shards)
        m = spd.binding.msd_merge_partials(parts, world)
        nparts = torch.cat([spd.binding.sd_nmax_shard_partial(pl, 64, m) for _, pl in shards])
        spd.binding.sd_nmax_merge_partials(nparts, world, 64, m)
        g = spd.msd_to_numpy(m)[0]
        if world == 1:   # one shard: the same bits as spd_msd
            assert g.tobytes() == whole.tobytes()
        assert g["n"] == whole["n"] and g["status"] == 0 and g["nmax"] == 64
        assert g["mean"] == pytest.approx(whole["mean"], rel=1e-12)
        assert g["sd"] == pytest.approx(whole["sd"], rel=1e-12)
        assert g["sd_nmax"] == pytest.approx(whole["sd_nmax"], rel=1e-9)
        P.check_msd(np.atleast_1d(g), mean_o, sd_o)
        assert g["sd_nmax"] == pytest.approx(float(sdn_o[0]), rel=1e-5)


def test_merge_order_invariance(spd):
    """Eq. 2 is associative: the gathered parts merged in any order give the
    same MSD up to FP64 rounding."""
    sp = synth.ska_like(16, 30000, n_pulses=4, device=DEV, seed=62)
    shards = _shards(spd, sp.data, 7)
    parts = _gathered(spd, shards).view(7, -1)
    ref = spd.msd_to_numpy(spd.binding.msd_merge_partials(parts.reshape(-1), 7))[0]
    g = torch.Generator().manual_seed(1)
    for _ in range(5):
        perm = torch.randperm(7, generator=g).to(parts.device)
        r = spd.msd_to_numpy(spd.binding.msd_merge_partials(parts[perm].reshape(-1), 7))[0]
        assert r["mean"] == pytest.approx(ref["mean"], rel=1e-14)
        assert r["sd"] == pytest.approx(ref["sd"], rel=1e-13)


def test_empty_shard_and_bad_args(spd):
    sp = synth.plain_tophat(3, 5000, device=DEV, seed=63)
    parts = _gathered(spd, _shards(spd, sp.data, 5))     # shards 3, 4 hold no rows
    g = spd.msd_to_numpy(spd.binding.msd_merge_partials(parts, 5))[0]
    w = spd.msd_to_numpy(spd.msd(sp.data))[0]
    assert g["n"] == w["n"] and g["mean"] == pytest.approx(w["mean"], rel=1e-12)
    with pytest.raises(spd.SpdError):
        spd.binding.msd_merge_partials(parts, 0)


@pytest.mark.parametrize("world", [1, 3])
def test_sharded_search_matches_one_shot_and_oracle(spd, world):
    from paper_1611_09704_gb300.sharding import ShardedSearch
    sp = synth.ska_like(12, 60000, n_pulses=10, device=DEV, seed=64)
    x = sp.data
    widths = list(range(1, 17)) + list(range(24, 257, 8))
    thr, cap = 7.0, 1 << 20
    shards = _shards(spd, x, world)
    parts = _gathered(spd, shards)
    recs = []
    for (r0, r1), pl in shards:
        ss = ShardedSearch(pl, widths, thr, cap, dm_offset=r0, gather=lambda t: parts)
        ss.run()
        recs.append(ss.candidates())
    got = np.sort(np.concatenate(recs), order=["dm", "sample"])
    out, res, _ = spd.search(x, widths, thr, cap)
    cnt, st = spd.read_result(res)
    one = np.sort(spd.candidates_to_numpy(out, cnt), order=["dm", "sample"])
    if world == 1:
        assert np.array_equal(got, one)
    op = oracle.Plane(synth.to_host_numpy(x))
    mean, sd, sdn, tab = oracle.msd_and_sigma(op, widths)
    best, win = oracle.boxcar_snr(op, mean, sd, tab, widths)
    P.check_candidates(got, len(got), cap, best, thr, win_o=win, plane=op, mean=mean,
                       sigma_of=lambda e, w: float(np.sqrt(w) * sd[0]))
