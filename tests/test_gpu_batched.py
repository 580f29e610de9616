"""The batched search (several DM ranges in one persistent launch, captured in
a CUDA graph) against the FP64 oracle range by range (the stated rule for
candidate sets, SNRs and widths), against per-range searches, and the
autotuner."""
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


def _key(recs):
    return np.sort(recs, order=["dm", "sample"])


def _specs(spd, scale=0.02):
    specs, off = [], 0
    for sp, dec, widths in synth.batched_ranges(scale, device=DEV, seed=5):
        specs.append(spd.RangeSpec(sp.data, widths, 6.0, dm_offset=off, decimation=dec))
        off += sp.n_dm
    # a range whose widths step by 8 (its own launch class) and a per-row one
    sp = synth.ska_like(5, 30000, n_pulses=4, device=DEV, seed=9)
    specs.append(spd.RangeSpec(sp.data, list(range(1, 17)) + list(range(24, 257, 8)), 7.0,
                               dm_offset=off))
    off += 5
    sp2 = synth.ska_like(3, 20000, n_pulses=2, device=DEV, seed=10)
    specs.append(spd.RangeSpec(sp2.data, list(range(1, 33)), 6.0, scope=1, dm_offset=off))
    return specs


def _oracle_check(spd, specs, recs, capacity):
    """Every range's records against the oracle's search of that range."""
    for r in specs:
        x = r.x.data if isinstance(r.x, spd.Plane) else r.x
        scale = r.x.scale if isinstance(r.x, spd.Plane) else None
        n_dm = x.shape[0]
        sel = recs[(recs["dm"] >= r.dm_offset) & (recs["dm"] < r.dm_offset + n_dm)].copy()
        sel["dm"] -= r.dm_offset
        dt = {torch.float32: "f32", torch.float16: "f16", torch.bfloat16: "bf16"}[x.dtype]
        op = oracle.Plane(synth.to_host_numpy(x), dtype=dt,
                          scale=None if scale is None else scale.cpu().numpy())
        mean, sd, sdn, tab = oracle.msd_and_sigma(op, r.widths, r.sigma_mode, r.scope, r.nmax)
        best, win = oracle.boxcar_snr(op, mean, sd, tab, r.widths, r.scope)
        nm = int(r.nmax or r.widths[-1]) if r.sigma_mode else 0

        def sigma_of(e, w, sd=sd, sdn=sdn, mode=r.sigma_mode, nm=nm):
            return float(oracle.sigma_table(mode, float(np.atleast_1d(sd)[e]), [w],
                                            float(np.atleast_1d(sdn)[e]), nm)[0])

        P.check_candidates(sel, len(sel), capacity, best, r.threshold, win_o=win, plane=op,
                           mean=mean, sigma_of=sigma_of, scope=r.scope)


def _single(spd, specs):
    recs = []
    for r in specs:
        out, res, _ = spd.search(r.x, r.widths, r.threshold, 2_000_000, r.sigma_mode, r.scope,
                                 r.nmax)
        c, st = spd.read_result(res)
        assert st == 0
        a = spd.candidates_to_numpy(out, c).copy()
        a["dm"] += r.dm_offset
        recs.append(a)
    return _key(np.concatenate(recs))


def test_batched_equals_per_range_searches(spd):
    specs = _specs(spd)
    want = _single(spd, specs)
    out, res, msd = spd.search_batched(specs, 2_000_000)
    c, st = spd.read_result(res)
    assert st == 0 and c == want.size
    got = _key(spd.candidates_to_numpy(out, c))
    _oracle_check(spd, specs, got, 2_000_000)
    assert np.array_equal(got, want)
    m = spd.msd_to_numpy(msd)
    assert m.size == sum(1 if r.scope == 0 else r.x.shape[0] for r in specs)


def test_batched_mixed_storage_types(spd):
    """FP32, FP16 (per-row scale) and BF16 ranges in one call: one launch per
    storage type, the same records as per-range searches."""
    specs, off = [], 0
    for k, dt in enumerate(("f32", "f16", "bf16")):
        sp = synth.ska_like(6, 20000 + 3000 * k, n_pulses=4, device=DEV, seed=40 + k)
        if dt == "f32":
            specs.append(spd.RangeSpec(sp.data, list(range(1, 33)), 6.0, dm_offset=off))
        else:
            q = synth.quantise_rows(sp, dt)
            specs.append(spd.RangeSpec(spd.Plane(q.data, scale=q.scale), list(range(1, 33)), 6.0,
                                       dm_offset=off))
        off += 6
    want = _single(spd, specs)
    out, res, _ = spd.search_batched(specs, 1_000_000)
    c, st = spd.read_result(res)
    assert st == 0 and c == want.size and c > 0
    # three launches shared the result word: the search's work counter in it
    # is back at 0 after each
    assert res.cpu()[12:16].view(torch.int32).item() == 0
    got = _key(spd.candidates_to_numpy(out, c))
    _oracle_check(spd, specs, got, 1_000_000)
    assert np.array_equal(got, want)


def test_batched_eq5_ranges(spd):
    """Ranges under Eq. 5 (as printed, with the default Nmax = last width, and
    the linear-excess reading with an explicit Nmax; one per-row) beside an
    Eq. 4 range in one call: the same records as per-range searches."""
    specs, off = [], 0
    for k, (mode, scope, nmax) in enumerate([(0, 0, 0), (1, 0, 0), (2, 0, 96), (1, 1, 64)]):
        sp = synth.ska_like(5, 24000 + 2000 * k, n_pulses=4, device=DEV, seed=60 + k)
        synth.inject_pulse_train(sp.data, row=1, t0=3000, n_pulses=40, width=8, period=32,
                                 amp=6.0 * 12.0, n_samp=sp.n_samp)
        widths = list(range(1, 17)) + list(range(24, 129, 8))
        specs.append(spd.RangeSpec(sp.data, widths, 5.0, sigma_mode=mode, scope=scope,
                                   nmax=nmax, dm_offset=off))
        off += 5
    want = _single(spd, specs)
    out, res, msd = spd.search_batched(specs, 1_000_000)
    c, st = spd.read_result(res)
    assert st == 0 and c == want.size and c > 0
    got = _key(spd.candidates_to_numpy(out, c))
    _oracle_check(spd, specs, got, 1_000_000)
    assert np.array_equal(got, want)
    m = spd.msd_to_numpy(msd)
    assert list(m["nmax"][1:3]) == [128, 96] and np.all(m["nmax"][3:] == 64)
    assert np.all(m["sd_nmax"][1:] > 0)


@pytest.mark.parametrize("tuning", [{"ctas_per_sm": 1, "group_scale": 2},
                                    {"ctas_per_sm": 0, "group_scale": 4},
                                    {"ctas_per_sm": 0, "group_scale": 1, "tile_threads": 128}])
def test_batched_graph_replays(spd, tuning):
    """A captured graph replayed twice, under launch shapes other than the
    default (group size, CTAs per SM, tile length): each replay meets the
    stated rule against the oracle, range by range."""
    specs = _specs(spd)
    bs = spd.BatchedSearch(specs, 2_000_000, tuning=tuning, graph=True)
    for _ in range(2):
        out, res = bs.run()
        torch.cuda.synchronize()
        c, st = spd.read_result(res)
        assert st == 0 and c > 0
        _oracle_check(spd, specs, _key(spd.candidates_to_numpy(out, c)), 2_000_000)


def test_autotune_picks_a_candidate(spd, tmp_path):
    from paper_1611_09704_gb300 import autotune
    specs = _specs(spd, scale=0.01)[:2]
    path = str(tmp_path / "tune.json")
    r1 = autotune.autotune(specs, 1_000_000, cache_path=path, reps=2)
    assert r1["tuning"] in autotune.CANDIDATES and not r1["cached"]
    r2 = autotune.autotune(specs, 1_000_000, cache_path=path, reps=2)
    assert r2["cached"] and r2["tuning"] == r1["tuning"]
