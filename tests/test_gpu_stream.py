"""Streaming search (spd_stream_* through the C ABI) against the oracle's
replay of the same chunk schedule, and the serving loop: each beam's results
are the same served alone and in a mix of beams that overlap on the device."""
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


def _sorted(recs):
    return np.sort(recs, order=["dm", "sample"])


def _push_all(spd, bs, chunks, capacity, scale=None, in_place=False, msd=False):
    """Push every chunk then flush; returns per-call (count, status, records[, msd])."""
    max_chunk = max([c.shape[1] for c in chunks] + [0])
    ws = torch.empty(max(bs.workspace_bytes(max_chunk), 1), dtype=torch.uint8, device=DEV)
    out = torch.empty((max(capacity, 1), 4), dtype=torch.int32, device=DEV)
    res = torch.empty(16, dtype=torch.uint8, device=DEV)
    n_ent = bs.n_dm if bs.scope == 1 else 1
    mo = torch.empty(n_ent * spd.binding.MSD_BYTES, dtype=torch.uint8, device=DEV)
    calls = []
    for c in chunks:
        src = c
        if in_place:
            v = bs.chunk_view(c.shape[1], ws)
            v.copy_(c)
            src = v
        bs.push(spd.Plane(src, scale=scale), out, capacity, res, ws, msd_out=mo)
        cnt, st = spd.read_result(res)
        entry = (cnt, st, spd.candidates_to_numpy(out, cnt))
        if msd:
            entry = entry + (spd.msd_to_numpy(mo),)
        calls.append(entry)
    bs.flush(out, capacity, res, ws)
    cnt, st = spd.read_result(res)
    calls.append((cnt, st, spd.candidates_to_numpy(out, cnt)))
    return calls


def _check_against_replay(calls, rep, capacity, scope, thr):
    assert len(calls) == len(rep)
    for k, ((cnt, st, recs, *rest), r) in enumerate(zip(calls, rep)):
        assert st == 0, (k, st)
        lo, hi = r["lo"], r["hi"]
        if hi <= lo:
            assert cnt == 0, (k, cnt)
            continue
        assert np.all((recs["sample"] >= lo) & (recs["sample"] < hi)), k
        if rest:
            P.check_msd(rest[0], r["mean"], r["sd"])
        shifted = recs.copy()
        shifted["sample"] -= lo
        sd = np.atleast_1d(r["sd"])
        P.check_candidates(shifted, cnt, capacity, r["best"], thr, win_o=r["win"],
                           plane=r["sub"], mean=r["mean"], scope=scope,
                           sigma_of=lambda e, w: math.sqrt(w) * float(sd[e]))


SCHEDULES = {
    # ragged lengths, chunks shorter than wmax - 1, single samples, an empty chunk
    "ragged": [4000, 7, 1, 0, 130, 9000, 4096, 333, 12000],
    "even": [8192] * 4,
}


@pytest.mark.parametrize("sched", list(SCHEDULES))
@pytest.mark.parametrize("scope", [0, 1])
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_stream_matches_oracle_replay(spd, sched, scope, dtype):
    lengths = SCHEDULES[sched]
    n_dm, total = 12, sum(lengths)
    sp = synth.plain_tophat(n_dm, total, widths=(1, 3, 8, 17, 30, 77, 128), device=DEV,
                            seed=31 + scope)
    x = sp.data
    scale = None
    if dtype != "f32":
        sp = synth.quantise_rows(sp, dtype)
        x, scale = sp.data, sp.scale
    widths = list(range(1, 17)) + list(range(24, 129, 8))
    thr = 6.0
    bounds = np.cumsum([0] + lengths)
    chunks = [x[:, a:b].contiguous() for a, b in zip(bounds[:-1], bounds[1:])]
    bs = spd.binding.BeamStream(n_dm, x.dtype, widths, thr, scope, device=DEV)
    cap = 1 << 14
    calls = _push_all(spd, bs, chunks, cap, scale=scale, msd=True)
    host = [synth.to_host_numpy(c) for c in chunks]
    rep = oracle.stream_replay(host, widths, thr, scope, dtype=dtype,
                               scale=None if scale is None else scale.cpu().numpy(),
                               detail=True)
    _check_against_replay(calls, rep, cap, scope, thr)
    assert bs.seen == total and bs.halo == 0
    found = np.concatenate([c[2] for c in calls])
    for p in sp.pulses:   # every injected pulse is found somewhere in the stream
        assert np.any((found["dm"] == p.dm) & (np.abs(found["sample"] - p.sample) <= 2))


def test_stream_in_place_and_host_chunks_match(spd):
    """Chunks written in place through the chunk view, and chunks pushed from
    page-locked host memory, give the same bits as device chunks."""
    n_dm, lengths = 9, [3000, 50, 7000, 2048]
    sp = synth.plain_tophat(n_dm, sum(lengths), device=DEV, seed=41)
    sp = synth.quantise_rows(sp, "f16")
    b = np.cumsum([0] + lengths)
    chunks = [sp.data[:, i:j].contiguous() for i, j in zip(b[:-1], b[1:])]
    widths = list(range(1, 65))
    runs = []
    for mode in ("device", "in_place", "host"):
        bs = spd.binding.BeamStream(n_dm, torch.float16, widths, 5.0, 0, device=DEV)
        cs = [c.cpu().pin_memory() for c in chunks] if mode == "host" else chunks
        runs.append(_push_all(spd, bs, cs, 1 << 12, scale=sp.scale,
                              in_place=(mode == "in_place")))
    for other in runs[1:]:
        for (c0, s0, r0), (c1, s1, r1) in zip(runs[0], other):
            assert (c0, s0) == (c1, s1)
            assert np.array_equal(_sorted(r0), _sorted(r1))


def test_stream_single_chunk_equals_one_shot_search(spd):
    """One push plus the flush is the one-shot search of the same plane."""
    sp = synth.plain_tophat(16, 20000, device=DEV, seed=43)
    widths = list(range(1, 33))
    bs = spd.binding.BeamStream(16, torch.float32, widths, 6.0, 0, device=DEV)
    calls = _push_all(spd, bs, [sp.data], 1 << 12)
    got = _sorted(np.concatenate([c[2] for c in calls]))
    out, res, _ = spd.search(sp.data, widths, 6.0, 1 << 12)
    cnt, st = spd.read_result(res)
    want = _sorted(spd.candidates_to_numpy(out, cnt))
    assert np.array_equal(got[["dm", "sample", "width"]], want[["dm", "sample", "width"]])
    assert np.allclose(got["snr"], want["snr"], rtol=2e-6, atol=2e-6)


def test_stream_rejects_linear_sigma_and_bad_chunks(spd):
    b = spd.binding
    bs = b.BeamStream(4, torch.float32, [1, 2, 4], 6.0, 0, device=DEV)
    ws = torch.empty(bs.workspace_bytes(100), dtype=torch.uint8, device=DEV)
    out = torch.empty((16, 4), dtype=torch.int32, device=DEV)
    res = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(b.SpdError):      # wrong row count
        bs.push(torch.zeros((5, 100), device=DEV), out, 16, res, ws)
    with pytest.raises(b.SpdError):      # wrong storage type
        bs.push(torch.zeros((4, 100), dtype=torch.float16, device=DEV), out, 16, res, ws)
    with pytest.raises(b.SpdError):      # longer than the workspace allows
        bs.push(torch.zeros((4, 5000), device=DEV), out, 16, res, ws)
    prm, keep = b._params([1, 2, 4], 6.0, b.SIGMA_LINEAR, 0, 0)
    assert b.load().spd_stream_state_bytes(4, b.F32, prm) == 0


# ------------------------------------------------------------------ serving

SERVE_CAP = 1 << 16

def _serve(spd, beams, n_dm, widths, thr, n_slots, realtime=False, compress=1.0,
           mem_budget=1 << 28, which=None):
    from paper_1611_09704_gb300 import serving
    which = range(len(beams)) if which is None else which
    max_chunk = max(max(beams[b].lengths) for b in which)
    srv = serving.Server(n_dm, widths, thr, max_chunk, dtype=spd.F16, capacity=SERVE_CAP,
                         host_records=64, n_slots=n_slots, mem_budget=mem_budget, device=DEV)
    chunks = []
    for b in which:
        srv.add_beam(b)
        t = 0
        for k, (c, L) in enumerate(zip(beams[b].chunks, beams[b].lengths)):
            t += L
            arr = t * synth.SAMPLE_TIME_S / compress
            chunks.append(serving.Chunk(b, k, c, L, arrival=arr,
                                        deadline=L * synth.SAMPLE_TIME_S / compress))
        chunks.append(serving.Chunk(b, len(beams[b].lengths), None, 0, arrival=arr, flush=True))
    res = srv.serve(chunks, realtime=realtime)
    return {(r.beam, r.index): r for r in res}, srv


def test_serving_alone_equals_mix(spd):
    n_dm, widths, thr = 64, list(range(1, 129)), 7.0
    beams = synth.serving_beams(6, n_dm, 4, length_range=(700, 9000), rate_hz=10.0,
                                seed=17, pin_memory=True)
    mix, srv = _serve(spd, beams, n_dm, widths, thr, n_slots=4)
    assert srv.scheduler.max_inflight > 1           # chunks overlapped on the device
    assert len(mix) == sum(len(b.lengths) + 1 for b in beams)
    n_cand = 0
    for b in range(len(beams)):
        alone, _ = _serve(spd, beams, n_dm, widths, thr, n_slots=1, which=[b])
        for k in range(len(beams[b].lengths) + 1):
            a, m = alone[(b, k)], mix[(b, k)]
            assert (a.count, a.status) == (m.count, m.status)
            assert a.status == 0, (b, k, a.count)       # no overflow: full lists compared
            assert np.array_equal(_sorted(a.candidates), _sorted(m.candidates)), (b, k)
            n_cand += a.count
    assert n_cand > 0
    # and one beam against the oracle's replay of its chunk schedule
    b = 0
    rep = oracle.stream_replay([synth.to_host_numpy(c) for c in beams[b].chunks], widths, thr,
                               dtype="f16", detail=True)
    calls = [(mix[(b, k)].count, mix[(b, k)].status, mix[(b, k)].candidates)
             for k in range(len(rep))]
    _check_against_replay(calls, rep, SERVE_CAP, 0, thr)


def test_serving_admission_by_memory(spd):
    """With room for about one chunk's push at a time the server still serves
    every chunk, fewer at once, with the same results."""
    n_dm, widths, thr = 32, list(range(1, 65)), 7.0
    beams = synth.serving_beams(3, n_dm, 3, length_range=(2000, 6000), rate_hz=10.0,
                                seed=23, pin_memory=True)
    free, srv_free = _serve(spd, beams, n_dm, widths, thr, n_slots=3)
    assert srv_free.scheduler.max_inflight == 3
    from paper_1611_09704_gb300 import serving
    probe = serving.Server(n_dm, widths, thr, 6000, dtype=spd.F16, capacity=SERVE_CAP,
                           host_records=64, n_slots=1, mem_budget=1 << 24, device=DEV)
    one = max(probe.need(serving.Chunk(0, 0, None, L)) for b in beams for L in b.lengths)
    budget = 3 * probe._state_bytes + 3 * 256 + one + 256
    tight, srv = _serve(spd, beams, n_dm, widths, thr, n_slots=3, mem_budget=budget)
    # two data chunks never fit together (only a flush may join one)
    assert 1 <= srv.scheduler.max_inflight <= 2
    assert srv.arena.peak <= srv.arena.capacity
    for key, r in free.items():
        assert (r.count, r.status) == (tight[key].count, tight[key].status)
        assert np.array_equal(_sorted(r.candidates), _sorted(tight[key].candidates))


def test_serving_realtime_latency(spd):
    """Time-compressed arrivals: every chunk gets a latency and the summary
    reports percentiles and throughput."""
    from paper_1611_09704_gb300 import serving
    n_dm, widths = 64, list(range(1, 129))
    beams = synth.serving_beams(4, n_dm, 3, length_range=(2000, 8000), rate_hz=50.0,
                                seed=29, pin_memory=True)
    res, srv = _serve(spd, beams, n_dm, widths, 7.0, n_slots=4, realtime=True, compress=20.0)
    s = serving.summarize(list(res.values()), n_dm)
    assert s["chunks"] == 12 and s["p99_ms"] >= s["p50_ms"] > 0
    assert all(r.done >= r.arrival for r in res.values())
