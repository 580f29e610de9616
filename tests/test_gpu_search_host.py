"""spd_search_host: the whole search of a plane held in host memory through
the C ABI (copies in, MSD, search in row blocks with each block's records
copied out while the next runs).  Its records must meet the stated rule
against the FP64 oracle and equal spd_search's on the same plane; with too
small a capacity the count stays exact."""
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


def _sorted(r):
    return np.sort(r, order=["dm", "sample"])


@pytest.mark.parametrize("dtype,n_dm,n_samp,scope", [
    ("f32", 600, 20001, 0),     # two row blocks of 300, ragged length
    ("f16", 300, 12000, 1),     # one block, per-row MSD, host per-row scale
    ("bf16", 520, 9000, 1),     # two blocks, per-row MSD: each block's tables offset by its rows
])
def test_search_host_matches_oracle_and_device(spd, dtype, n_dm, n_samp, scope):
    sp = synth.ska_like(n_dm, n_samp, n_pulses=8, device=DEV, seed=71)
    x, scale = sp.data, None
    if dtype != "f32":
        q = synth.quantise_rows(sp, dtype)
        x, scale = q.data, q.scale
    widths = list(range(1, 17)) + list(range(24, 129, 8))
    thr = 7.0
    xh = x.cpu().pin_memory()
    sh = None if scale is None else scale.cpu().pin_memory()
    cap = n_dm * n_samp // 2
    # a workspace holding stale bytes: the call must reset its own count word
    ws = torch.full((spd.search_host_workspace_bytes(xh, widths, thr, cap, 0, scope, scale=sh),),
                    0xA5, dtype=torch.uint8, device=DEV)
    out = torch.empty((cap, 4), dtype=torch.int32).pin_memory()
    count, status = spd.search_host(xh, widths, thr, out, 0, scope, workspace=ws, scale=sh)
    assert status == 0 and 0 < count <= cap
    got = _sorted(out[:count].numpy().view(spd.CAND_DTYPE).reshape(-1))

    # the device path on the same plane: the same records
    o2, r2, _ = spd.search(x, widths, thr, cap, 0, scope, scale=scale)
    c2, s2 = spd.read_result(r2)
    assert (c2, s2) == (count, 0)
    assert np.array_equal(got, _sorted(spd.candidates_to_numpy(o2, c2)))

    op = oracle.Plane(synth.to_host_numpy(x), dtype=dtype,
                      scale=None if scale is None else scale.cpu().numpy())
    _, best, win, (mean, sd, _, _) = oracle.search(op, widths, thr, scope=scope)
    P.check_candidates(got, count, cap, best, thr, win_o=win, plane=op, mean=mean, scope=scope,
                       sigma_of=lambda e, w: math.sqrt(w) * float(np.atleast_1d(sd)[e]))


def test_search_host_overflow_keeps_the_count(spd):
    sp = synth.ska_like(300, 9000, n_pulses=4, device=DEV, seed=72)   # drift: many candidates
    xh = sp.data.cpu().pin_memory()
    widths = list(range(1, 33))
    ws = torch.full((spd.search_host_workspace_bytes(xh, widths, 7.0, 1000),), 0x5A,
                    dtype=torch.uint8, device=DEV)
    out = torch.zeros((1000, 4), dtype=torch.int32)
    count, status = spd.search_host(xh, widths, 7.0, out, workspace=ws)
    o2, r2, _ = spd.search(sp.data, widths, 7.0, 1 << 22)
    assert status == 0 and count == spd.read_result(r2)[0] > 1000
    recs = out.numpy().view(spd.CAND_DTYPE).reshape(-1)
    full = spd.candidates_to_numpy(o2, count)
    keys = set(zip(full["dm"].tolist(), full["sample"].tolist()))
    assert all((int(d), int(s)) in keys for d, s in zip(recs["dm"], recs["sample"]))


def test_search_host_from_two_threads(spd):
    """Two host threads, each with its own stream, workspace and output,
    search two planes at once (the copy stream of each call belongs to its
    thread): every call gives the records of its plane alone."""
    import threading
    planes = [synth.ska_like(300, 20000, n_pulses=6, device=DEV, seed=80 + k).data.cpu().pin_memory()
              for k in range(2)]
    widths = list(range(1, 17)) + list(range(24, 129, 8))
    cap = 300 * 20000 // 2

    def run(xh, stream):
        ws = torch.empty(spd.search_host_workspace_bytes(xh, widths, 7.0, cap), dtype=torch.uint8,
                         device=DEV)
        out = torch.empty((cap, 4), dtype=torch.int32).pin_memory()
        got = []
        for _ in range(3):
            c, st = spd.search_host(xh, widths, 7.0, out, workspace=ws, stream=stream)
            got.append((c, st, _sorted(out[:c].numpy().view(spd.CAND_DTYPE).reshape(-1)).copy()))
        return got

    want = [run(xh, None)[0] for xh in planes]
    results = [None, None]

    def worker(k):
        torch.cuda.set_device(0)
        results[k] = run(planes[k], torch.cuda.Stream(device=DEV))

    th = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for k in range(2):
        assert results[k] is not None
        for c, st, recs in results[k]:
            assert (c, st) == want[k][:2] and np.array_equal(recs, want[k][2])
