"""PlanePipeline: planes searched from page-locked host memory with two in
flight give the same records as one-shot searches of the same planes."""
import numpy as np
import pytest
import torch

import synth

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


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipeline_equals_one_shot(spd, depth):
    from paper_1611_09704_gb300.pipeline import PlanePipeline
    widths = list(range(1, 17)) + list(range(24, 129, 8))
    planes = [synth.ska_like(24, 50000, n_pulses=8, device=DEV, seed=70 + k).data
              for k in range(4)]
    hosts = [p.cpu().pin_memory() for p in planes]
    cap = 1 << 20
    pp = PlanePipeline(24, 50000, widths, 7.0, cap, depth=depth, device=DEV, dm_offset=100)
    tickets = [pp.submit(h) for h in hosts[:depth]]
    got = []
    for k in range(len(hosts)):
        count, status, recs = pp.collect(tickets[k])
        got.append((count, status, recs.copy()))   # the view lasts until the slot's reuse
        if k + depth < len(hosts):
            tickets.append(pp.submit(hosts[k + depth]))
    for (count, status, recs), p in zip(got, planes):
        out, res, _ = spd.search(p, widths, 7.0, cap)
        c, st = spd.read_result(res)
        want = spd.candidates_to_numpy(out, c).copy()
        want["dm"] += 100
        assert (count, status) == (c, st) and c > 0
        assert np.array_equal(_sorted(recs), _sorted(want))


def test_pipeline_host_overflow_is_reported(spd):
    from paper_1611_09704_gb300.binding import SPD_ERR_OVERFLOW
    from paper_1611_09704_gb300.pipeline import PlanePipeline
    p = synth.ska_like(8, 30000, n_pulses=4, device=DEV, seed=75).data
    pp = PlanePipeline(8, 30000, list(range(1, 33)), 3.0, 1 << 20, depth=1, device=DEV,
                       host_capacity=10)
    count, status, recs = pp.collect(pp.submit(p.cpu().pin_memory()))
    assert count > 10 and status == SPD_ERR_OVERFLOW and recs.shape[0] == 10
    h = p.cpu().pin_memory()
    pp.submit(h)
    with pytest.raises(RuntimeError):   # the only slot holds an uncollected plane
        pp.submit(h)
    torch.cuda.synchronize()
