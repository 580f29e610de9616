"""Host logic of the serving loop, without a GPU: the arena allocator and the
scheduler's admission rules (slots, memory, first come first served, per-beam
order), driven by a fake device whose work finishes after a set time."""
import random

import pytest

from paper_1611_09704_gb300.serving import ALIGN, Arena, Chunk, Scheduler, summarize


def test_arena_first_fit_and_coalescing():
    a = Arena(10 * ALIGN + 17)
    assert a.capacity == 10 * ALIGN
    x = a.alloc(1)
    y = a.alloc(3 * ALIGN)
    z = a.alloc(2 * ALIGN + 1)
    assert (x, y, z) == (0, ALIGN, 4 * ALIGN)
    assert a.used == 7 * ALIGN and a.alloc(4 * ALIGN) is None
    a.free(y)
    assert a.alloc(4 * ALIGN) is None            # the hole is 3, the tail 3
    a.free(x)                                     # coalesces with y's hole
    assert a.largest_free == 4 * ALIGN
    assert a.alloc(4 * ALIGN) == 0
    a.free(z)
    a.free(0)
    assert a.used == 0 and a.largest_free == a.capacity


def test_arena_random_alloc_free_never_overlaps():
    rng = random.Random(3)
    a = Arena(1 << 20)
    live = {}
    for _ in range(3000):
        if live and rng.random() < 0.45:
            off = rng.choice(list(live))
            a.free(off)
            del live[off]
        else:
            n = rng.randint(1, 40000)
            off = a.alloc(n)
            if off is not None:
                live[off] = n
        spans = sorted((o, o + ((n + ALIGN - 1) // ALIGN) * ALIGN) for o, n in live.items())
        assert all(e0 <= s1 for (_, e0), (s1, _) in zip(spans, spans[1:]))
        assert all(o % ALIGN == 0 and e <= a.capacity for o, e in spans)
    for off in list(live):
        a.free(off)
    assert a.largest_free == a.capacity


class FakeDevice:
    """Work of a chunk takes `cost` seconds after its issue; chunks of one beam
    run one after the other (as the event wait orders them on the GPU)."""

    def __init__(self, clock, cost):
        self.clock, self.cost = clock, cost
        self.issued = []
        self.beam_free = {}
        self.running = 0
        self.peak = 0

    def start(self, c, slot, off):
        t = max(self.clock.t, self.beam_free.get(c.beam, 0.0)) + self.cost(c)
        self.beam_free[c.beam] = t
        self.issued.append((c.beam, c.index, slot, off))
        return (t, c)

    def poll(self, h):
        t, c = h
        if self.clock.t >= t:
            return (c.index, 0, None)
        return None


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def tick(self):
        self.t += 1e-3


def _chunks(n_beams, per_beam, seed=0):
    rng = random.Random(seed)
    out = []
    for b in range(n_beams):
        t = 0.0
        for k in range(per_beam):
            L = rng.randint(10, 100)
            t += L * 1e-3
            out.append(Chunk(b, k, None, L, arrival=t, deadline=L * 1e-3))
    return out


def _run(chunks, n_slots, capacity, need):
    clock = Clock()
    dev = FakeDevice(clock, cost=lambda c: c.n_samp * 2e-4)
    s = Scheduler(Arena(capacity), n_slots, need, dev.start, dev.poll, clock=clock,
                  idle=clock.tick)
    res = s.run(chunks)
    return res, dev, s


def test_scheduler_serves_every_chunk_in_beam_order():
    chunks = _chunks(5, 6)
    res, dev, s = _run(chunks, 3, 1 << 20, lambda c: 1000)
    assert len(res) == len(chunks)
    for b in range(5):
        order = [k for bb, k, _, _ in dev.issued if bb == b]
        assert order == sorted(order)
    assert 1 < s.max_inflight <= 3
    assert all(r.done >= r.arrival and r.admitted >= r.arrival for r in res)
    assert {(r.beam, r.index) for r in res} == {(c.beam, c.index) for c in chunks}


def test_scheduler_memory_bounds_concurrency():
    chunks = _chunks(4, 4, seed=1)
    need = lambda c: c.n_samp * 1000            # noqa: E731
    cap = 150 * 1000 // ALIGN * ALIGN + ALIGN   # room for at most one 100-sample chunk + a bit
    clock = Clock()
    dev = FakeDevice(clock, cost=lambda c: 5e-3)
    arena = Arena(cap)
    in_use = []
    orig_alloc = arena.alloc

    def alloc(n):
        off = orig_alloc(n)
        in_use.append(arena.used)
        return off
    arena.alloc = alloc
    s = Scheduler(arena, 8, need, dev.start, dev.poll, clock=clock, idle=clock.tick)
    res = s.run(chunks)
    assert len(res) == len(chunks)
    assert max(in_use) <= arena.capacity


def test_scheduler_fifo_no_overtaking():
    """A large chunk at the head waits for memory; smaller later chunks do not
    overtake it (per-beam order and fairness)."""
    chunks = [Chunk(0, 0, None, 90, arrival=0.0), Chunk(1, 0, None, 90, arrival=0.001),
              Chunk(0, 1, None, 10, arrival=0.002)]
    need = lambda c: c.n_samp * 1000            # noqa: E731
    res, dev, s = _run(chunks, 4, 100 * 1000, need)
    assert [(b, k) for b, k, _, _ in dev.issued] == [(0, 0), (1, 0), (0, 1)]
    assert s.max_inflight == 1


def test_scheduler_rejects_chunk_larger_than_arena():
    with pytest.raises(MemoryError):
        _run([Chunk(0, 0, None, 10)], 1, 1000, lambda c: 5000)


def test_summarize_percentiles_and_throughput():
    from paper_1611_09704_gb300.serving import ChunkResult
    rs = [ChunkResult(0, k, 100, False, count=1, arrival=k * 1.0, done=k * 1.0 + 0.01 * (k + 1),
                      deadline=0.05) for k in range(10)]
    rs.append(ChunkResult(0, 10, 0, True, arrival=9.0, done=9.5))
    s = summarize(rs, n_dm=4)
    assert s["chunks"] == 10 and s["samples"] == 4000
    assert s["p50_ms"] == pytest.approx(55.0) and s["max_ms"] == pytest.approx(100.0)
    assert s["deadline_misses"] == 5
    assert s["span_s"] == pytest.approx(9.5)
