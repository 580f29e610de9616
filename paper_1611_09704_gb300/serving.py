"""Streaming search of several beams with continuous batching.

Every beam is a :class:`~.binding.BeamStream`: its running MSD (Eq. 2 adds
each chunk to it) and its halo of wmax - 1 samples stay on the device between
chunks.  Chunks arrive from the beams over time in page-locked host memory.
The :class:`Scheduler` admits the oldest waiting chunk as soon as a stream
slot is free and the device memory its push needs fits in the arena, so a
chunk that arrives while others are on the GPU starts at once and its copies
and kernels overlap theirs on the device.  Chunks of one beam run in arrival
order: each waits on the device for the event of the beam's previous chunk.

The :class:`Server` issues one chunk on its slot's CUDA stream as:
wait for the beam's previous chunk, spd_stream_push (host -> device copy of
the chunk into the push workspace, MSD update, fused search), copy of the
result word and of the first records to page-locked host memory, event.  The
host polls the events; a chunk's latency runs from its arrival to the moment
its candidates are in host memory.  The scheduler is plain host logic with
the device behind two callbacks, so its admission rules run without a GPU.
"""
from __future__ import annotations

import bisect
import collections
import time
from dataclasses import dataclass, field

import numpy as np

ALIGN = 256
SPD_ERR_OVERFLOW = 4     # spd_status of include/spd.h


def _up(n: int) -> int:
    return (int(n) + ALIGN - 1) // ALIGN * ALIGN


class Arena:
    """First-fit allocator of byte ranges in [0, capacity), 256-byte aligned,
    coalescing neighbours on free (bookkeeping only; the bytes are a device
    tensor owned by the caller)."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity) // ALIGN * ALIGN
        self._free = [(0, self.capacity)] if self.capacity > 0 else []   # sorted by offset
        self._live: dict[int, int] = {}
        self.peak = 0

    @property
    def used(self) -> int:
        return sum(self._live.values())

    @property
    def largest_free(self) -> int:
        return max((s for _, s in self._free), default=0)

    def alloc(self, nbytes: int):
        n = _up(max(int(nbytes), 1))
        for i, (o, s) in enumerate(self._free):
            if s >= n:
                if s == n:
                    del self._free[i]
                else:
                    self._free[i] = (o + n, s - n)
                self._live[o] = n
                self.peak = max(self.peak, self.used)
                return o
        return None

    def free(self, off: int):
        n = self._live.pop(off)
        i = bisect.bisect_left(self._free, (off, 0))
        self._free.insert(i, (off, n))
        if i + 1 < len(self._free) and off + n == self._free[i + 1][0]:
            self._free[i] = (off, n + self._free[i + 1][1])
            del self._free[i + 1]
        if i > 0 and self._free[i - 1][0] + self._free[i - 1][1] == off:
            o, s = self._free[i - 1]
            self._free[i - 1] = (o, s + self._free[i][1])
            del self._free[i]


@dataclass
class Chunk:
    """One chunk of a beam: ``data`` [n_dm, n_samp] in host memory (None for
    the end-of-stream flush), ``arrival`` and ``deadline`` in seconds on the
    serving clock (deadline relative to arrival)."""
    beam: int
    index: int
    data: object
    n_samp: int
    arrival: float = 0.0
    deadline: float = float("inf")
    flush: bool = False


@dataclass
class ChunkResult:
    beam: int
    index: int
    n_samp: int
    flush: bool
    count: int = 0
    status: int = 0
    candidates: np.ndarray | None = None
    arrival: float = 0.0
    admitted: float = 0.0
    done: float = 0.0
    deadline: float = float("inf")

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Flight:
    chunk: Chunk
    slot: int
    block: int
    handle: object
    result: ChunkResult


class Scheduler:
    """Continuous batching of beam chunks over ``n_slots`` stream slots and an
    :class:`Arena` of device memory.

    need(chunk) -> bytes its push needs; start(chunk, slot, block_offset) ->
    handle once its work is issued; poll(handle) -> None while it runs, else
    (count, status, candidates).  Admission is first come, first served: the
    oldest waiting chunk goes first, and nothing overtakes it while it waits
    for a slot or for memory, so chunks of one beam are issued in order."""

    def __init__(self, arena: Arena, n_slots: int, need, start, poll, clock=time.perf_counter,
                 idle=None):
        if n_slots < 1:
            raise ValueError("n_slots must be >= 1")
        self.arena = arena
        self.n_slots = int(n_slots)
        self.need, self.start, self.poll = need, start, poll
        self.clock = clock
        self.idle = idle or (lambda: None)
        self.max_inflight = 0

    def run(self, chunks, realtime: bool = True):
        """Serve every chunk; returns ChunkResults in completion order.  With
        realtime=False every chunk is taken to arrive at the start."""
        order = sorted(chunks, key=lambda c: c.arrival)   # stable: beam order kept
        for c in order:
            if _up(self.need(c)) > self.arena.capacity:
                raise MemoryError(f"chunk {c.beam}/{c.index} needs {self.need(c)} bytes, "
                                  f"arena holds {self.arena.capacity}")
        future = collections.deque(order)
        waiting: collections.deque = collections.deque()
        flights: list[_Flight] = []
        free_slots = list(range(self.n_slots))[::-1]
        done: list[ChunkResult] = []
        t0 = self.clock()
        while future or waiting or flights:
            now = self.clock() - t0
            while future and (not realtime or future[0].arrival <= now):
                waiting.append(future.popleft())
            progressed = False
            for f in list(flights):
                r = self.poll(f.handle)
                if r is None:
                    continue
                f.result.count, f.result.status, f.result.candidates = r
                f.result.done = self.clock() - t0
                self.arena.free(f.block)
                free_slots.append(f.slot)
                flights.remove(f)
                done.append(f.result)
                progressed = True
            while waiting and free_slots:
                c = waiting[0]
                off = self.arena.alloc(self.need(c))
                if off is None:
                    break
                waiting.popleft()
                slot = free_slots.pop()
                res = ChunkResult(c.beam, c.index, c.n_samp, c.flush,
                                  arrival=c.arrival if realtime else 0.0,
                                  admitted=self.clock() - t0, deadline=c.deadline)
                flights.append(_Flight(c, slot, off, self.start(c, slot, off), res))
                self.max_inflight = max(self.max_inflight, len(flights))
                progressed = True
            if not progressed:
                self.idle()
        return done


def summarize(results, n_dm: int) -> dict:
    """p50 / p99 latency, deadline misses and throughput of a serving run."""
    data = [r for r in results if not r.flush]
    lat = np.array([r.latency for r in data]) if data else np.zeros(1)
    t_first = min((r.arrival for r in results), default=0.0)
    t_last = max((r.done for r in results), default=0.0)
    samples = sum(r.n_samp for r in data) * n_dm
    span = max(t_last - t_first, 1e-12)
    return {
        "chunks": len(data),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "max_ms": float(lat.max() * 1e3),
        "deadline_misses": int(sum(1 for r in data if r.latency > r.deadline)),
        "samples": int(samples),
        "span_s": float(span),
        "samples_per_s": float(samples / span),
        "candidates": int(sum(r.count for r in results)),
        "overflows": int(sum(1 for r in results if r.status != 0)),
    }


@dataclass
class _Beam:
    stream: object
    last_event: object = None
    scale: object = None
    offset: object = None


@dataclass
class Server:
    """Serves chunks of many beams through spd_stream_push on one GPU.

    n_dm, widths, threshold, dtype, scope: the search of every beam.
    max_chunk: longest chunk (samples per row).  capacity: candidate records
    a chunk may produce (more sets the overflow status).  host_records:
    records copied back with the result word (more take a second copy).
    mem_budget: bytes of device memory the server may hold (default: free
    memory minus ``reserve``); beam states and each chunk's push come out of
    it, and a chunk waits until its push fits."""
    n_dm: int
    widths: list
    threshold: float
    max_chunk: int
    dtype: int = 1
    scope: int = 0
    capacity: int = 1 << 16
    host_records: int = 4096
    n_slots: int = 4
    mem_budget: int | None = None
    reserve: int = 1 << 30
    device: str = "cuda"
    beams: dict = field(default_factory=dict)

    def __post_init__(self):
        import torch

        from .binding import BeamStream
        self._torch = torch
        self._BeamStream = BeamStream
        dev = torch.device(self.device)
        free, _ = torch.cuda.mem_get_info(dev)
        # memory torch has cached but not handed out is free for the arena too
        free += torch.cuda.memory_reserved(dev) - torch.cuda.memory_allocated(dev)
        budget = free - self.reserve
        if self.mem_budget is not None:
            budget = min(budget, int(self.mem_budget))
        if budget <= 0:
            raise MemoryError("no device memory for the serving arena")
        self.arena = Arena(budget)
        self.pool = torch.empty(self.arena.capacity, dtype=torch.uint8, device=self.device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.n_slots)]
        self.host_out = [torch.empty((self.host_records, 4), dtype=torch.int32, pin_memory=True)
                         for _ in range(self.n_slots)]
        self.host_res = [torch.empty(16, dtype=torch.uint8, pin_memory=True)
                         for _ in range(self.n_slots)]
        probe = BeamStream(self.n_dm, self.dtype, self.widths, self.threshold, self.scope,
                           device=self.device)
        self._state_bytes = probe.state_bytes()
        self._ws = {}
        self._probe = probe
        torch.cuda.synchronize(self.device)

    # ------------------------------------------------------------ memory
    def ws_bytes(self, n_samp: int) -> int:
        if n_samp not in self._ws:
            self._ws[n_samp] = self._probe.workspace_bytes(n_samp)
        return self._ws[n_samp]

    def need(self, c: Chunk) -> int:
        return _up(self.ws_bytes(c.n_samp)) + _up(self.capacity * 16) + ALIGN

    def add_beam(self, beam: int, scale=None, offset=None):
        """Allocate and reset a beam's state (from the arena)."""
        if beam in self.beams:
            raise ValueError(f"beam {beam} exists")
        off = self.arena.alloc(self._state_bytes)
        if off is None:
            raise MemoryError("no arena memory for a beam state")
        st = self.pool[off:off + self._state_bytes]
        bs = self._BeamStream(self.n_dm, self.dtype, self.widths, self.threshold, self.scope,
                              device=self.device, state=st)
        ev = self._torch.cuda.Event()
        ev.record()            # the reset ran on the current stream: slots wait for it
        self.beams[beam] = _Beam(bs, ev, scale, offset)
        return bs

    def remove_beam(self, beam: int):
        b = self.beams.pop(beam)
        if b.last_event is not None:
            b.last_event.synchronize()
        self.arena.free(b.stream.state.data_ptr() - self.pool.data_ptr())

    # ------------------------------------------------------------ device work
    def _start(self, c: Chunk, slot: int, off: int):
        torch = self._torch
        from .binding import Plane
        b = self.beams[c.beam]
        s = self.streams[slot]
        wsb = self.ws_bytes(c.n_samp)
        ws = self.pool[off:off + wsb]
        o2 = off + _up(wsb)
        out = self.pool[o2:o2 + self.capacity * 16].view(torch.int32).view(-1, 4)
        o3 = o2 + _up(self.capacity * 16)
        res = self.pool[o3:o3 + 16]
        with torch.cuda.stream(s):
            if b.last_event is not None:
                s.wait_event(b.last_event)
            if c.flush:
                b.stream.flush(out, self.capacity, res, ws, stream=s)
            else:
                b.stream.push(Plane(c.data, scale=b.scale, offset=b.offset), out,
                              self.capacity, res, ws, stream=s)
            self.host_res[slot].copy_(res, non_blocking=True)
            k = min(self.host_records, self.capacity)
            self.host_out[slot][:k].copy_(out[:k], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        b.last_event = ev
        return (ev, slot, out, c)

    def _poll(self, h):
        ev, slot, out, c = h
        if not ev.query():
            return None
        from .binding import CAND_DTYPE
        r = self.host_res[slot].numpy()
        count = int(r[:8].view(np.uint64)[0])
        status = int(r[8:12].view(np.int32)[0])
        if status == 0 and count > self.capacity:
            status = SPD_ERR_OVERFLOW          # records beyond capacity were dropped
        n = min(count, self.capacity)
        k = min(n, self.host_records)
        recs = self.host_out[slot][:k].numpy().copy()
        if n > k:
            recs = np.concatenate([recs, out[k:n].cpu().numpy()])
        return count, status, recs.view(CAND_DTYPE).reshape(-1)

    def serve(self, chunks, realtime: bool = True):
        """Serve the chunks (see :class:`Scheduler`); returns ChunkResults."""
        for c in chunks:
            if c.beam not in self.beams:
                raise KeyError(f"beam {c.beam} not added")
            if not c.flush and c.n_samp > self.max_chunk:
                raise ValueError(f"chunk {c.beam}/{c.index}: {c.n_samp} > max_chunk")
        self.scheduler = Scheduler(self.arena, self.n_slots, self.need, self._start, self._poll)
        return self.scheduler.run(chunks, realtime=realtime)
