"""Back-to-back searches of DM x time planes held in page-locked host memory.

A plane's search has three parts that use different engines: the host ->
device copy of the plane, the search on the SMs (shard partial, Eq. 2 merge,
fused detect), and the device -> host copy of the candidate records.
:class:`PlanePipeline` keeps ``depth`` planes in flight in slots of their own
(device plane, output buffer, page-locked record buffer), so that the copy in
of plane k+1 and the copy out of plane k's records overlap the search of the
planes around them.  Every plane still makes the whole trip: its copy in, its
search, its count and every record back in host memory.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import binding as b
from .sharding import ShardedSearch


@dataclass
class _Slot:
    x: torch.Tensor            # device plane
    search: ShardedSearch
    rec_host: torch.Tensor     # page-locked records
    res_host: torch.Tensor     # page-locked result word
    ev_free: torch.cuda.Event  # the search no longer reads x
    ev_found: torch.cuda.Event # result word copied to the host
    ev_out: torch.cuda.Event   # records copied to the host
    busy: bool = False


class PlanePipeline:
    """Searches [n_dm, n_samp] planes submitted from page-locked host memory.

    submit(x_host) queues one plane and returns a ticket; collect(ticket)
    waits for that plane's candidates and returns (count, status, records),
    records being a view of the slot's page-locked buffer (valid until the
    slot is reused, ``depth`` submissions later).  Tickets are collected in
    submission order."""

    def __init__(self, n_dm, n_samp, widths, threshold, capacity, *, dtype=torch.float32,
                 depth=2, device="cuda", gather=None, dm_offset=0, host_capacity=None):
        self.dev = torch.device(device)
        self.capacity = int(capacity)
        self.host_capacity = int(self.capacity if host_capacity is None else host_capacity)
        self.copy_in = torch.cuda.Stream(self.dev)
        self.compute = torch.cuda.Stream(self.dev)
        self.copy_out = torch.cuda.Stream(self.dev)
        self.slots = []
        for _ in range(int(depth)):
            x = torch.empty((n_dm, n_samp), dtype=dtype, device=self.dev)
            ss = ShardedSearch(x, widths, threshold, capacity, gather=gather, dm_offset=dm_offset)
            self.slots.append(_Slot(
                x, ss,
                torch.empty((max(self.host_capacity, 1), 4), dtype=torch.int32, pin_memory=True),
                torch.empty(b.RESULT_BYTES, dtype=torch.uint8, pin_memory=True),
                torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()))
        self.next = 0
        self.h2d_bytes = n_dm * n_samp * torch.empty((), dtype=dtype).element_size()

    def submit(self, x_host: torch.Tensor) -> int:
        k = self.next
        s = self.slots[k % len(self.slots)]
        if s.busy:
            raise RuntimeError("slot still holds an uncollected plane; collect it first")
        s.busy = True
        self.next += 1
        with torch.cuda.stream(self.copy_in):
            self.copy_in.wait_event(s.ev_free)      # the previous search of this slot is done
            s.x.copy_(x_host, non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(self.copy_in)
        with torch.cuda.stream(self.compute):
            self.compute.wait_event(ev_in)
            s.search.run()
            s.ev_free.record(self.compute)
            s.res_host.copy_(s.search.result, non_blocking=True)
            s.ev_found.record(self.compute)
        return k

    def collect(self, ticket: int):
        """(count, status, records): the exact count; status SPD_ERR_OVERFLOW
        when more records exist than the device or host buffer holds (those
        that fit are returned); records carry DM rows of the whole plane."""
        s = self.slots[ticket % len(self.slots)]
        s.ev_found.synchronize()
        r = s.res_host.numpy()
        count = int(r[:8].view(np.uint64)[0])
        status = int(r[8:12].view(np.int32)[0])
        n = min(count, self.capacity, self.host_capacity)
        if status == b.SPD_OK and n < count:
            status = b.SPD_ERR_OVERFLOW
        with torch.cuda.stream(self.copy_out):
            self.copy_out.wait_event(s.ev_found)
            if n:
                s.rec_host[:n].copy_(s.search.out[:n], non_blocking=True)
            s.ev_out.record(self.copy_out)
        s.ev_out.synchronize()
        s.busy = False
        recs = s.rec_host[:n].numpy().view(b.CAND_DTYPE).reshape(-1)
        if n and s.search.dm_offset:
            recs["dm"] += s.search.dm_offset
        return count, status, recs
