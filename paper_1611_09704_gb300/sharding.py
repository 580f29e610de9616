"""DM-row sharding of the search over ranks, one GPU per rank.

Rows are independent for the boxcars, the SNR and the threshold (Sec. 2.3,
2.4); the one quantity shared by all rows is the MSD of the whole plane
(Sec. 2.1).  Each rank reduces its rows to one Chan partial (n, T, S) with
spd_msd_shard_partial, the ranks all-gather the 40-byte partials, and every
rank merges them with Eq. 2 in rank order (spd_msd_merge_partials), so every
rank holds the same MSD bits.  With Eq. 5 a second round does the same for
the B_Nmax series, centred on the merged mean.  Candidates stay on their
rank, with the shard's first DM row added when they are decoded.
"""
from __future__ import annotations

import numpy as np


def shard_rows(n_dm: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) of `rank`: contiguous, sizes differing by at most one,
    the larger shards first."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world / rank")
    base, extra = divmod(int(n_dm), int(world))
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def allgather_parts(part, group=None):
    """All-gather one partial (a 40-byte uint8 tensor) from every rank;
    returns the parts concatenated in rank order.  Without an initialised
    process group (one rank) the part itself."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return part
    world = dist.get_world_size(group)
    if world == 1:
        return part
    bufs = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(bufs, part, group=group)
    return torch.cat(bufs)


class ShardedSearch:
    """The search of one rank's shard with the MSD of the whole plane.

    x: this rank's rows (device tensor or binding.Plane); dm_offset: its first
    DM row in the whole plane; gather: the all-gather of a partial (default
    :func:`allgather_parts` over `group`).  run() issues partial, exchange,
    merge and the fused detect on the current stream.

    msd_slots > 1 keeps that many MSD states (partials, merged MSD, MSD
    workspace) apart from the detect workspace, so that the MSD of the next
    plane (msd_step(slot=1)) may run on another stream while detect_step(0)
    searches with slot 0's MSD."""

    def __init__(self, x, widths, threshold, capacity, *, dm_offset=0, sigma_mode=0,
                 nmax_sigma=0, group=None, gather=None, msd_slots=1):
        import torch

        from . import binding as b
        self.b = b
        self.pl = b.as_plane(x)
        self.widths = list(widths)
        self.threshold = float(threshold)
        self.capacity = int(capacity)
        self.dm_offset = int(dm_offset)
        self.sigma_mode = int(sigma_mode)
        self.nmax = int(nmax_sigma or (self.widths[-1] if sigma_mode else 0))
        self.gather = gather or (lambda t: allgather_parts(t, group))
        dev = self.pl.data.device
        lib = b.load()
        cp = self.pl.c()
        prm, keep = b._params(self.widths, self.threshold, self.sigma_mode, b.MSD_GLOBAL,
                              self.nmax)
        msd_ws = lib.spd_msd_workspace_bytes(cp, b.MSD_GLOBAL, self.nmax)
        det_ws = lib.spd_detect_workspace_bytes(cp, prm)
        self.ws_det = b._workspace(det_ws, dev)
        self.slots = []
        for _ in range(max(1, int(msd_slots))):
            self.slots.append({
                "part": torch.empty(b.PART_BYTES, dtype=torch.uint8, device=dev),
                "npart": torch.empty(b.PART_BYTES, dtype=torch.uint8, device=dev),
                "msd": torch.empty(b.MSD_BYTES, dtype=torch.uint8, device=dev),
                "ws": b._workspace(msd_ws, dev)})
        self.msd = self.slots[0]["msd"]
        self.out = torch.empty((max(self.capacity, 1), 4), dtype=torch.int32, device=dev)
        self.result = torch.zeros(b.RESULT_BYTES, dtype=torch.uint8, device=dev)

    def msd_step(self, slot=0):
        b, st = self.b, self.slots[slot]
        b.msd_shard_partial(self.pl, out=st["part"], workspace=st["ws"])
        parts = self.gather(st["part"])
        b.msd_merge_partials(parts, parts.numel() // b.PART_BYTES, out=st["msd"])
        if self.sigma_mode:
            b.sd_nmax_shard_partial(self.pl, self.nmax, st["msd"], out=st["npart"],
                                    workspace=st["ws"])
            nparts = self.gather(st["npart"])
            b.sd_nmax_merge_partials(nparts, nparts.numel() // b.PART_BYTES, self.nmax,
                                     st["msd"])
        return st["msd"]

    def detect_step(self, slot=0):
        return self.b.detect(self.pl, self.slots[slot]["msd"], self.widths, self.threshold,
                             self.capacity, self.sigma_mode, self.b.MSD_GLOBAL, self.nmax,
                             out=self.out, result=self.result, workspace=self.ws_det)

    def run(self):
        self.msd_step()
        return self.detect_step()

    def candidates(self) -> np.ndarray:
        """This rank's records (synchronises), DM rows of the whole plane."""
        count, status = self.b.read_result(self.result)
        if status != 0:
            raise self.b.SpdError(status, "sharded search")
        recs = self.b.candidates_to_numpy(self.out, count).copy()
        recs["dm"] += self.dm_offset
        return recs
