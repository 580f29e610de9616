"""The multi-rank path on CPU: DM-row shards, the all-gather of Chan partials
over gloo groups of 2 and 3 ranks, the Eq. 2 merge in rank order (and the
second round for Eq. 5's sigma_Nmax), and the
sharded search's orchestration (with the device calls replaced by FP64 CPU
arithmetic, since this machine has no GPU)."""
import os
import socket
import types

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1611_09704_gb300 import binding as B
from paper_1611_09704_gb300.sharding import ShardedSearch, allgather_parts, shard_rows


def test_shard_rows_partition():
    for n_dm in (0, 1, 5, 64, 4097):
        for world in (1, 2, 3, 8):
            spans = [shard_rows(n_dm, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n_dm
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [r1 - r0 for r0, r1 in spans]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard_rows(10, 2, 2)


def _part_bytes(x):
    """(n, T, S, lo, hi) of a sample by definition (two-pass), as 40 bytes."""
    x = np.asarray(x, np.float64).ravel()
    n = float(x.size)
    T = float(x.sum())
    S = float(((x - T / n) ** 2).sum()) if x.size else 0.0
    lo, hi = (float(x.min()), float(x.max())) if x.size else (0.0, 0.0)
    return torch.from_numpy(np.array([n, T, S, lo, hi], np.float64).view(np.uint8).copy())


def _merge(parts_u8):
    """Eq. 2 over gathered parts in order (the oracle's merge)."""
    p = parts_u8.numpy().view(np.float64).reshape(-1, 5)
    n, T, S = 0.0, 0.0, 0.0
    for m, t, s, _, _ in p:
        if m == 0:
            continue
        if n == 0:
            n, T, S = m, t, s
            continue
        T2, S2 = oracle.chan_merge(n, T, S, m, t, s)
        n, T, S = n + m, T2, S2
    return n, T / n, np.sqrt(S / n)


def _plane(n_dm=11, n_samp=3000, seed=3):
    rng = np.random.default_rng(seed)
    x = rng.normal(5.0, 2.0, (n_dm, n_samp)).astype(np.float32)
    x[7, 1200:1216] += 4.0
    x[2, 40:41] += 9.0
    return x


def _fake_binding(real):
    """The device calls of ShardedSearch on CPU tensors, in FP64."""
    f = types.SimpleNamespace(**{k: getattr(real, k) for k in dir(real) if not k.startswith("__")})

    def msd_shard_partial(pl, out=None, workspace=None):
        out.copy_(_part_bytes(pl.data[:, :pl.n_samp].numpy()))
        return out

    def msd_merge_partials(parts, n_shards, out=None):
        assert parts.numel() == n_shards * real.PART_BYTES
        n, mu, sd = _merge(parts)
        rec = np.zeros(1, real.MSD_DTYPE)
        rec["mean"], rec["sd"], rec["n"] = mu, sd, n
        out.copy_(torch.from_numpy(rec.view(np.uint8).copy()))
        return out

    def sd_nmax_shard_partial(pl, nmax, msd, out=None, workspace=None):
        # (n, T, S) of the shard's B_Nmax series over full windows, by definition
        x = np.asarray(pl.data[:, :pl.n_samp].numpy(), np.float64)
        b = np.lib.stride_tricks.sliding_window_view(x, nmax, axis=1).sum(axis=2)
        out.copy_(_part_bytes(b))
        return out

    def sd_nmax_merge_partials(parts, n_shards, nmax, out):
        assert parts.numel() == n_shards * real.PART_BYTES
        _, _, sdn = _merge(parts)
        rec = out.numpy().view(real.MSD_DTYPE).copy()
        rec["sd_nmax"], rec["nmax"] = sdn, nmax
        out.copy_(torch.from_numpy(rec.view(np.uint8).copy()))
        return out

    def detect(pl, msd, widths, thr, cap, mode, scope, nmax, out=None, result=None,
               workspace=None):
        m = msd.numpy().view(real.MSD_DTYPE)[0]
        if mode:
            assert int(m["nmax"]) == nmax
        tab = oracle.sigma_table(mode, float(m["sd"]), widths, float(m["sd_nmax"]), nmax)
        best, win = oracle.boxcar_snr(pl.data.numpy(), [m["mean"]], [m["sd"]], [tab], widths)
        c = oracle.threshold(best, win, thr)
        recs = np.zeros(len(c), real.CAND_DTYPE)
        for k in ("dm", "sample", "width"):
            recs[k] = c[k]
        recs["snr"] = c["snr"]
        out[:len(c)] = torch.from_numpy(recs.view(np.int32).reshape(-1, 4))
        r = np.zeros(16, np.uint8)
        r[:8] = np.array([len(c)], np.uint64).view(np.uint8)
        result.copy_(torch.from_numpy(r))
        return out, result

    f.msd_shard_partial, f.msd_merge_partials, f.detect = (msd_shard_partial,
                                                           msd_merge_partials, detect)
    f.sd_nmax_shard_partial, f.sd_nmax_merge_partials = (sd_nmax_shard_partial,
                                                         sd_nmax_merge_partials)
    return f


def _rank(rank, world, port, q, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x = _plane()
        r0, r1 = shard_rows(x.shape[0], world, rank)
        # 1. the all-gather returns every rank's part, in rank order
        mine = _part_bytes(x[r0:r1])
        got = allgather_parts(mine)
        want = torch.cat([_part_bytes(x[slice(*shard_rows(x.shape[0], world, k))])
                          for k in range(world)])
        assert torch.equal(got, want)
        # 2. the sharded search's orchestration over the group
        widths = list(range(1, 33))
        ss = ShardedSearch(torch.from_numpy(np.ascontiguousarray(x[r0:r1])), widths, 5.0,
                           4096, dm_offset=r0, sigma_mode=mode)
        ss.b = _fake_binding(B)
        ss.run()
        sdn = float(ss.msd.numpy().view(B.MSD_DTYPE)[0]["sd_nmax"])
        q.put((rank, _merge(got), sdn, ss.candidates()))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,mode", [(2, 0), (2, 1), (3, 2)])
def test_gloo_ranks_match_the_whole_plane(world, mode):
    """Eq. 4, and Eq. 5 in both readings (the second exchange: sigma_Nmax
    partials of the B_Nmax series, merged in rank order)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, mode)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda t: t[0])
    x = _plane()
    mu, sd = oracle.twopass(x)
    want, _, _, (_, _, want_sdn, _) = oracle.search(x, list(range(1, 33)), 5.0, sigma_mode=mode)
    for _, (n, m, s), sdn, _ in out:
        assert n == x.size
        assert m == pytest.approx(mu, rel=1e-13) and s == pytest.approx(sd, rel=1e-12)
        if mode:
            assert sdn == pytest.approx(float(want_sdn[0]), rel=1e-10)
    # candidates of all ranks == the one-shot search of the whole plane
    got = np.concatenate([c for _, _, _, c in out])
    got.sort(order=["dm", "sample"])
    assert len(want) > 0
    assert np.array_equal(got["dm"], want["dm"]) and np.array_equal(got["sample"],
                                                                      want["sample"])
    assert np.array_equal(got["width"], want["width"])
    assert np.allclose(got["snr"], want["snr"], rtol=1e-6)
