"""ctypes binding of libspd (include/spd.h): argument marshalling only.

Every function here has the name of the C call it wraps (without the ``spd_``
prefix), takes torch tensors that already live on the GPU, allocates the
workspace the call asks for with torch, and raises :class:`SpdError` on a
non-zero status.  All arithmetic of the search runs in the CUDA kernels of
``_build/libspd.so``; if that library is missing this module raises instead of
computing anything itself.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import builder as _build

# ----------------------------------------------------------------- ABI types

SPD_OK, SPD_ERR_INVALID_ARG, SPD_ERR_CUDA, SPD_ERR_NO_MEMORY = 0, 1, 2, 3
SPD_ERR_OVERFLOW, SPD_ERR_DEGENERATE_SIGMA, SPD_ERR_TIMEOUT, SPD_ERR_UNSUPPORTED = 4, 5, 6, 7
F32, F16, BF16 = 0, 1, 2
SIGMA_SQRTN, SIGMA_LINEAR, SIGMA_LINEAR_EXCESS = 0, 1, 2
MSD_GLOBAL, MSD_PER_ROW = 0, 1


class SpdPlane(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("n_dm", ctypes.c_int64),
                ("n_samp", ctypes.c_int64), ("row_stride", ctypes.c_int64),
                ("row_scale", ctypes.c_void_p), ("row_offset", ctypes.c_void_p)]


class SpdMsdStats(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("sd", ctypes.c_double),
                ("sd_nmax", ctypes.c_double), ("n", ctypes.c_int64),
                ("nmax", ctypes.c_int32), ("status", ctypes.c_int32)]


class SpdCandidate(ctypes.Structure):
    _fields_ = [("dm", ctypes.c_int32), ("sample", ctypes.c_int32),
                ("snr", ctypes.c_float), ("width", ctypes.c_int32)]


class SpdResult(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


class SpdSearchParams(ctypes.Structure):
    _fields_ = [("widths", ctypes.POINTER(ctypes.c_int32)), ("n_widths", ctypes.c_int32),
                ("threshold", ctypes.c_float), ("sigma_mode", ctypes.c_int32),
                ("msd_scope", ctypes.c_int32), ("nmax_sigma", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


class SpdRange(ctypes.Structure):
    _fields_ = [("plane", SpdPlane), ("params", SpdSearchParams), ("dm_offset", ctypes.c_int32),
                ("decimation", ctypes.c_int32)]


class SpdTuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("group_scale", ctypes.c_int32),
                ("tile_threads", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


class SpdStreamInfo(ctypes.Structure):
    _fields_ = [("n_dm", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("msd_scope", ctypes.c_int32), ("seen", ctypes.c_int64),
                ("halo", ctypes.c_int64), ("chunks", ctypes.c_int64), ("wmax", ctypes.c_int32),
                ("halo_cap", ctypes.c_int32), ("has_scale", ctypes.c_int32),
                ("has_offset", ctypes.c_int32)]


class SpdLevel(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("n_widths", ctypes.c_int32),
                ("widths", ctypes.POINTER(ctypes.c_int32))]


class SpdMsdPart(ctypes.Structure):
    _fields_ = [("n", ctypes.c_double), ("T", ctypes.c_double), ("S", ctypes.c_double),
                ("lo", ctypes.c_double), ("hi", ctypes.c_double)]


MSD_BYTES = ctypes.sizeof(SpdMsdStats)      # 40
PART_BYTES = ctypes.sizeof(SpdMsdPart)      # 40
CAND_BYTES = ctypes.sizeof(SpdCandidate)    # 16
RESULT_BYTES = ctypes.sizeof(SpdResult)     # 16

MSD_DTYPE = np.dtype([("mean", "<f8"), ("sd", "<f8"), ("sd_nmax", "<f8"), ("n", "<i8"),
                      ("nmax", "<i4"), ("status", "<i4")])
CAND_DTYPE = np.dtype([("dm", "<i4"), ("sample", "<i4"), ("snr", "<f4"), ("width", "<i4")])
CLUSTER_DTYPE = np.dtype([("dm", "<i4"), ("first", "<i4"), ("last", "<i4"),
                          ("peak_sample", "<i4"), ("peak_snr", "<f4"), ("peak_width", "<i4"),
                          ("members", "<i4"), ("reserved0", "<i4")])

# Every symbol include/spd.h declares, for the export check.
EXPORTS = ["spd_version", "spd_status_string", "spd_last_cuda_error",
           "spd_msd_workspace_bytes", "spd_msd", "spd_boxcar_snr_workspace_bytes",
           "spd_boxcar_snr", "spd_threshold_candidates", "spd_detect_workspace_bytes",
           "spd_search_workspace_bytes", "spd_detect", "spd_search", "spd_boxcar_sums",
           "spd_msd_noalloc", "spd_search_batched_workspace_bytes", "spd_search_batched",
           "spd_stream_state_bytes", "spd_stream_workspace_bytes", "spd_stream_reset",
           "spd_stream_push", "spd_stream_chunk_view", "spd_stream_flush",
           "spd_msd_shard_partial", "spd_msd_merge_partials", "spd_sd_nmax_shard_partial",
           "spd_sd_nmax_merge_partials", "spd_threshold_plane",
           "spd_search_decimated_workspace_bytes", "spd_search_decimated",
           "spd_debug_set_copy_wait", "spd_cluster_rows", "spd_dedisperse",
           "spd_search_host_workspace_bytes", "spd_search_host"]


class SpdError(RuntimeError):
    def __init__(self, status: int, what: str):
        lib = _lib
        msg = lib.spd_status_string(status).decode() if lib else str(status)
        extra = ""
        if lib is not None and status == SPD_ERR_CUDA:
            extra = f" (cudaError {lib.spd_last_cuda_error()})"
        super().__init__(f"{what}: {msg}{extra}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libspd.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libspd is not built ({path} missing); run "
                           "paper_1611_09704_gb300.build() first")
    lib = ctypes.CDLL(path)
    P, I32, I64, SZ, F = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t,
                          ctypes.c_float)
    pp = ctypes.POINTER(SpdPlane)
    pq = ctypes.POINTER(SpdSearchParams)
    lib.spd_version.restype = I32
    lib.spd_status_string.argtypes = [I32]
    lib.spd_status_string.restype = ctypes.c_char_p
    lib.spd_last_cuda_error.restype = I32
    lib.spd_msd_workspace_bytes.argtypes = [pp, I32, I32]
    lib.spd_msd_workspace_bytes.restype = SZ
    lib.spd_msd.argtypes = [pp, I32, I32, P, P, SZ, P]
    lib.spd_msd.restype = I32
    lib.spd_boxcar_snr_workspace_bytes.argtypes = [pp, I32, P, I32]
    lib.spd_boxcar_snr_workspace_bytes.restype = SZ
    lib.spd_boxcar_snr.argtypes = [pp, P, I32, P, I32, I32, P, P, I64, P, SZ, P]
    lib.spd_boxcar_snr.restype = I32
    lib.spd_threshold_candidates.argtypes = [P, P, I64, I64, I64, F, P, I64, P, P]
    lib.spd_threshold_candidates.restype = I32
    lib.spd_detect_workspace_bytes.argtypes = [pp, pq]
    lib.spd_detect_workspace_bytes.restype = SZ
    lib.spd_search_workspace_bytes.argtypes = [pp, pq]
    lib.spd_search_workspace_bytes.restype = SZ
    lib.spd_detect.argtypes = [pp, pq, P, P, I64, P, P, SZ, P]
    lib.spd_detect.restype = I32
    lib.spd_search.argtypes = [pp, pq, P, I64, P, P, P, SZ, P]
    lib.spd_search.restype = I32
    lib.spd_search_host_workspace_bytes.argtypes = [pp, pq, I64]
    lib.spd_search_host_workspace_bytes.restype = SZ
    lib.spd_search_host.argtypes = [pp, pq, P, I64, ctypes.POINTER(SpdResult), P, P, SZ, P]
    lib.spd_search_host.restype = I32
    lib.spd_boxcar_sums.argtypes = [pp, I32, P, I64, P]
    lib.spd_boxcar_sums.restype = I32
    lib.spd_dedisperse.argtypes = [pp, P, I64, P, I32, I64, I64, P, P]
    lib.spd_dedisperse.restype = I32
    pr = ctypes.POINTER(SpdRange)
    pt = ctypes.POINTER(SpdTuning)
    lib.spd_search_batched_workspace_bytes.argtypes = [pr, I32, pt]
    lib.spd_search_batched_workspace_bytes.restype = SZ
    lib.spd_search_batched.argtypes = [pr, I32, pt, P, I64, P, P, P, SZ, P]
    lib.spd_search_batched.restype = I32
    lib.spd_debug_set_copy_wait.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
    lib.spd_debug_set_copy_wait.restype = I32
    plv = ctypes.POINTER(SpdLevel)
    lib.spd_search_decimated_workspace_bytes.argtypes = [pp, plv, I32]
    lib.spd_search_decimated_workspace_bytes.restype = SZ
    lib.spd_search_decimated.argtypes = [pp, plv, I32, F, P, I64, P, P, P, SZ, P]
    lib.spd_search_decimated.restype = I32
    lib.spd_threshold_plane.argtypes = [P, P, I64, I64, I64, F, P]
    lib.spd_threshold_plane.restype = I32
    lib.spd_cluster_rows.argtypes = [P, P, I64, I64, I64, F, I32, P, I64, P, P]
    lib.spd_cluster_rows.restype = I32
    lib.spd_msd_shard_partial.argtypes = [pp, P, P, SZ, P]
    lib.spd_msd_shard_partial.restype = I32
    lib.spd_msd_merge_partials.argtypes = [P, I32, P, P]
    lib.spd_msd_merge_partials.restype = I32
    lib.spd_sd_nmax_shard_partial.argtypes = [pp, I32, P, P, P, SZ, P]
    lib.spd_sd_nmax_shard_partial.restype = I32
    lib.spd_sd_nmax_merge_partials.argtypes = [P, I32, I32, P, P]
    lib.spd_sd_nmax_merge_partials.restype = I32
    pi = ctypes.POINTER(SpdStreamInfo)
    lib.spd_stream_state_bytes.argtypes = [I64, I32, pq]
    lib.spd_stream_state_bytes.restype = SZ
    lib.spd_stream_workspace_bytes.argtypes = [I64, I64, I32, pq]
    lib.spd_stream_workspace_bytes.restype = SZ
    lib.spd_stream_reset.argtypes = [pi, P, I64, I32, pq, P]
    lib.spd_stream_reset.restype = I32
    lib.spd_stream_push.argtypes = [pi, P, pp, pq, P, I64, P, P, P, SZ, P]
    lib.spd_stream_push.restype = I32
    lib.spd_stream_chunk_view.argtypes = [pi, pq, I64, P, SZ, ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.POINTER(ctypes.c_int64)]
    lib.spd_stream_chunk_view.restype = I32
    lib.spd_stream_flush.argtypes = [pi, P, pq, P, I64, P, P, SZ, P]
    lib.spd_stream_flush.restype = I32
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != SPD_OK:
        raise SpdError(status, what)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


_DT = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}


@dataclass
class Plane:
    """A device plane: ``data`` [n_dm, row_stride] (float32 / float16 / bfloat16,
    row-major, unit stride along time); ``n_samp`` valid samples per row;
    optional float32 per-row ``scale`` / ``offset``."""
    data: torch.Tensor
    n_samp: int | None = None
    scale: torch.Tensor | None = None
    offset: torch.Tensor | None = None

    def __post_init__(self):
        if self.data.dtype not in _DT:
            raise TypeError(f"plane dtype {self.data.dtype} not supported")
        if self.data.dim() != 2 or self.data.stride(1) != 1:
            raise ValueError("plane must be 2-D with unit stride along time")
        if self.n_samp is None:
            self.n_samp = self.data.shape[1]

    @property
    def n_dm(self):
        return self.data.shape[0]

    def c(self) -> SpdPlane:
        d = self.data
        return SpdPlane(d.data_ptr() if d.numel() else 0, _DT[d.dtype], 0, d.shape[0],
                        self.n_samp, d.stride(0) if d.shape[0] else self.n_samp,
                        self.scale.data_ptr() if self.scale is not None else None,
                        self.offset.data_ptr() if self.offset is not None else None)


def as_plane(x, **kw) -> Plane:
    return x if isinstance(x, Plane) else Plane(x, **kw)


def _params(widths, threshold, sigma_mode, scope, nmax_sigma):
    w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
    p = SpdSearchParams(w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), w.size,
                        float(threshold), int(sigma_mode), int(scope), int(nmax_sigma), 0)
    return p, w


def _workspace(nbytes: int, device) -> torch.Tensor:
    # 256-byte aligned: torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def entries(plane: Plane, scope: int) -> int:
    return plane.n_dm if scope == MSD_PER_ROW else 1


# --------------------------------------------------------------------- calls

def msd(x, scope=MSD_GLOBAL, nmax_sigma=0, *, stream=None, out=None, workspace=None,
        **kw) -> torch.Tensor:
    """spd_msd: returns a uint8 device tensor holding 1 or n_dm spd_msd_stats."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    n = entries(pl, scope)
    if out is None:
        out = torch.empty(max(n, 1) * MSD_BYTES, dtype=torch.uint8, device=pl.data.device)
    wsb = lib.spd_msd_workspace_bytes(ctypes.byref(cp), scope, nmax_sigma)
    ws = workspace if workspace is not None else _workspace(wsb, pl.data.device)
    _check(lib.spd_msd(ctypes.byref(cp), scope, nmax_sigma, _ptr(out), _ptr(ws), wsb,
                       _stream(stream)), "spd_msd")
    return out


def msd_shard_partial(x, *, stream=None, out=None, workspace=None, **kw) -> torch.Tensor:
    """spd_msd_shard_partial: the shard's spd_msd_part (uint8 device tensor, 40 B)."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    if out is None:
        out = torch.empty(PART_BYTES, dtype=torch.uint8, device=pl.data.device)
    wsb = lib.spd_msd_workspace_bytes(ctypes.byref(cp), MSD_GLOBAL, 0)
    ws = workspace if workspace is not None else _workspace(wsb, pl.data.device)
    _check(lib.spd_msd_shard_partial(ctypes.byref(cp), _ptr(out), _ptr(ws), ws.numel(),
                                     _stream(stream)), "spd_msd_shard_partial")
    return out


def msd_merge_partials(parts: torch.Tensor, n_shards: int, *, stream=None, out=None):
    """spd_msd_merge_partials over n_shards gathered parts (shard order)."""
    lib = load()
    if out is None:
        out = torch.empty(MSD_BYTES, dtype=torch.uint8, device=parts.device)
    _check(lib.spd_msd_merge_partials(_ptr(parts), int(n_shards), _ptr(out), _stream(stream)),
           "spd_msd_merge_partials")
    return out


def sd_nmax_shard_partial(x, nmax, msd_dev, *, stream=None, out=None, workspace=None, **kw):
    """spd_sd_nmax_shard_partial: the shard's B_Nmax-series partial."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    if out is None:
        out = torch.empty(PART_BYTES, dtype=torch.uint8, device=pl.data.device)
    wsb = lib.spd_msd_workspace_bytes(ctypes.byref(cp), MSD_GLOBAL, int(nmax))
    ws = workspace if workspace is not None else _workspace(wsb, pl.data.device)
    _check(lib.spd_sd_nmax_shard_partial(ctypes.byref(cp), int(nmax), _ptr(msd_dev), _ptr(out),
                                         _ptr(ws), ws.numel(), _stream(stream)),
           "spd_sd_nmax_shard_partial")
    return out


def sd_nmax_merge_partials(parts: torch.Tensor, n_shards: int, nmax: int, out: torch.Tensor, *,
                           stream=None):
    """spd_sd_nmax_merge_partials: sd_nmax / nmax of `out` from the gathered parts."""
    _check(load().spd_sd_nmax_merge_partials(_ptr(parts), int(n_shards), int(nmax), _ptr(out),
                                             _stream(stream)), "spd_sd_nmax_merge_partials")
    return out


def msd_to_numpy(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(MSD_DTYPE)


def boxcar_snr(x, msd_dev, widths, sigma_mode=SIGMA_SQRTN, scope=MSD_GLOBAL, *, stream=None,
               snr_out=None, width_out=None, **kw):
    """spd_boxcar_snr: (snr float32 [n_dm, n_samp], width int16 [n_dm, n_samp]
    holding uint16 widths)."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
    dev = pl.data.device
    if snr_out is None:
        snr_out = torch.empty((pl.n_dm, pl.n_samp), dtype=torch.float32, device=dev)
    if width_out is None:
        width_out = torch.empty((pl.n_dm, pl.n_samp), dtype=torch.int16, device=dev)
    wsb = lib.spd_boxcar_snr_workspace_bytes(ctypes.byref(cp), scope, w.ctypes.data, w.size)
    ws = _workspace(wsb, dev)
    _check(lib.spd_boxcar_snr(ctypes.byref(cp), _ptr(msd_dev), scope, w.ctypes.data, w.size,
                              sigma_mode, _ptr(snr_out), _ptr(width_out), snr_out.stride(0),
                              _ptr(ws), wsb, _stream(stream)), "spd_boxcar_snr")
    return snr_out, width_out


def threshold_candidates(snr, width, threshold, capacity, *, n_samp=None, stream=None,
                         out=None, result=None):
    """spd_threshold_candidates: (records int32 [capacity, 4], result uint8 [16])."""
    lib = load()
    dev = snr.device
    n_dm, n = snr.shape[0], (snr.shape[1] if n_samp is None else n_samp)
    if out is None:
        out = torch.empty((max(int(capacity), 1), 4), dtype=torch.int32, device=dev)
    if result is None:
        result = torch.empty(RESULT_BYTES, dtype=torch.uint8, device=dev)
    _check(lib.spd_threshold_candidates(_ptr(snr), _ptr(width), n_dm, n, snr.stride(0),
                                        float(threshold), _ptr(out), int(capacity),
                                        _ptr(result), _stream(stream)),
           "spd_threshold_candidates")
    return out, result


def cluster_rows(snr, width, threshold, max_gap, capacity, *, n_samp=None, stream=None,
                 out=None, result=None):
    """spd_cluster_rows: per-DM clusters of the candidates (snr >= threshold),
    a gap of at most max_gap samples joining neighbours; returns (records int32
    [capacity, 8], result uint8 [16]).  Decode with clusters_to_numpy."""
    # the C ABI reads raw float32 / 16-bit rows at one shared stride
    if snr.dtype != torch.float32:
        raise ValueError("snr plane must be float32")
    if width.dtype not in (torch.int16, torch.uint16):
        raise ValueError("width plane must be 16-bit (int16 or uint16)")
    if snr.device != width.device:
        raise ValueError("snr and width planes must be on the same device")
    if snr.dim() != 2 or width.dim() != 2 or snr.stride(1) != 1 or width.stride(1) != 1:
        raise ValueError("snr and width planes must be 2-D with contiguous rows")
    if width.stride(0) != snr.stride(0):
        raise ValueError("snr and width planes must share a row stride")
    lib = load()
    dev = snr.device
    n_dm, n = snr.shape[0], (snr.shape[1] if n_samp is None else n_samp)
    if out is None:
        out = torch.empty((max(int(capacity), 1), 8), dtype=torch.int32, device=dev)
    if result is None:
        result = torch.empty(RESULT_BYTES, dtype=torch.uint8, device=dev)
    _check(lib.spd_cluster_rows(_ptr(snr), _ptr(width), n_dm, n, snr.stride(0),
                                float(threshold), int(max_gap), _ptr(out), int(capacity),
                                _ptr(result), _stream(stream)), "spd_cluster_rows")
    return out, result


def clusters_to_numpy(out: torch.Tensor, count: int) -> np.ndarray:
    n = min(int(count), out.shape[0])
    return out[:n].detach().cpu().numpy().view(CLUSTER_DTYPE).reshape(-1)


def threshold_plane(snr, width, threshold, *, n_samp=None, stream=None):
    """spd_threshold_plane, in place: SNR (and width) kept where SNR >=
    threshold, 0 elsewhere (Sec. 2.4)."""
    n_samp = snr.shape[1] if n_samp is None else n_samp
    if width is not None and width.stride(0) != snr.stride(0):
        raise ValueError("snr and width planes must share a row stride")
    _check(load().spd_threshold_plane(_ptr(snr), _ptr(width), snr.shape[0], int(n_samp),
                                      snr.stride(0), float(threshold), _stream(stream)),
           "spd_threshold_plane")
    return snr, width


def detect(x, msd_dev, widths, threshold, capacity, sigma_mode=SIGMA_SQRTN, scope=MSD_GLOBAL,
           nmax_sigma=0, *, stream=None, out=None, result=None, workspace=None, **kw):
    """spd_detect (steps b-d given the MSD): (records, result)."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    dev = pl.data.device
    prm, keep = _params(widths, threshold, sigma_mode, scope, nmax_sigma)
    if out is None:
        out = torch.empty((max(int(capacity), 1), 4), dtype=torch.int32, device=dev)
    if result is None:
        result = torch.empty(RESULT_BYTES, dtype=torch.uint8, device=dev)
    wsb = lib.spd_detect_workspace_bytes(ctypes.byref(cp), ctypes.byref(prm))
    ws = workspace if workspace is not None else _workspace(wsb, dev)
    _check(lib.spd_detect(ctypes.byref(cp), ctypes.byref(prm), _ptr(msd_dev), _ptr(out),
                          int(capacity), _ptr(result), _ptr(ws), wsb, _stream(stream)),
           "spd_detect")
    del keep
    return out, result


def search_workspace_bytes(x, widths, threshold=0.0, sigma_mode=SIGMA_SQRTN,
                           scope=MSD_GLOBAL, nmax_sigma=0, **kw) -> int:
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    prm, keep = _params(widths, threshold, sigma_mode, scope, nmax_sigma)
    return int(lib.spd_search_workspace_bytes(ctypes.byref(cp), ctypes.byref(prm)))


def search(x, widths, threshold, capacity, sigma_mode=SIGMA_SQRTN, scope=MSD_GLOBAL,
           nmax_sigma=0, *, stream=None, out=None, result=None, msd_out=None,
           workspace=None, **kw):
    """spd_search (the whole path): (records int32 [capacity, 4], result, msd)."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    dev = pl.data.device
    prm, keep = _params(widths, threshold, sigma_mode, scope, nmax_sigma)
    if out is None:
        out = torch.empty((max(int(capacity), 1), 4), dtype=torch.int32, device=dev)
    if result is None:
        result = torch.empty(RESULT_BYTES, dtype=torch.uint8, device=dev)
    if msd_out is None:
        msd_out = torch.empty(max(entries(pl, scope), 1) * MSD_BYTES, dtype=torch.uint8,
                              device=dev)
    wsb = lib.spd_search_workspace_bytes(ctypes.byref(cp), ctypes.byref(prm))
    ws = workspace if workspace is not None else _workspace(wsb, dev)
    _check(lib.spd_search(ctypes.byref(cp), ctypes.byref(prm), _ptr(out), int(capacity),
                          _ptr(result), _ptr(msd_out), _ptr(ws), wsb, _stream(stream)),
           "spd_search")
    del keep
    return out, result, msd_out


def debug_set_copy_wait(limit_ns=2_000_000_000, extra_bytes=0):
    """spd_debug_set_copy_wait (test aid): bound of the fused kernel's waits
    for tile copies, and bytes expected beyond each copy (> 0 makes every wait
    run out); the defaults restore normal operation."""
    _check(load().spd_debug_set_copy_wait(int(limit_ns), int(extra_bytes)),
           "spd_debug_set_copy_wait")


def search_host_workspace_bytes(x, widths, threshold, capacity, sigma_mode=SIGMA_SQRTN,
                                scope=MSD_GLOBAL, nmax_sigma=0, **kw) -> int:
    lib = load()
    cp = as_plane(x, **kw).c()
    prm, keep = _params(widths, threshold, sigma_mode, scope, nmax_sigma)
    return int(lib.spd_search_host_workspace_bytes(ctypes.byref(cp), ctypes.byref(prm),
                                                   int(capacity)))


def search_host(x, widths, threshold, out, sigma_mode=SIGMA_SQRTN, scope=MSD_GLOBAL,
                nmax_sigma=0, *, workspace, stream=None, msd_out=None, **kw):
    """spd_search_host: the whole search of a plane in HOST memory (x and its
    scale / offset on the host, best page-locked); ``out``: host int32
    [capacity, 4] receiving the records; ``workspace``: device uint8 tensor of
    search_host_workspace_bytes.  Blocking.  Returns (count, status)."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    prm, keep = _params(widths, threshold, sigma_mode, scope, nmax_sigma)
    res = SpdResult()
    _check(lib.spd_search_host(ctypes.byref(cp), ctypes.byref(prm), _ptr(out), out.shape[0],
                               ctypes.byref(res), _ptr(msd_out), _ptr(workspace),
                               workspace.numel(), _stream(stream)), "spd_search_host")
    del keep
    return int(res.count), int(res.status)


def dedisperse(fb, delays, n_out, *, out=None, out_dtype=F32, status=None, stream=None, **kw):
    """spd_dedisperse: the DM x time plane of a filterbank (channel rows),
    out[d, t] = sum over channels c of fb[c, t + delays[d, c]].  ``delays``:
    device int32 [n_dm, n_chan]; ``out``: a [n_dm, n_out] device tensor with
    contiguous rows (e.g. BeamStream.chunk_view), made when None."""
    lib = load()
    pl = as_plane(fb, **kw)
    cp = pl.c()
    if not (isinstance(delays, torch.Tensor) and delays.dtype == torch.int32
            and delays.is_contiguous() and delays.dim() == 2):
        raise ValueError("delays must be a contiguous int32 [n_dm, n_chan] tensor")
    n_dm = delays.shape[0]
    if out is None:
        out = torch.empty((n_dm, int(n_out)), dtype=_TD[out_dtype], device=pl.data.device)
    dt = {v: k for k, v in _TD.items()}.get(out.dtype)
    if dt is None or out.dim() != 2 or out.stride(1) != 1 or out.shape[0] != n_dm:
        raise ValueError("out must be [n_dm, >= n_out] f32/f16/bf16 with contiguous rows")
    _check(lib.spd_dedisperse(ctypes.byref(cp), _ptr(delays), n_dm, _ptr(out), dt, int(n_out),
                              out.stride(0), _ptr(status), _stream(stream)), "spd_dedisperse")
    return out


def boxcar_sums(x, w, *, stream=None, out=None, **kw):
    """spd_boxcar_sums: raw B_w(i), NaN past the row end."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    if out is None:
        out = torch.empty((pl.n_dm, pl.n_samp), dtype=torch.float32, device=pl.data.device)
    _check(lib.spd_boxcar_sums(ctypes.byref(cp), int(w), _ptr(out), out.stride(0),
                               _stream(stream)), "spd_boxcar_sums")
    return out


# ------------------------------------------------------------------ batched

@dataclass
class RangeSpec:
    """One DM range of a batched search (see spd_range in include/spd.h)."""
    x: object                       # torch tensor or Plane
    widths: list
    threshold: float
    sigma_mode: int = SIGMA_SQRTN
    scope: int = MSD_GLOBAL
    nmax: int = 0
    dm_offset: int = 0
    decimation: int = 1


class _Ranges:
    """ctypes array of spd_range built from RangeSpecs (keeps the width arrays alive)."""

    def __init__(self, specs):
        self.specs = list(specs)
        self.planes = [as_plane(r.x) for r in self.specs]
        self.keep = []
        arr = (SpdRange * len(self.specs))()
        for i, (r, pl) in enumerate(zip(self.specs, self.planes)):
            prm, w = _params(r.widths, r.threshold, r.sigma_mode, r.scope, r.nmax)
            self.keep.append(w)
            arr[i] = SpdRange(pl.c(), prm, int(r.dm_offset), int(r.decimation))
        self.arr = arr

    def n_entries(self):
        return sum(entries(pl, r.scope) for r, pl in zip(self.specs, self.planes))


def _tuning(t):
    if t is None:
        return None
    if isinstance(t, SpdTuning):
        return t
    return SpdTuning(int(t.get("ctas_per_sm", 0)), int(t.get("group_scale", 1)),
                     int(t.get("tile_threads", 0)), 0)


def search_batched_workspace_bytes(specs, tuning=None) -> int:
    lib = load()
    rg = specs if isinstance(specs, _Ranges) else _Ranges(specs)
    t = _tuning(tuning)
    return int(lib.spd_search_batched_workspace_bytes(rg.arr, len(rg.specs),
                                                      ctypes.byref(t) if t else None))


def search_batched(specs, capacity, tuning=None, *, stream=None, out=None, result=None,
                   msd_out=None, workspace=None):
    """spd_search_batched: (records int32 [capacity, 4], result, msd of every range)."""
    lib = load()
    rg = specs if isinstance(specs, _Ranges) else _Ranges(specs)
    dev = rg.planes[0].data.device
    t = _tuning(tuning)
    if out is None:
        out = torch.empty((max(int(capacity), 1), 4), dtype=torch.int32, device=dev)
    if result is None:
        result = torch.empty(RESULT_BYTES, dtype=torch.uint8, device=dev)
    if msd_out is None:
        msd_out = torch.empty(max(rg.n_entries(), 1) * MSD_BYTES, dtype=torch.uint8, device=dev)
    wsb = lib.spd_search_batched_workspace_bytes(rg.arr, len(rg.specs),
                                                 ctypes.byref(t) if t else None)
    ws = workspace if workspace is not None else _workspace(wsb, dev)
    _check(lib.spd_search_batched(rg.arr, len(rg.specs), ctypes.byref(t) if t else None,
                                  _ptr(out), int(capacity), _ptr(result), _ptr(msd_out),
                                  _ptr(ws), wsb, _stream(stream)), "spd_search_batched")
    return out, result, msd_out


class BatchedSearch:
    """A batched search with every buffer allocated once; with graph=True the
    whole call (MSD launches, constants, the persistent detect launch) is
    captured in a CUDA graph and replayed by run()."""

    def __init__(self, specs, capacity, tuning=None, graph=True):
        self.ranges = _Ranges(specs)
        self.capacity = int(capacity)
        self.tuning = _tuning(tuning)
        dev = self.ranges.planes[0].data.device
        self.out = torch.empty((max(self.capacity, 1), 4), dtype=torch.int32, device=dev)
        self.result = torch.zeros(RESULT_BYTES, dtype=torch.uint8, device=dev)
        self.msd = torch.empty(max(self.ranges.n_entries(), 1) * MSD_BYTES, dtype=torch.uint8,
                               device=dev)
        wsb = search_batched_workspace_bytes(self.ranges, self.tuning)
        self.ws = _workspace(wsb, dev)
        self.graph = None
        if graph:
            s = torch.cuda.Stream(device=dev)
            s.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(s):
                self._call(s)          # warm-up outside capture (attributes, lazy loading)
            torch.cuda.current_stream(dev).wait_stream(s)
            torch.cuda.synchronize(dev)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._call(None)

    def _call(self, stream):
        search_batched(self.ranges, self.capacity, self.tuning, stream=stream, out=self.out,
                       result=self.result, msd_out=self.msd, workspace=self.ws)

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._call(None)
        return self.out, self.result


# ------------------------------------------------------------- decimation

def _levels(levels):
    arr = (SpdLevel * len(levels))()
    keep = []
    for i, (lvl, widths) in enumerate(levels):
        w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
        keep.append(w)
        arr[i] = SpdLevel(int(lvl), w.size, w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return arr, keep


def search_decimated_workspace_bytes(x, levels, **kw) -> int:
    pl = as_plane(x, **kw)
    cp = pl.c()
    arr, keep = _levels(levels)
    return int(load().spd_search_decimated_workspace_bytes(ctypes.byref(cp), arr, len(levels)))


def search_decimated(x, levels, threshold, capacity, *, stream=None, out=None, result=None,
                     msd_out=None, workspace=None, **kw):
    """spd_search_decimated: levels = [(level, widths in level samples), ...];
    returns (records in native units, result, msd of every level)."""
    lib = load()
    pl = as_plane(x, **kw)
    cp = pl.c()
    dev = pl.data.device
    arr, keep = _levels(levels)
    if out is None:
        out = torch.empty((max(int(capacity), 1), 4), dtype=torch.int32, device=dev)
    if result is None:
        result = torch.empty(RESULT_BYTES, dtype=torch.uint8, device=dev)
    if msd_out is None:
        msd_out = torch.empty(len(levels) * MSD_BYTES, dtype=torch.uint8, device=dev)
    wsb = lib.spd_search_decimated_workspace_bytes(ctypes.byref(cp), arr, len(levels))
    if wsb == 0:
        raise SpdError(SPD_ERR_INVALID_ARG, "spd_search_decimated_workspace_bytes")
    ws = workspace if workspace is not None else _workspace(wsb, dev)
    _check(lib.spd_search_decimated(ctypes.byref(cp), arr, len(levels), float(threshold),
                                    _ptr(out), int(capacity), _ptr(result), _ptr(msd_out),
                                    _ptr(ws), ws.numel(), _stream(stream)),
           "spd_search_decimated")
    return out, result, msd_out


# ---------------------------------------------------------------- streaming

_TD = {F32: torch.float32, F16: torch.float16, BF16: torch.bfloat16}


class BeamStream:
    """One beam's stream state (spd_stream_* in include/spd.h): a device state
    buffer holding the running MSD and the halo, and the host spd_stream_info.

    ``state`` may be a caller-provided uint8 device tensor of at least
    :meth:`state_bytes` bytes (256-byte aligned).  Every push / flush runs on
    the given CUDA stream; pushes of one beam must be ordered on the device
    (same stream, or an event wait) because they share the state."""

    def __init__(self, n_dm, dtype, widths, threshold, scope=MSD_GLOBAL, *, device="cuda",
                 state=None, stream=None):
        self.lib = load()
        self.n_dm = int(n_dm)
        self.dtype = dtype if isinstance(dtype, int) else _DT[dtype]
        self.widths = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
        self.threshold = float(threshold)
        self.scope = int(scope)
        self.params = SpdSearchParams(self.widths.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      self.widths.size, self.threshold, SIGMA_SQRTN,
                                      self.scope, 0, 0)
        nb = self.state_bytes()
        if nb == 0:
            raise SpdError(SPD_ERR_INVALID_ARG, "spd_stream_state_bytes")
        self.state = state if state is not None else _workspace(nb, device)
        self.info = SpdStreamInfo()
        self.reset(stream)

    def state_bytes(self) -> int:
        return int(self.lib.spd_stream_state_bytes(self.n_dm, self.dtype,
                                                   ctypes.byref(self.params)))

    def workspace_bytes(self, max_chunk: int) -> int:
        return int(self.lib.spd_stream_workspace_bytes(self.n_dm, int(max_chunk), self.dtype,
                                                       ctypes.byref(self.params)))

    def reset(self, stream=None):
        _check(self.lib.spd_stream_reset(ctypes.byref(self.info), _ptr(self.state), self.n_dm,
                                         self.dtype, ctypes.byref(self.params), _stream(stream)),
               "spd_stream_reset")

    @property
    def seen(self) -> int:
        return int(self.info.seen)

    @property
    def halo(self) -> int:
        return int(self.info.halo)

    def chunk_view(self, n_samp: int, workspace: torch.Tensor) -> torch.Tensor:
        """A [n_dm, n_samp] view into ``workspace`` where the next push of this
        beam reads a chunk in place (the caller fills it, then pushes it)."""
        ptr, stride = ctypes.c_void_p(), ctypes.c_int64()
        _check(self.lib.spd_stream_chunk_view(ctypes.byref(self.info), ctypes.byref(self.params),
                                              int(n_samp), _ptr(workspace), workspace.numel(),
                                              ctypes.byref(ptr), ctypes.byref(stride)),
               "spd_stream_chunk_view")
        td = _TD[self.dtype]
        eb = torch.empty((), dtype=td).element_size()
        off = ptr.value - workspace.data_ptr()
        n = ((self.n_dm - 1) * stride.value + int(n_samp)) * eb
        flat = workspace[off:off + n].view(td)
        return flat.as_strided((self.n_dm, int(n_samp)), (stride.value, 1))

    def push(self, chunk, out, capacity, result, workspace, *, msd_out=None, stream=None,
             **kw):
        """spd_stream_push of one chunk (a device Plane or tensor)."""
        pl = as_plane(chunk, **kw)
        cp = pl.c()
        _check(self.lib.spd_stream_push(ctypes.byref(self.info), _ptr(self.state),
                                        ctypes.byref(cp), ctypes.byref(self.params), _ptr(out),
                                        int(capacity), _ptr(result), _ptr(msd_out),
                                        _ptr(workspace), workspace.numel(), _stream(stream)),
               "spd_stream_push")

    def flush(self, out, capacity, result, workspace, *, stream=None):
        """spd_stream_flush: search the held-back starts at the end of the stream."""
        _check(self.lib.spd_stream_flush(ctypes.byref(self.info), _ptr(self.state),
                                         ctypes.byref(self.params), _ptr(out), int(capacity),
                                         _ptr(result), _ptr(workspace), workspace.numel(),
                                         _stream(stream)), "spd_stream_flush")


# ------------------------------------------------------------------ decoding

def read_result(result: torch.Tensor) -> tuple[int, int]:
    """(count, status) of a device spd_result (synchronises)."""
    r = result.detach().cpu().numpy()
    return int(r[:8].view(np.uint64)[0]), int(r[8:12].view(np.int32)[0])


def candidates_to_numpy(out: torch.Tensor, count: int) -> np.ndarray:
    n = min(int(count), out.shape[0])
    return out[:n].detach().cpu().numpy().view(CAND_DTYPE).reshape(-1)


def widths_to_numpy(width: torch.Tensor) -> np.ndarray:
    return width.detach().cpu().numpy().view(np.uint16).astype(np.int32)
