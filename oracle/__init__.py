"""FP64 CPU oracle for the single-pulse search (Adamek & Armour, arXiv:1611.09704).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
never does, and it shares no code with the CUDA path.

The arithmetic lives in ``spd_oracle.c`` (plain C, FP64), built into
``oracle/_build/liboracle.so`` by :func:`build`.  This module only marshals
numpy arrays.  Function by function:

- :func:`twopass`, :func:`chan_stream`, :func:`chan_merge` -- Sec. 2.1: the
  two-pass definition of mean and population sd, Eq. 1 and Eq. 2.
- :func:`plane_msd`, :func:`plane_msd_chan` -- the MSD of a DM x time plane
  (whole plane or per row), by definition and by the block scheme of Sec. 2.1.
- :func:`plane_sd_nmax`, :func:`sigma_table` -- Sec. 2.2, Eq. 4 and Eq. 5.
- :func:`boxcar_sums`, :func:`boxcar_snr` -- Sec. 2.3 and Algorithm 1.
- :func:`threshold` -- Sec. 2.4.
- :func:`search` -- the four steps in order.
- :func:`stream_replay` -- the same search over a stream delivered in chunks
  (running MSD, held-back starts, end-of-stream flush).
- :func:`decimate`, :func:`search_decimated` -- boxcars on data decimated in
  time (Sec. 3), level by level.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

SIGMA_SQRTN, SIGMA_LINEAR, SIGMA_LINEAR_EXCESS = 0, 1, 2
SCOPE_GLOBAL, SCOPE_PER_ROW = 0, 1
_DTYPES = {"f32": 0, "f16": 1, "bf16": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over rows, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
            "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.oracle_twopass.argtypes = [P, I64, P, P]
    lib.oracle_chan_stream.argtypes = [P, I64, P, P]
    lib.oracle_chan_merge.argtypes = [D, D, D, D, D, D, P, P]
    lib.oracle_plane_msd.argtypes = [P, I32, I64, I64, I64, P, P, I32, P, P]
    lib.oracle_plane_msd.restype = I32
    lib.oracle_plane_msd_chan.argtypes = [P, I32, I64, I64, I64, P, P, I64, I32, P, P]
    lib.oracle_plane_msd_chan.restype = I32
    lib.oracle_plane_sd_nmax.argtypes = [P, I32, I64, I64, I64, P, P, I32, I32, P]
    lib.oracle_plane_sd_nmax.restype = I32
    lib.oracle_sigma_table.argtypes = [I32, D, D, I32, P, I32, P]
    lib.oracle_sigma_table.restype = I32
    lib.oracle_boxcar_sums.argtypes = [P, I32, I64, I64, I64, P, P, I32, P]
    lib.oracle_boxcar_sums.restype = I32
    lib.oracle_boxcar_snr.argtypes = [P, I32, I64, I64, I64, P, P, I32, P, P, P, P,
                                      I32, I64, I64, P, P, I32]
    lib.oracle_boxcar_snr.restype = I32
    lib.oracle_threshold.argtypes = [P, P, I64, I64, I64, D, P, P, P, P, I64]
    lib.oracle_threshold.restype = I64
    lib.oracle_dequant_row.argtypes = [P, I32, I64, P, P, I64, I64, P]
    lib.oracle_num_threads.restype = I32
    lib.oracle_snr_at.argtypes = [P, I32, I64, I64, P, P, I64, I64, I32, D, D]
    lib.oracle_snr_at.restype = D
    lib.oracle_dedisperse.argtypes = [P, I32, I64, I64, I64, P, P, P, I64, I64, P]
    lib.oracle_dedisperse.restype = I32
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def num_threads() -> int:
    """OpenMP threads the oracle's row loops use."""
    return int(_load().oracle_num_threads())


@dataclass
class Plane:
    """A DM x time plane on the host: ``data`` is float32 [n_dm, stride] or the
    uint16 bit patterns of FP16 / BF16; ``n_samp`` <= stride valid samples per
    row; optional float32 per-row ``scale`` / ``offset``
    (value = fmaf(scale, q, offset))."""
    data: np.ndarray
    dtype: str = "f32"
    n_samp: int | None = None
    scale: np.ndarray | None = None
    offset: np.ndarray | None = None

    def __post_init__(self):
        if self.dtype not in _DTYPES:
            raise ValueError(f"dtype {self.dtype!r}")
        want = np.float32 if self.dtype == "f32" else np.uint16
        self.data = np.ascontiguousarray(self.data, dtype=want)
        if self.data.ndim != 2:
            raise ValueError("plane must be 2-D")
        if self.n_samp is None:
            self.n_samp = self.data.shape[1]
        if self.scale is not None:
            self.scale = np.ascontiguousarray(self.scale, dtype=np.float32)
        if self.offset is not None:
            self.offset = np.ascontiguousarray(self.offset, dtype=np.float32)

    @property
    def n_dm(self) -> int:
        return self.data.shape[0]

    @property
    def stride(self) -> int:
        return self.data.shape[1]

    def args(self):
        return (_ptr(self.data), _DTYPES[self.dtype], self.n_dm, self.n_samp,
                self.stride, _ptr(self.scale), _ptr(self.offset))

    def values(self) -> np.ndarray:
        """Dequantised float64 values [n_dm, n_samp] (small planes only)."""
        out = np.empty((self.n_dm, self.n_samp), dtype=np.float64)
        lib = _load()
        for r in range(self.n_dm):
            lib.oracle_dequant_row(_ptr(self.data), _DTYPES[self.dtype], self.stride,
                                   _ptr(self.scale), _ptr(self.offset), r, self.n_samp,
                                   out[r].ctypes.data)
        return out


def as_plane(x, **kw) -> Plane:
    return x if isinstance(x, Plane) else Plane(np.asarray(x), **kw)


# ----------------------------------------------------------------- Sec. 2.1

def twopass(x) -> tuple[float, float]:
    """Definition: (mean, population sd) of a 1-D sample."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m, s = ctypes.c_double(), ctypes.c_double()
    _load().oracle_twopass(_ptr(x), x.size, ctypes.byref(m), ctypes.byref(s))
    return m.value, s.value


def chan_stream(x) -> tuple[float, float]:
    """Eq. 1 over a 1-D sample: returns (T, S)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    T, S = ctypes.c_double(), ctypes.c_double()
    _load().oracle_chan_stream(_ptr(x), x.size, ctypes.byref(T), ctypes.byref(S))
    return T.value, S.value


def chan_merge(m, Ta, Sa, n, Tb, Sb) -> tuple[float, float]:
    """Eq. 2: (T, S) of the union of an m-sample set and an n-sample set."""
    T, S = ctypes.c_double(), ctypes.c_double()
    _load().oracle_chan_merge(float(m), float(Ta), float(Sa), float(n), float(Tb),
                              float(Sb), ctypes.byref(T), ctypes.byref(S))
    return T.value, S.value


def plane_msd(plane, scope: int = SCOPE_GLOBAL):
    """Two-pass MSD of a plane: arrays (mean, sd) of length 1 or n_dm."""
    p = as_plane(plane)
    k = 1 if scope == SCOPE_GLOBAL else p.n_dm
    mean, sd = np.zeros(k), np.zeros(k)
    rc = _load().oracle_plane_msd(*p.args(), scope, _ptr(mean), _ptr(sd))
    if rc:
        raise ValueError(f"oracle_plane_msd rc={rc}")
    return mean, sd


def plane_msd_chan(plane, block: int, scope: int = SCOPE_GLOBAL):
    """Block scheme of Sec. 2.1 (Eq. 1 per block, Eq. 2 merges)."""
    p = as_plane(plane)
    k = 1 if scope == SCOPE_GLOBAL else p.n_dm
    mean, sd = np.zeros(k), np.zeros(k)
    rc = _load().oracle_plane_msd_chan(*p.args(), int(block), scope, _ptr(mean), _ptr(sd))
    if rc:
        raise ValueError(f"oracle_plane_msd_chan rc={rc}")
    return mean, sd


# ----------------------------------------------------------------- Sec. 2.2

def plane_sd_nmax(plane, nmax: int, scope: int = SCOPE_GLOBAL) -> np.ndarray:
    """sigma_Nmax of Eq. 5: measured sd of the Nmax-sample boxcar series."""
    p = as_plane(plane)
    k = 1 if scope == SCOPE_GLOBAL else p.n_dm
    out = np.zeros(k)
    rc = _load().oracle_plane_sd_nmax(*p.args(), int(nmax), scope, _ptr(out))
    if rc:
        raise ValueError(f"oracle_plane_sd_nmax rc={rc}")
    return out


def sigma_table(mode: int, sd: float, widths, sd_nmax: float = 0.0, nmax: int = 0):
    """sigma_N per width: Eq. 4 (mode 0) or Eq. 5 (modes 1, 2)."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    out = np.zeros(w.size)
    rc = _load().oracle_sigma_table(int(mode), float(sd), float(sd_nmax), int(nmax),
                                    _ptr(w), w.size, _ptr(out))
    if rc:
        raise ValueError("sigma_table: Eq. 5 needs nmax >= 2")
    return out


# ----------------------------------------------------------------- Sec. 2.3

def boxcar_sums(plane, w: int) -> np.ndarray:
    """B_w(i) for every start i (NaN where the window passes the row end)."""
    p = as_plane(plane)
    out = np.empty((p.n_dm, p.n_samp))
    _load().oracle_boxcar_sums(*p.args(), int(w), _ptr(out))
    return out


def boxcar_snr(plane, mean, sd, sigma_tab, widths, scope: int = SCOPE_GLOBAL,
               rows: tuple[int, int] | None = None, start_w1: bool = True):
    """Algorithm 1: per-sample (highest SNR, winning width) for rows [r0, r1).

    mean, sd: arrays of length 1 (global scope) or n_dm (per row);
    sigma_tab: [entries, n_widths] sigma_w.  start_w1=False evaluates only the
    listed widths (no width-1 start; -inf and width 0 where none fits)."""
    p = as_plane(plane)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    r0, r1 = rows if rows is not None else (0, p.n_dm)
    mean = np.ascontiguousarray(np.atleast_1d(mean), dtype=np.float64)
    sd = np.ascontiguousarray(np.atleast_1d(sd), dtype=np.float64)
    tab = np.ascontiguousarray(np.atleast_2d(sigma_tab), dtype=np.float64)
    best = np.empty((r1 - r0, p.n_samp))
    win = np.empty((r1 - r0, p.n_samp), dtype=np.int32)
    rc = _load().oracle_boxcar_snr(*p.args(), scope, _ptr(mean), _ptr(sd), _ptr(tab),
                                   _ptr(w), w.size, r0, r1, _ptr(best), _ptr(win),
                                   1 if start_w1 else 0)
    if rc:
        raise ValueError(f"oracle_boxcar_snr rc={rc}")
    return best, win


def snr_at(plane, row: int, sample: int, width: int, mean: float, sigma_w: float) -> float:
    """(B_w(i) - w mu) / sigma_w for one (row, start, width), NaN past the row end."""
    p = as_plane(plane)
    return float(_load().oracle_snr_at(_ptr(p.data), _DTYPES[p.dtype], p.n_samp, p.stride,
                                       _ptr(p.scale), _ptr(p.offset), int(row), int(sample),
                                       int(width), float(mean), float(sigma_w)))


# ----------------------------------------------------------------- Sec. 2.4

def threshold(best, width, thr: float, row0: int = 0):
    """Candidates with best >= thr, in (dm, sample) order, as a structured array."""
    best = np.ascontiguousarray(best, dtype=np.float64)
    width = np.ascontiguousarray(width, dtype=np.int32)
    n_rows, n_samp = best.shape
    lib = _load()
    cnt = lib.oracle_threshold(_ptr(best), _ptr(width), n_rows, n_samp, row0, float(thr),
                               None, None, None, None, 0)
    dm = np.empty(cnt, np.int32)
    sm = np.empty(cnt, np.int32)
    snr = np.empty(cnt, np.float64)
    wd = np.empty(cnt, np.int32)
    lib.oracle_threshold(_ptr(best), _ptr(width), n_rows, n_samp, row0, float(thr),
                         _ptr(dm), _ptr(sm), _ptr(snr), _ptr(wd), cnt)
    out = np.empty(cnt, dtype=[("dm", np.int32), ("sample", np.int32),
                               ("snr", np.float64), ("width", np.int32)])
    out["dm"], out["sample"], out["snr"], out["width"] = dm, sm, snr, wd
    return out


def threshold_plane(best, width, thr: float):
    """Sec. 2.4's thresholding on the plane: a value is kept where it is >= thr
    and becomes 0 below (NaN, never >= thr, becomes 0); widths likewise."""
    best = np.asarray(best, dtype=np.float64)
    keep = best >= thr
    return np.where(keep, best, 0.0), np.where(keep, np.asarray(width), 0)


def cluster_rows(best, width, thr: float, max_gap: int, row0: int = 0):
    """Per-DM clustering of the candidates in time -- an extension after Sec.
    2.4, whose list is unordered and unclustered.  Per row, the candidates
    (best >= thr) in sample order; a candidate joins the previous one's
    cluster when it lies at most max_gap samples after it, else it opens a
    new cluster.  Per cluster: first and last sample, the sample of the
    highest SNR (the earliest among equals), that SNR and width, and the
    number of members.  Returned in (dm, first) order."""
    best = np.asarray(best, dtype=np.float64)
    width = np.asarray(width)
    recs = []
    for r in range(best.shape[0]):
        cur = None
        for i in range(best.shape[1]):
            v = best[r, i]
            if not v >= thr:             # NaN is never a candidate
                continue
            if cur is not None and i - cur["last"] <= max_gap:
                cur["last"] = i
                cur["members"] += 1
                if v > cur["peak_snr"]:
                    cur.update(peak_sample=i, peak_snr=v, peak_width=int(width[r, i]))
            else:
                if cur is not None:
                    recs.append(cur)
                cur = dict(dm=row0 + r, first=i, last=i, peak_sample=i, peak_snr=v,
                           peak_width=int(width[r, i]), members=1)
        if cur is not None:
            recs.append(cur)
    out = np.zeros(len(recs), dtype=[("dm", np.int32), ("first", np.int32), ("last", np.int32),
                                     ("peak_sample", np.int32), ("peak_snr", np.float64),
                                     ("peak_width", np.int32), ("members", np.int32)])
    for k, c in enumerate(recs):
        for f in out.dtype.names:
            out[k][f] = c[f]
    return out


# ------------------------------------------------------------ de-dispersion

def dedisperse(fb, delays, n_out: int) -> np.ndarray:
    """The DM x time plane of a filterbank (Sec. 1: the detector's input):
    out[d, t] = sum over channels c of fb[c, t + delays[d, c]], FP64.
    fb: a Plane (or array) of channel rows; delays: int [n_dm, n_chan]."""
    p = as_plane(fb)
    dl = np.ascontiguousarray(delays, dtype=np.int32)
    if dl.ndim != 2 or dl.shape[1] != p.n_dm:
        raise ValueError("delays must be [n_dm, n_chan]")
    out = np.empty((dl.shape[0], int(n_out)), dtype=np.float64)
    rc = _load().oracle_dedisperse(*p.args(), _ptr(dl), dl.shape[0], int(n_out), _ptr(out))
    if rc:
        raise ValueError("delay outside 0 .. n_samp - n_out")
    return out


# ------------------------------------------------------------ whole path

def msd_and_sigma(plane, widths, sigma_mode=SIGMA_SQRTN, scope=SCOPE_GLOBAL, nmax=0):
    """Steps (a) and the sigma_w of (c): (mean, sd, sd_nmax, sigma_tab)."""
    p = as_plane(plane)
    mean, sd = plane_msd(p, scope)
    widths = np.asarray(widths, dtype=np.int32)
    if sigma_mode != SIGMA_SQRTN:
        nmax = int(nmax or widths[-1])
        sdn = plane_sd_nmax(p, nmax, scope)
    else:
        sdn = np.zeros_like(sd)
    tab = np.stack([sigma_table(sigma_mode, sd[e], widths, sdn[e], nmax)
                    for e in range(sd.size)])
    return mean, sd, sdn, tab


def search(plane, widths, thr, sigma_mode=SIGMA_SQRTN, scope=SCOPE_GLOBAL, nmax=0,
           rows=None, start_w1=True):
    """The four steps in the paper's order; returns (candidates, best, width, msd)."""
    p = as_plane(plane)
    mean, sd, sdn, tab = msd_and_sigma(p, widths, sigma_mode, scope, nmax)
    best, win = boxcar_snr(p, mean, sd, tab, widths, scope, rows, start_w1)
    r0 = rows[0] if rows else 0
    cands = threshold(best, win, thr, row0=r0)
    return cands, best, win, (mean, sd, sdn, tab)


# ----------------------------------------------------------------- streaming

def stream_replay(chunks, widths, thr, scope=SCOPE_GLOBAL, dtype="f32", scale=None,
                  offset=None, detail=False):
    """The search over a stream delivered as `chunks` ([n_dm, L_k] host arrays:
    float32, or the uint16 bits of FP16 / BF16 with one per-row scale/offset
    for the whole stream).  The paper defines one MSD for the dataset
    (Sec. 2.1) and is silent on streams; the reading followed here: a start i
    is searched by the first push whose data hold its full window
    (i + wmax <= samples seen), with the MSD of every sample seen up to and
    including that push (Eq. 4 sigma_w); the starts no push could finish are
    searched at the end (flush) with the row-end truncation of Algorithm 1
    over the whole stream.  Returns one candidate array per push and one for
    the flush, samples counted from the stream's first sample; with detail,
    one dict per call instead: cands, lo, hi (the starts searched), mean, sd,
    best / win over starts [lo, hi) and sub (the plane from sample lo on)."""
    widths = np.asarray(widths, dtype=np.int32)
    wmax = int(widths[-1])
    empty = np.empty(0, dtype=[("dm", np.int32), ("sample", np.int32), ("snr", np.float64),
                                ("width", np.int32)])

    def search_range(full, lo, hi):
        # starts [lo, hi) of the stream so far, `full` = every sample seen
        if full is None or hi <= lo:
            return dict(cands=empty.copy(), lo=lo, hi=lo) if detail else empty.copy()
        mean, sd = plane_msd(Plane(full, dtype=dtype, scale=scale, offset=offset), scope)
        tab = np.stack([sigma_table(SIGMA_SQRTN, sd[e], widths) for e in range(sd.size)])
        sub = Plane(np.ascontiguousarray(full[:, lo:]), dtype=dtype, scale=scale, offset=offset)
        best, win = boxcar_snr(sub, mean, sd, tab, widths, scope)
        best, win = best[:, :hi - lo], win[:, :hi - lo]
        c = threshold(best, win, thr)
        c["sample"] += lo
        if detail:
            return dict(cands=c, lo=lo, hi=hi, mean=mean, sd=sd, best=best, win=win, sub=sub)
        return c

    parts, out = [], []
    emitted = n = 0
    for ch in chunks:
        parts.append(np.asarray(ch))
        n += parts[-1].shape[1]
        full = np.concatenate(parts, axis=1)
        hi = max(emitted, n - (wmax - 1))
        out.append(search_range(full, emitted, hi))
        emitted = hi
    out.append(search_range(np.concatenate(parts, axis=1) if parts else None, emitted, n))
    return out


# ------------------------------------------------------- decimation in time

def decimate(plane, level: int) -> np.ndarray:
    """x_l[j] = x[2^l j] + ... + x[2^l j + 2^l - 1] of the dequantised values,
    in FP64, complete groups only: [n_dm, n_samp >> level]."""
    p = as_plane(plane)
    x = p.values()
    m = 1 << level
    n = p.n_samp >> level
    return x[:, :n * m].reshape(p.n_dm, n, m).sum(axis=2)


def search_decimated(plane, levels, thr):
    """Sec. 3 names decimation in time as the way to widen the boxcars and
    gives no details; the reading here: level l searches its decimated series
    (rounded to FP32, the precision a search takes its samples in) with its
    listed widths (level samples), its own MSD (global scope, Eq. 4) and the
    threshold, as one plain search -- except that a level above 0 evaluates
    only its listed widths: Algorithm 1's width-1 start belongs to the native
    series.  Records are reported in native units (sample j 2^l, width w 2^l)
    with the level.  Returns the records of every level, concatenated in level
    order, and per level (mean, sd)."""
    out, msds = [], []
    for level, widths in levels:
        xl = decimate(plane, level)
        if xl.shape[1] == 0:
            msds.append((np.nan, np.nan))
            continue
        start_w1 = level == 0 or widths[0] == 1
        cands, best, win, (mean, sd, _, _) = search(xl.astype(np.float32), widths, thr,
                                                    start_w1=start_w1)
        c = np.empty(len(cands), dtype=[("dm", np.int32), ("sample", np.int64),
                                        ("snr", np.float64), ("width", np.int64),
                                        ("level", np.int32)])
        c["dm"], c["snr"] = cands["dm"], cands["snr"]
        c["sample"] = cands["sample"].astype(np.int64) << level
        c["width"] = cands["width"].astype(np.int64) << level
        c["level"] = level
        out.append(c)
        msds.append((float(mean[0]), float(sd[0])))
    return (np.concatenate(out) if out else np.empty(0)), msds
