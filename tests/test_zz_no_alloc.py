"""spd_msd_noalloc through the C ABI: the MSD for callers that cannot give the
library a workspace (for instance a real-time backend that fixes its device
memory at start-up and must not call cudaMalloc later).  Its block partials
live in a static device array inside the library; its results must equal
spd_msd's, call after call, and meet the MSD tolerance against the FP64
oracle's two-pass definition.

This file is collected last, so a run that stops at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
MAX_UNITS = 32768      # SPD_MSD_NOALLOC_MAX_UNITS
UNIT = 65536           # SPD_MSD_UNIT_SAMPLES


@pytest.fixture(scope="module")
def lib():
    import paper_1611_09704_gb300 as spd
    spd.build()
    lib = spd.load()
    from paper_1611_09704_gb300.binding import SpdPlane
    lib.spd_msd_noalloc.argtypes = [ctypes.POINTER(SpdPlane), ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p]
    lib.spd_msd_noalloc.restype = ctypes.c_int32
    return lib


def _noalloc(lib, x, scope, n_samp=None):
    from paper_1611_09704_gb300.binding import MSD_BYTES, Plane
    pl = Plane(x, n_samp=n_samp)
    cp = pl.c()
    n = pl.n_dm if scope == 1 else 1
    out = torch.full((max(n, 1) * MSD_BYTES,), 0xAB, dtype=torch.uint8, device=DEV)
    rc = lib.spd_msd_noalloc(ctypes.byref(cp), scope, ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


def _close(a, b):
    # the MSD tolerance of the parity tests; both calls run the same kernels
    assert np.all(np.abs(a["mean"] - b["mean"]) <= 2e-7 * np.abs(b["mean"]) + 1e-6 * b["sd"])
    assert np.all(np.abs(a["sd"] / b["sd"] - 1.0) <= 2e-6)
    assert np.array_equal(a["n"], b["n"]) and np.array_equal(a["status"], b["status"])


@pytest.mark.parametrize("scope", [0, 1])
def test_noalloc_matches_workspace_msd_twice(lib, scope):
    import oracle
    import paper_1611_09704_gb300 as spd
    import synth
    from tests import _parity as P
    planes = [synth.ska_like(64, 200003, n_pulses=8, device=DEV, seed=31).data,
              synth.plain_tophat(48, 65536, device=DEV, seed=32).data[:, :65000]]
    for x in planes:
        n_samp = x.shape[1]
        ref = spd.msd_to_numpy(spd.msd(x, scope, n_samp=n_samp))
        mean_o, sd_o = oracle.plane_msd(synth.to_host_numpy(x.contiguous()), scope)
        for _ in range(2):          # two calls in a row share the static array
            rc, out = _noalloc(lib, x, scope, n_samp=n_samp)
            assert rc == 0
            torch.cuda.synchronize()
            got = spd.msd_to_numpy(out)
            _close(got, ref)
            P.check_msd(got, mean_o, sd_o)


def test_noalloc_limit_and_empty(lib):
    rows = MAX_UNITS // 8 + 1             # 8 units per row: one unit too many
    x = torch.empty((rows, 8 * UNIT), dtype=torch.float16, device=DEV)
    rc, _ = _noalloc(lib, x, 0)
    assert rc == 3                          # SPD_ERR_NO_MEMORY, nothing launched
    rc, out = _noalloc(lib, torch.empty((0, 10), device=DEV), 0)
    assert rc == 0
    import paper_1611_09704_gb300 as spd
    m = spd.msd_to_numpy(out)
    assert m["n"][0] == 0 and m["status"][0] == 5
