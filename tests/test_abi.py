"""The C ABI library (CPU-only checks): it builds for sm_103a, loads, exports
every function include/spd.h declares, and rejects bad arguments on the host
before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_1611_09704_gb300 as spd
    spd.build()
    return spd.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "spd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spd_[a-z_]+)\s*\(", src)))


def test_header_declares_the_calls():
    names = _declared()
    for must in ("spd_msd", "spd_boxcar_snr", "spd_threshold_candidates", "spd_search",
                 "spd_detect"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1611_09704_gb300.binding import EXPORTS
    names = _declared()
    assert sorted(EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_sizes_match_header():
    from paper_1611_09704_gb300 import binding as b
    assert ctypes.sizeof(b.SpdMsdStats) == 40
    assert ctypes.sizeof(b.SpdCandidate) == 16
    assert ctypes.sizeof(b.SpdResult) == 16
    assert ctypes.sizeof(b.SpdPlane) == 56
    assert b.MSD_DTYPE.itemsize == 40 and b.CAND_DTYPE.itemsize == 16
    assert b.CLUSTER_DTYPE.itemsize == 32


def test_ctypes_layouts_match_the_c_compiler(tmp_path):
    """gcc compiles include/spd.h; every struct's size and field offsets equal
    the ctypes mirror's."""
    import subprocess
    from paper_1611_09704_gb300 import binding as b
    structs = {"spd_plane": b.SpdPlane, "spd_msd_stats": b.SpdMsdStats,
               "spd_candidate": b.SpdCandidate, "spd_result": b.SpdResult,
               "spd_search_params": b.SpdSearchParams, "spd_range": b.SpdRange,
               "spd_tuning": b.SpdTuning, "spd_stream_info": b.SpdStreamInfo,
               "spd_msd_part": b.SpdMsdPart, "spd_level": b.SpdLevel}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "spd.h"',
             "int main(void) {"]
    for cname, ct in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in ct._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    # the numpy record dtypes the binding decodes device arrays with
    dtypes = {"spd_candidate": b.CAND_DTYPE, "spd_cluster": b.CLUSTER_DTYPE,
              "spd_msd_stats": b.MSD_DTYPE}
    for cname, dt in dtypes.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in dt.names:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                             text=True).stdout.splitlines():
        cname, key, val = ln.split()
        got[(cname, key)] = int(val)
    for cname, ct in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(ct), cname
        for f, _ in ct._fields_:
            assert got[(cname, f)] == getattr(ct, f).offset, (cname, f)
    for cname, dt in dtypes.items():
        assert got[(cname, "size")] == dt.itemsize, cname
        for f in dt.names:
            assert got[(cname, f)] == dt.fields[f][1], (cname, f)


def test_stream_host_validation(lib):
    from paper_1611_09704_gb300.binding import SPD_ERR_INVALID_ARG, SpdStreamInfo
    prm, keep = _params(np.arange(1, 129))
    sb = lib.spd_stream_state_bytes(2048, 1, ctypes.byref(prm))
    # running MSD + halo of 127 samples (rounded to 128) + scale + offset
    assert sb >= 2048 * 128 * 2 + 2 * 2048 * 4
    assert lib.spd_stream_workspace_bytes(2048, 65536, 1, ctypes.byref(prm)) > 2048 * 65536 * 2
    assert lib.spd_stream_state_bytes(0, 1, ctypes.byref(prm)) == 0
    assert lib.spd_stream_state_bytes(16, 9, ctypes.byref(prm)) == 0
    lin, k2 = _params(np.arange(1, 9), mode=1)
    assert lib.spd_stream_state_bytes(16, 0, ctypes.byref(lin)) == 0
    info = SpdStreamInfo()
    # misaligned state / no state: rejected on the host
    assert lib.spd_stream_reset(ctypes.byref(info), ctypes.c_void_p(4097), 16, 0,
                                ctypes.byref(prm), None) == SPD_ERR_INVALID_ARG
    assert lib.spd_stream_reset(ctypes.byref(info), None, 16, 0, ctypes.byref(prm),
                                None) == SPD_ERR_INVALID_ARG


def test_decimated_host_validation(lib):
    from paper_1611_09704_gb300.binding import SpdLevel
    p = _plane(4, 1000)

    def levels(*lv):
        arr = (SpdLevel * len(lv))()
        keep = []
        for i, (l, w) in enumerate(lv):
            a = np.ascontiguousarray(w, dtype=np.int32)
            keep.append(a)
            arr[i] = SpdLevel(l, a.size, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return arr, keep

    ok, k1 = levels((0, [1, 2, 4]), (1, [3, 4]), (3, [2, 4]))
    assert lib.spd_search_decimated_workspace_bytes(ctypes.byref(p), ok, 3) > 4 * 500 * 4
    # native widths must ascend across levels (level 1 width 2 = native 4 <= 4)
    bad, k2 = levels((0, [1, 2, 4]), (1, [2, 4]))
    assert lib.spd_search_decimated_workspace_bytes(ctypes.byref(p), bad, 2) == 0
    # levels must ascend and stay within range
    bad, k3 = levels((1, [2]), (1, [4]))
    assert lib.spd_search_decimated_workspace_bytes(ctypes.byref(p), bad, 2) == 0
    bad, k4 = levels((13, [2]),)
    assert lib.spd_search_decimated_workspace_bytes(ctypes.byref(p), bad, 1) == 0


def test_debug_copy_wait_validation(lib):
    from paper_1611_09704_gb300.binding import SPD_ERR_INVALID_ARG
    assert lib.spd_debug_set_copy_wait(100, 0) == SPD_ERR_INVALID_ARG          # under 1 ms
    assert lib.spd_debug_set_copy_wait(20_000_000, 8) == SPD_ERR_INVALID_ARG   # not 16-byte
    assert lib.spd_debug_set_copy_wait(20_000_000, 8192) == SPD_ERR_INVALID_ARG
    assert lib.spd_debug_set_copy_wait(2_000_000_000, 0) == 0


def _plane(n_dm=4, n_samp=100, stride=None, data=4096, dtype=0):
    from paper_1611_09704_gb300.binding import SpdPlane
    return SpdPlane(data, dtype, 0, n_dm, n_samp, stride or n_samp, None, None)


def _params(widths, thr=6.0, mode=0, scope=0, nmax=0):
    from paper_1611_09704_gb300.binding import SpdSearchParams
    w = np.ascontiguousarray(widths, dtype=np.int32)
    return SpdSearchParams(w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), w.size,
                           float(thr), mode, scope, nmax, 0), w


def test_host_validation(lib):
    from paper_1611_09704_gb300.binding import SPD_ERR_INVALID_ARG
    p = _plane()
    ws = lib.spd_msd_workspace_bytes(ctypes.byref(p), 0, 0)
    assert ws > 0
    assert lib.spd_msd_workspace_bytes(ctypes.byref(_plane(stride=50)), 0, 0) == 0
    assert lib.spd_msd_workspace_bytes(ctypes.byref(p), 7, 0) == 0
    prm, keep = _params(np.arange(1, 33))
    assert lib.spd_search_workspace_bytes(ctypes.byref(p), ctypes.byref(prm)) > ws
    # width lists: not ascending, zero, too wide -> no workspace size
    for bad in ([3, 2], [0, 1], [1, 5000], [4, 4]):
        q, k = _params(bad)
        assert lib.spd_search_workspace_bytes(ctypes.byref(p), ctypes.byref(q)) == 0
    q, k = _params([1, 2], thr=float("nan"))
    assert lib.spd_search_workspace_bytes(ctypes.byref(p), ctypes.byref(q)) == 0
    # calls fail before any launch
    assert lib.spd_search(ctypes.byref(p), ctypes.byref(prm), None, 0, None, None, None, 0,
                          None) == SPD_ERR_INVALID_ARG
    assert lib.spd_search(None, ctypes.byref(prm), None, 0, None, None, None, 0,
                          None) == SPD_ERR_INVALID_ARG
    assert lib.spd_threshold_candidates(None, None, 4, 10, 10, 6.0, None, 5, None,
                                        None) == SPD_ERR_INVALID_ARG
    assert lib.spd_boxcar_sums(ctypes.byref(p), 0, None, 100, None) == SPD_ERR_INVALID_ARG
    # misaligned data pointer for f32
    bad = _plane(data=4098)
    assert lib.spd_msd_workspace_bytes(ctypes.byref(bad), 0, 0) == 0


def test_workspace_grows_with_scope_and_widths(lib):
    p = _plane(n_dm=64, n_samp=65536)
    a, k1 = _params(np.arange(1, 33))
    b, k2 = _params(np.arange(1, 33), scope=1)
    c, k3 = _params(np.arange(1, 513))
    wa = lib.spd_detect_workspace_bytes(ctypes.byref(p), ctypes.byref(a))
    wb = lib.spd_detect_workspace_bytes(ctypes.byref(p), ctypes.byref(b))
    wc = lib.spd_detect_workspace_bytes(ctypes.byref(p), ctypes.byref(c))
    assert 0 < wa < wb and wa < wc


def test_status_strings(lib):
    for s in range(8):
        assert lib.spd_status_string(s)
    assert lib.spd_version() >= 100


def test_missing_library_fails_loudly():
    """Without the built CUDA library the product raises: no CPU fallback
    computes anything in its place."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import torch, paper_1611_09704_gb300 as spd\n"
        "from paper_1611_09704_gb300 import builder\n"
        "builder.LIB = '/nonexistent/libspd.so'\n"
        "x = torch.zeros((2, 64))\n"
        "for call in (lambda: spd.msd(x), lambda: spd.search(x, [1, 2], 6.0, 16)):\n"
        "    try:\n"
        "        call()\n"
        "    except RuntimeError as e:\n"
        "        assert 'not built' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('returned without the library')\n"
        "print('raised')\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root,
                       timeout=300)
    assert r.returncode == 0 and "raised" in r.stdout, r.stderr[-2000:]
