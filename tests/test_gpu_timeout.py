"""Failure detection without a GPU fault: the fused kernel's waits for tile
copies are bounded.  With the test aid that makes every wait run out (more
bytes expected than any copy delivers) and a 20 ms bound, the search reports
SPD_ERR_TIMEOUT in its result word instead of hanging, and the context stays
usable: the next search, with normal waits, gives the normal result."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def spd():
    import paper_1611_09704_gb300 as m
    m.build()
    m.load()
    return m


def test_copy_wait_timeout_is_reported_and_the_context_survives(spd):
    from paper_1611_09704_gb300.binding import SPD_ERR_TIMEOUT, debug_set_copy_wait
    x = synth.plain_tophat(16, 20000, device=DEV, seed=5).data   # rows 16-byte aligned
    widths = list(range(1, 33))
    out, res, _ = spd.search(x, widths, 6.0, 1 << 16)
    c0, s0 = spd.read_result(res)
    want = np.sort(spd.candidates_to_numpy(out, c0), order=["dm", "sample"])
    assert s0 == 0 and c0 > 0
    try:
        debug_set_copy_wait(20_000_000, 16)
        out, res, _ = spd.search(x, widths, 6.0, 1 << 16)
        c1, s1 = spd.read_result(res)
        assert s1 == SPD_ERR_TIMEOUT
    finally:
        debug_set_copy_wait()
    out, res, _ = spd.search(x, widths, 6.0, 1 << 16)
    c2, s2 = spd.read_result(res)
    assert (c2, s2) == (c0, 0)
    assert np.array_equal(np.sort(spd.candidates_to_numpy(out, c2), order=["dm", "sample"]), want)
