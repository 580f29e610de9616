"""Autotuner bookkeeping without a GPU: keys, choice and the cache file."""
import json
from types import SimpleNamespace

import torch

from paper_1611_09704_gb300 import autotune


def _spec(n_dm, n, widths):
    return SimpleNamespace(x=torch.empty((n_dm, n)), widths=widths, threshold=6.0,
                           sigma_mode=0, scope=0, nmax=0)


def test_key_depends_on_shape_and_widths():
    a = autotune.batch_key([_spec(4, 100, [1, 2])], "dev")
    assert a == autotune.batch_key([_spec(4, 100, [1, 2])], "dev")
    assert a != autotune.batch_key([_spec(4, 101, [1, 2])], "dev")
    assert a != autotune.batch_key([_spec(4, 100, [1, 3])], "dev")
    assert a != autotune.batch_key([_spec(4, 100, [1, 2])], "other")


def test_choose_fastest_first_on_ties():
    t = {json.dumps({"a": 1}): 2.0, json.dumps({"a": 2}): 1.0, json.dumps({"a": 3}): 1.0}
    assert autotune.choose(t) == {"a": 2}


def test_cache_round_trip(tmp_path, monkeypatch):
    path = str(tmp_path / "t.json")
    calls = []

    def timer(specs, cap, cand, reps):
        calls.append(cand)
        return 1.0 + cand["group_scale"] + 0.5 * cand["ctas_per_sm"] + (cand["tile_threads"] == 128)

    monkeypatch.setattr(torch.cuda, "get_device_name", lambda d=None: "fake")
    specs = [_spec(2, 50, [1, 2, 3])]
    r = autotune.autotune(specs, 10, cache_path=path, timer=timer)
    assert r["tuning"] == {"ctas_per_sm": 0, "group_scale": 1, "tile_threads": 256}
    assert not r["cached"]
    assert len(calls) == len(autotune.CANDIDATES)
    r2 = autotune.autotune(specs, 10, cache_path=path, timer=timer)
    assert r2["cached"] and len(calls) == len(autotune.CANDIDATES)
