"""Autotuner policy without a GPU: picks the fastest candidate, caches by
shape key in memory and on disk, and does not re-time a cached key."""
import json

from paper_1403_6854_gb300.tune import Autotuner, shape_key


def test_shape_key_buckets():
    assert shape_key("ihs", 5000, 79) == "ihs:n8192:ld79"
    assert shape_key("ihs", 4097, 65) == shape_key("ihs", 8000, 65)
    assert shape_key("xpehh", 414, 8) != shape_key("ihs", 414, 8)


def test_choose_fastest_and_cache(tmp_path):
    cands = [dict(schedule=1, warps_per_cta=w, smem_entries=e) for w in (4, 8) for e in (256, 512)]
    calls = []

    def timer(c):
        calls.append(c)
        return 10.0 + c["warps_per_cta"] - c["smem_entries"] / 1000.0

    path = str(tmp_path / "tune.json")
    t = Autotuner(cache_path=path, candidates=cands, reps=2)
    best = t.choose("k", timer)
    assert best == dict(schedule=1, warps_per_cta=4, smem_entries=512)
    assert len(calls) == 2 * len(cands)
    assert t.choose("k", timer) == best and len(calls) == 2 * len(cands)   # cached
    t2 = Autotuner(cache_path=path, candidates=cands)
    assert t2.choose("k", lambda c: 1 / 0) == best                           # from disk
    data = json.load(open(path))
    assert len(data["k"]["tried"]) == len(cands)
