"""Seeded input generator: determinism, layout and the planted structure."""
import numpy as np
import pytest

import synth


def test_deterministic_and_layout():
    a = synth.generate(synth.spec("plain"))
    b = synth.generate(synth.spec("plain"))
    assert np.array_equal(a.rows, b.rows) and np.array_equal(a.pos, b.pos)
    assert np.array_equal(a.gmap, b.gmap)
    assert a.rows.shape == (2000, 2)
    assert np.all(np.diff(a.pos) > 0) and a.pos[0] >= 1 and a.pos[-1] <= 2_000_000
    assert np.all(np.diff(a.gmap) >= 0)
    # pad bits above n = 100 in the last word are zero
    assert np.all(a.rows[:, 1] >> np.uint64(36) == 0)
    c = synth.generate(synth.spec("plain", seed=1))
    assert not np.array_equal(a.rows, c.rows)


def test_chr22_gaps_and_sweep():
    s = synth.spec("chr22")
    d = synth.generate(s)
    steps = np.diff(d.pos)
    for idx, bp in s.gaps:
        assert steps[idx - 1] == bp
    # the planted sweep: carriers (allele 1 at the core) are identical over +-200 kb
    hap = synth.unpack(d.rows, 204)
    core = int(np.argmin(np.abs(d.pos - 17_500_000)))
    car = np.flatnonzero(hap[core])
    assert len(car) == round(0.6 * 204)
    win = np.flatnonzero(np.abs(d.pos - d.pos[core]) <= 200_000)
    sub = hap[np.ix_(win, car)]
    assert np.all(sub == sub[:, :1])


def test_xpehh_layout_word_aligned():
    d = synth.generate(synth.spec("xpehh"))
    assert d.rows.shape == (22147, 8)
    assert np.all(d.rows[:, 3] >> np.uint64(12) == 0)   # 204 = 3*64 + 12
    assert np.all(d.rows[:, 7] >> np.uint64(18) == 0)   # 210 = 3*64 + 18
    a = synth.generate(synth.spec("chr22"))
    assert np.array_equal(a.rows, d.rows[:, :4])         # pop A is the chr22 population


def test_pack_roundtrip():
    hap, pos, gmap = synth.tiny_random(131, 17, 3)
    rows = synth.pack(hap, ld=4)
    assert rows.shape == (17, 4) and np.all(rows[:, 3] == 0)
    assert np.array_equal(synth.unpack(rows, 131), hap)


def test_served_requests_in_range():
    for i in range(20):
        s = synth.served_request(i)
        assert 10_000 <= s.m <= 500_000
        for p in s.pops:
            assert 100 <= p.n <= 5000
        assert s.mode in ("ihs", "xpehh")


def test_complexity_spec_scales_noise_with_density():
    a, b = synth.complexity_spec(1000, 2500), synth.complexity_spec(1000, 10000)
    assert (a.m, b.m) == (50_000, 200_000) and a.len_bp == b.len_bp == 20_000_000
    # allele noise per Mb is the same at both densities
    assert a.pops[0].flip_prob * 2500 == pytest.approx(b.pops[0].flip_prob * 10000)
    d = synth.generate(synth.complexity_spec(64, 100, len_bp=1_000_000))
    assert d.rows.shape == (100, 1) and np.all(np.diff(d.pos) > 0)


def test_loglog_slope():
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench_mod", os.path.join(os.path.dirname(os.path.dirname(__file__)), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    x = [250, 500, 1000, 2000]
    assert bench.loglog_slope(x, [7.0 * v ** 2 for v in x]) == pytest.approx(2.0)
    assert bench.loglog_slope(x, [3.0 for _ in x]) == pytest.approx(0.0, abs=1e-12)
