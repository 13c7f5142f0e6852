"""Sorted-sweep schedule vs the CPU oracle, through the C ABI.

The sweep keeps each chunk's haplotypes sorted by their sequence read
outward from the core and applies, at walk step i, only the neighbour pairs
that part there; walks that outrun a chunk's sorted history finish in a
second per-step pass.  Every launch shape below must reproduce the oracle:
integers bit for bit, iHH within 1e-12 relative, ln ratios within 1e-9.
Small warm-ups force many walks through the hand-off; one-core stages
exercise the state carried between stage launches."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import assert_ihs_equal, assert_xpehh_equal, to_np

pytestmark = pytest.mark.gpu

SHAPES = [dict(), dict(sweep_warmup=16, sweep_stage_cores=7), dict(sweep_warmup=40, sweep_stage_cores=1),
          dict(sweep_warmup=300, sweep_stage_cores=4096), dict(sweep_threads=512),
          dict(sweep_threads=256, sweep_warmup=64, sweep_stage_cores=33),
          dict(sweep_split_tile=16), dict(sweep_split_tile=16, sweep_warmup=16, sweep_stage_cores=5),
          dict(sweep_split_tile=32), dict(sweep_threads=32), dict(sweep_threads=128),
          dict(sweep_threads=64, sweep_warmup=40, sweep_stage_cores=9), dict(sweep_threads=256),
          # chunk counts set by the sorting CTAs per SM (one, and four of 256 threads)
          dict(sweep_threads=256, sweep_ctas_per_sm=1, sweep_warmup=64),
          dict(sweep_threads=256, sweep_ctas_per_sm=4, sweep_warmup=64, sweep_stage_cores=50)]


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg
    return sg


def sweep(sg, **kw):
    return sg.make_launch(sg.SCHED_SWEEP, **kw)


def run_ihs(sg, rows, n, pos, gmap, **kw):
    hap, p, g = sg.to_device(rows, pos, gmap)
    out = sg.selscan_ihs(hap, n, p, g, **kw)
    sg.check(out)
    return to_np(out)


def run_xpehh(sg, rows, nA, nB, pos, gmap, **kw):
    hap, p, g = sg.to_device(rows, pos, gmap)
    out = sg.selscan_xpehh(hap, nA, nB, p, g, **kw)
    sg.check(out)
    return to_np(out)


@pytest.fixture(scope="module")
def chr22():
    d = synth.generate(synth.spec("chr22"))
    return d, oracle.ihs(d.rows, 204, d.pos, d.gmap)


@pytest.fixture(scope="module")
def xp():
    d = synth.generate(synth.spec("xpehh"))
    return d, oracle.xpehh(d.rows, 204, 210, d.pos, d.gmap)


@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_plain_config(sg, shape):
    d = synth.generate(synth.spec("plain"))
    ref = oracle.ihs(d.rows, 100, d.pos, d.gmap)
    assert_ihs_equal(run_ihs(sg, d.rows, 100, d.pos, d.gmap, launch=sweep(sg, **SHAPES[shape])), ref)


@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_chr22_all_cores(sg, chr22, shape):
    d, ref = chr22
    assert_ihs_equal(run_ihs(sg, d.rows, 204, d.pos, d.gmap, launch=sweep(sg, **SHAPES[shape])), ref)


@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_xpehh_all_cores(sg, xp, shape):
    d, ref = xp
    got = run_xpehh(sg, d.rows, 204, 210, d.pos, d.gmap, launch=sweep(sg, **SHAPES[shape]))
    assert_xpehh_equal(got, ref)


@pytest.mark.parametrize("n", [2, 3, 31, 32, 33, 63, 64, 65, 200])
@pytest.mark.parametrize("m", [1, 2, 7, 40, 300])
def test_small_shapes(sg, n, m):
    hap, pos, gmap = synth.tiny_mosaic(n, m, 3000 + 7 * n + m, founders=3, switch=0.1, flip=0.03)
    rows = synth.pack(hap)
    for p in (oracle.params(maf=(0, 1)), oracle.params()):
        ref = oracle.ihs(rows, n, pos, gmap, p=p)
        for kw in (dict(), dict(sweep_warmup=16, sweep_stage_cores=3),
                   dict(sweep_split_tile=16, sweep_warmup=16)):
            got = run_ihs(sg, rows, n, pos, gmap, launch=sweep(sg, **kw),
                          params=sg.selscan_default_params(maf=(p.maf_num, p.maf_den)))
            assert_ihs_equal(got, ref)


def test_gap_rules_and_parameters(sg):
    n, m = 40, 60
    hap, pos, gmap = synth.tiny_mosaic(n, m, 5, founders=2, switch=0.04, flip=0.01,
                                       dyadic_map=False)
    steps = np.diff(pos)
    steps[[5, 12, 20, 33, 41, 50]] = [20_000, 20_001, 200_000, 200_001, 45_000, 1_000_000]
    pos = np.concatenate([[pos[0]], pos[0] + np.cumsum(steps)]).astype(np.int64)
    rows = synth.pack(hap)
    rx = np.concatenate([synth.pack(hap[:, :17]), synth.pack(hap[:, 17:])], 1)
    cases = [dict(), dict(include_crossing_term=1), dict(ehh_cut=(1, 4)), dict(ehh_cut=(3, 100)),
             dict(gap_scale_bp=5000, max_gap_bp=60_000), dict(maf=(1, 5))]
    for c in cases:
        op = oracle.params(**c)
        for kw in (dict(), dict(sweep_warmup=16, sweep_stage_cores=2)):
            L = sweep(sg, **kw)
            got = run_ihs(sg, rows, n, pos, gmap, params=sg.selscan_default_params(**c), launch=L)
            assert_ihs_equal(got, oracle.ihs(rows, n, pos, gmap, p=op))
            gotx = run_xpehh(sg, rx, 17, n - 17, pos, gmap, params=sg.selscan_default_params(**c),
                             launch=L)
            assert_xpehh_equal(gotx, oracle.xpehh(rx, 17, n - 17, pos, gmap, p=op))


def test_xpehh_small_and_maf_flag(sg):
    # pooled sizes 32, 64 and 128 too: the population flags' last word then holds
    # only position n
    for nA, nB in ((2, 2), (5, 64), (64, 65), (100, 31), (20, 12), (40, 24), (64, 64)):
        hap, pos, gmap = synth.tiny_mosaic(nA + nB, 35, nA * 31 + nB, founders=3, switch=0.1,
                                           flip=0.03)
        rows = np.concatenate([synth.pack(hap[:, :nA]), synth.pack(hap[:, nA:])], 1)
        for flag in (0, 1):
            ref = oracle.xpehh(rows, nA, nB, pos, gmap, p=oracle.params(xpehh_maf_filter=flag))
            for kw in (dict(), dict(sweep_warmup=16, sweep_stage_cores=5)):
                got = run_xpehh(sg, rows, nA, nB, pos, gmap, launch=sweep(sg, **kw),
                                params=sg.selscan_default_params(xpehh_maf_filter=flag))
                assert_xpehh_equal(got, ref)


def test_identical_haplotypes_and_long_walks(sg):
    """All carriers identical over long stretches (a sweep in miniature): the
    walks outrun small warm-ups and finish in the second pass."""
    n, m = 150, 500
    hap, pos, gmap = synth.tiny_mosaic(n, m, 99, founders=2, switch=0.002, flip=0.0)
    rows = synth.pack(hap)
    ref = oracle.ihs(rows, n, pos, gmap)
    for kw in (dict(), dict(sweep_warmup=16, sweep_stage_cores=9), dict(sweep_warmup=100)):
        assert_ihs_equal(run_ihs(sg, rows, n, pos, gmap, launch=sweep(sg, **kw)), ref)


def test_first_window_shorter_than_64_steps(sg):
    """3,000 haplotypes, half i.i.d. and half near-copies of one sequence: the
    i.i.d. half parts more than 1,024 neighbour pairs within the first dozen
    steps, so the slot's first window stops short of 64 steps (each step at
    most doubles the runs, so it still covers 9 or more), while the copies keep
    one class's walks going for about a hundred steps through windows the
    walker builds itself from the first window's end on."""
    n, m = 3000, 300
    rng = np.random.Generator(np.random.PCG64(77))
    hap = np.empty((m, n), dtype=np.uint8)
    hap[:, :1500] = rng.random((m, 1500)) < 0.5
    base = (rng.random(m) < 0.5).astype(np.uint8)
    hap[:, 1500:] = base[:, None] ^ (rng.random((m, 1500)) < 0.01)
    _, pos, gmap = synth.tiny_mosaic(4, m, 78)
    rows = synth.pack(hap)
    cores = np.array([60, 150, 151, 240])
    ref = oracle.ihs(rows, n, pos, gmap, cores=cores)
    assert ref["stop"].max() > 64                         # walks outlive a 64-step window
    for kw in (dict(), dict(sweep_warmup=40, sweep_stage_cores=7)):
        assert_ihs_equal(run_ihs(sg, rows, n, pos, gmap, launch=sweep(sg, **kw)), ref, idx=cores)


@pytest.mark.parametrize("n,threads", [(6000, 256), (6000, 512), (9000, 0), (9000, 256), (13000, 0),
                                       (500, 0), (900, 32), (2000, 64), (3000, 64), (1500, 0),
                                       (3000, 256), (4000, 256), (4500, 256), (7000, 256), (8000, 256)])
def test_elements_per_thread(sg, n, threads):
    """Samples near the register-cached limit of each CTA width, ones that
    re-read their elements from shared memory (more than 24 per thread),
    requests above 32 elements per thread (taken by the next wider CTA), and
    each exact element count of the 256-thread sort (4, 8, ..., 24 a thread:
    n = 3000, 4000 and 4500 give 12, 16 and 20 with padding), and 28 / 32 a
    thread on 256 threads (n = 7000, 8000: elements re-read from shared memory)."""
    m = 90
    hap, pos, gmap = synth.tiny_mosaic(n, m, n + threads, founders=5, switch=0.05, flip=0.003)
    rows = synth.pack(hap)
    cores = np.array([0, 3, 44, 45, 88, 89])
    ref = oracle.ihs(rows, n, pos, gmap, cores=cores)
    got = run_ihs(sg, rows, n, pos, gmap,
                  launch=sweep(sg, sweep_warmup=24, sweep_stage_cores=10, sweep_threads=threads))
    assert_ihs_equal(got, ref, idx=cores)


def test_xpehh_widest_rows(sg):
    """n_A + n_B = 16383 over 129 + 128 words: rows of 514 32-bit words."""
    nA, nB, m = 8193, 8190, 60
    hap, pos, gmap = synth.tiny_mosaic(nA + nB, m, 4242, founders=5, switch=0.05, flip=0.003)
    rows = np.concatenate([synth.pack(hap[:, :nA]), synth.pack(hap[:, nA:])], 1)
    cores = np.array([0, 29, 30, 59])
    ref = oracle.xpehh(rows, nA, nB, pos, gmap, cores=cores)
    got = run_xpehh(sg, rows, nA, nB, pos, gmap, launch=sweep(sg, sweep_warmup=20, sweep_stage_cores=8))
    assert_xpehh_equal(got, ref, idx=cores)


@pytest.mark.parametrize("n", [16383, 16384])
def test_haplotype_limit(sg, n):
    """16383 haplotypes is the largest sample sorted on chip; 16384 falls back
    to the in-order schedule.  Both agree with the oracle on sampled cores."""
    m = 120
    hap, pos, gmap = synth.tiny_mosaic(n, m, n, founders=6, switch=0.05, flip=0.002)
    rows = synth.pack(hap)
    cores = np.array([0, 1, 17, 59, 60, 101, 119])
    ref = oracle.ihs(rows, n, pos, gmap, cores=cores)
    got = run_ihs(sg, rows, n, pos, gmap, launch=sweep(sg, sweep_warmup=32, sweep_stage_cores=16))
    assert_ihs_equal(got, ref, idx=cores)


def longest_walk_cores(got, k):
    """The k cores with the largest sum of stop indices on the GPU."""
    tot = got["stop"].astype(np.int64).sum(1)
    return np.argsort(-tot, kind="stable")[:k]


def sweep_region_cores(d, m, half):
    c = synth.sweep_cores(d)
    near = (c[:, None] + np.arange(-half, half + 1)[None, :]).ravel()
    return near[(near >= 0) & (near < m)]


def test_xpehh_at_scale_sampled_cores(sg):
    """1,000 + 1,000 haplotypes x 200,000 SNPs with four planted sweeps in A:
    the default launch takes the sorted sweep; random cores, every sweep
    centre with its +-16 neighbours and the 64 longest GPU walks match the
    oracle."""
    d = synth.generate(synth.spec("xpehh200k"))
    got = run_xpehh(sg, d.rows, 1000, 1000, d.pos, d.gmap)
    rng = np.random.default_rng(1)
    cores = np.unique(np.concatenate([rng.choice(d.spec.m, 24, replace=False),
                                      sweep_region_cores(d, d.spec.m, 16),
                                      longest_walk_cores(got, 64)]))
    ref = oracle.xpehh(d.rows, 1000, 1000, d.pos, d.gmap, cores=cores)
    assert_xpehh_equal(got, ref, idx=cores)
    assert np.array_equal(np.isfinite(got["lnratio"]), got["status"] == 0)


def test_xpehh_1m_sampled_cores(sg):
    """The bench's XPEHH workload at full size (2,500 + 2,500 haplotypes x
    1,000,000 SNPs, 20 planted sweeps in A) in the launch the bench times (the
    default: the sorted sweep): random cores, every sweep centre with its +-8
    neighbours and the 128 longest GPU walks match the oracle, and every
    locus has a finite ratio exactly when it is OK."""
    d = synth.generate(synth.spec("xpehh1m"))
    got = run_xpehh(sg, d.rows, 2500, 2500, d.pos, d.gmap)
    rng = np.random.default_rng(2)
    cores = np.unique(np.concatenate([rng.choice(d.spec.m, 24, replace=False),
                                      sweep_region_cores(d, d.spec.m, 8),
                                      longest_walk_cores(got, 128)]))
    ref = oracle.xpehh(d.rows, 2500, 2500, d.pos, d.gmap, cores=cores)
    assert_xpehh_equal(got, ref, idx=cores)
    assert np.array_equal(np.isfinite(got["lnratio"]), got["status"] == 0)


def test_split_tile_16_against_32(sg, chr22, xp):
    """16-lane split walks keep 16 trapezoid partial sums instead of 32: every
    integer result (status, n1, stops, digests) is the 32-lane result bit for
    bit, the iHH values agree to rounding."""
    from parity_util import to_np
    for (d, _), mode in ((chr22, "ihs"), (xp, "xpehh")):
        hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
        outs = []
        for tile in (32, 16):
            L = sweep(sg, sweep_split_tile=tile, sweep_warmup=64, sweep_stage_cores=500)
            if mode == "ihs":
                o = sg.selscan_ihs(hap, 204, pos, gmap, launch=L)
            else:
                o = sg.selscan_xpehh(hap, 204, 210, pos, gmap, launch=L)
            sg.check(o)
            outs.append(to_np(o))
        a, b = outs
        for k in a:
            if a[k].dtype.kind == "f":
                ok = ~np.isnan(a[k])
                assert np.array_equal(ok, ~np.isnan(b[k])), k
                np.testing.assert_allclose(b[k][ok], a[k][ok], rtol=1e-12, atol=1e-12, err_msg=k)
            else:
                assert np.array_equal(a[k], b[k]), k
