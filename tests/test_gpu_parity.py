"""GPU (sm_103a) vs CPU oracle, through the C ABI.

Integers (status, n_1, stop indices, S digests) must match bit for bit;
iHH within 1e-12 relative; ln ratios within 1e-9 absolute.  Schedules and
on-chip capacities must not change any output bit.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import assert_bitwise_equal, assert_ihs_equal, assert_xpehh_equal, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg
    return sg


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
def plain():
    return synth.generate(synth.spec("plain"))


@pytest.fixture(scope="module")
def chr22():
    return synth.generate(synth.spec("chr22"))


@pytest.fixture(scope="module")
def xp():
    return synth.generate(synth.spec("xpehh"))


def test_plain_all_cores(sg, plain):
    got = run_ihs(sg, plain.rows, 100, plain.pos, plain.gmap)
    ref = oracle.ihs(plain.rows, 100, plain.pos, plain.gmap)
    assert_ihs_equal(got, ref)


@pytest.mark.parametrize("schedule", ["default", "sweep"])
def test_chr22_all_cores(sg, chr22, schedule):
    """The default launch and the sorted sweep (the per-step walk is covered
    against the oracle by the default)."""
    L = None if schedule == "default" else sg.make_launch(sg.SCHED_SWEEP)
    got = run_ihs(sg, chr22.rows, 204, chr22.pos, chr22.gmap, launch=L)
    ref = oracle.ihs(chr22.rows, 204, chr22.pos, chr22.gmap)
    assert_ihs_equal(got, ref)
    # the planted gaps made both abort kinds appear
    assert (ref["status"] == oracle.ABORT_GAP).any() and (ref["status"] == oracle.ABORT_EDGE).any()


@pytest.mark.parametrize("schedule", ["default", "sweep"])
def test_xpehh_all_cores(sg, xp, schedule):
    L = None if schedule == "default" else sg.make_launch(sg.SCHED_SWEEP)
    got = run_xpehh(sg, xp.rows, 204, 210, xp.pos, xp.gmap, launch=L)
    ref = oracle.xpehh(xp.rows, 204, 210, xp.pos, xp.gmap)
    assert_xpehh_equal(got, ref)


def test_schedules_and_capacities_bitwise_equal(sg, chr22):
    base = run_ihs(sg, chr22.rows, 204, chr22.pos, chr22.gmap,
                   launch=sg.make_launch(sg.SCHED_IN_ORDER))
    variants = [sg.make_launch(sg.SCHED_LONGEST_FIRST, probe_steps=4),
                sg.make_launch(sg.SCHED_LONGEST_FIRST, warps_per_cta=2, ctas_per_sm=3),
                sg.make_launch(sg.SCHED_PLAIN),
                sg.make_launch(sg.SCHED_IN_ORDER, smem_entries=8),       # spills to global
                sg.make_launch(sg.SCHED_IN_ORDER, smem_entries=2048, warps_per_cta=4),
                sg.make_launch(sg.SCHED_IN_ORDER, window_rows=2, cores_per_fetch=7),
                sg.make_launch(sg.SCHED_IN_ORDER, window_rows=64, cores_per_fetch=64),
                sg.make_launch(sg.SCHED_IN_ORDER, min_ctas_per_sm=3, smem_entries=256)]
    for L in variants:
        assert_bitwise_equal(base, run_ihs(sg, chr22.rows, 204, chr22.pos, chr22.gmap, launch=L))


def test_xpehh_schedules_bitwise_equal(sg, xp):
    base = run_xpehh(sg, xp.rows, 204, 210, xp.pos, xp.gmap)
    for L in (sg.make_launch(sg.SCHED_PLAIN), sg.make_launch(sg.SCHED_IN_ORDER, smem_entries=8),
              sg.make_launch(sg.SCHED_LONGEST_FIRST, probe_steps=3)):
        assert_bitwise_equal(base, run_xpehh(sg, xp.rows, 204, 210, xp.pos, xp.gmap, launch=L))


@pytest.mark.parametrize("n", [2, 3, 63, 64, 65, 127, 129, 200])
@pytest.mark.parametrize("m", [1, 2, 7, 40])
def test_small_shapes(sg, n, m):
    hap, pos, gmap = synth.tiny_mosaic(n, m, 1000 + 7 * n + m, founders=3, switch=0.1, flip=0.03)
    rows = synth.pack(hap)
    for p in (oracle.params(maf=(0, 1)), oracle.params()):
        ref = oracle.ihs(rows, n, pos, gmap, p=p)
        got = run_ihs(sg, rows, n, pos, gmap, params=sg.selscan_default_params(
            maf=(p.maf_num, p.maf_den)))
        assert_ihs_equal(got, ref)


def test_pad_bits_and_row_stride_ignored(sg):
    n, m = 70, 30
    hap, pos, gmap = synth.tiny_mosaic(n, m, 77, founders=3, switch=0.1, flip=0.02)
    rows = synth.pack(hap, ld=5)
    ref = oracle.ihs(rows, n, pos, gmap)
    dirty = rows.copy()
    dirty[:, 1] |= np.uint64(0xFFFFFFFFFFFFFFFF) << np.uint64(6)   # pad bits of word 1
    dirty[:, 2:] = np.uint64(0xDEADBEEFDEADBEEF)                   # words beyond W
    assert_ihs_equal(run_ihs(sg, dirty, n, pos, gmap), ref)


def test_gap_rules_and_parameters(sg):
    n, m = 40, 60
    hap, pos, gmap = synth.tiny_mosaic(n, m, 5, founders=2, switch=0.04, flip=0.01,
                                       dyadic_map=False)
    steps = np.diff(pos)
    steps[[5, 12, 20, 33, 41, 50]] = [20_000, 20_001, 200_000, 200_001, 45_000, 1_000_000]
    pos = np.concatenate([[pos[0]], pos[0] + np.cumsum(steps)]).astype(np.int64)
    rows = synth.pack(hap)
    cases = [dict(), dict(include_crossing_term=1), dict(ehh_cut=(1, 4)), dict(ehh_cut=(3, 100)),
             dict(gap_scale_bp=5000, max_gap_bp=60_000), dict(maf=(1, 5))]
    for c in cases:
        op = oracle.params(**c)
        ref = oracle.ihs(rows, n, pos, gmap, p=op)
        got = run_ihs(sg, rows, n, pos, gmap, params=sg.selscan_default_params(**c))
        assert_ihs_equal(got, ref)
        refx = oracle.xpehh(np.concatenate([synth.pack(hap[:, :17]), synth.pack(hap[:, 17:])], 1),
                            17, n - 17, pos, gmap, p=op)
        gotx = run_xpehh(sg, np.concatenate([synth.pack(hap[:, :17]), synth.pack(hap[:, 17:])], 1),
                         17, n - 17, pos, gmap, params=sg.selscan_default_params(**c))
        assert_xpehh_equal(gotx, refx)


@pytest.mark.parametrize("schedule", ["in_order", "sweep"])
def test_physical_map_on_gpu(sg, chr22, xp, schedule):
    """use_physical_map on both the per-step and the sorted-sweep walks: g is the
    position difference; a decreasing map is passed to show it is neither read
    for g nor rejected."""
    L = sg.make_launch(sg.SCHED_IN_ORDER if schedule == "in_order" else sg.SCHED_SWEEP)
    p = sg.selscan_default_params(use_physical_map=1)
    bad_map = chr22.gmap[::-1].copy()
    ref = oracle.ihs(chr22.rows, 204, chr22.pos, bad_map, p=oracle.params(use_physical_map=1))
    got = run_ihs(sg, chr22.rows, 204, chr22.pos, bad_map, params=p, launch=L)
    assert_ihs_equal(got, ref)
    refx = oracle.xpehh(xp.rows, 204, 210, xp.pos, xp.gmap, p=oracle.params(use_physical_map=1))
    gotx = run_xpehh(sg, xp.rows, 204, 210, xp.pos, xp.gmap, params=p, launch=L)
    assert_xpehh_equal(gotx, refx)


def test_physical_map_single_locus(sg, chr22):
    hap, pos, gmap = sg.to_device(chr22.rows, chr22.pos, chr22.gmap)
    p = sg.selscan_default_params(use_physical_map=1)
    for locus in (5, 11_000, 22_000):
        got = sg.selscan_ehh(hap, 204, pos, gmap, locus, capacity=64, params=p)
        ref = oracle.ehh(chr22.rows, 204, chr22.pos, chr22.gmap, locus, capacity=64,
                         p=oracle.params(use_physical_map=1))
        np.testing.assert_allclose(got["ihh"].cpu().numpy().reshape(ref["ihh"].shape), ref["ihh"],
                                   rtol=1e-12, atol=0)


def _norm_equal(got, ref):
    g = {k: v.cpu().numpy() for k, v in got.items() if not k.startswith("_")}
    assert np.array_equal(g["count"], ref["count"])
    assert np.array_equal(np.isnan(g["score"]), np.isnan(ref["score"]))
    ok = ~np.isnan(ref["score"])
    np.testing.assert_allclose(g["score"][ok], ref["score"][ok], rtol=0, atol=1e-9)
    okm = ~np.isnan(ref["mean"])
    np.testing.assert_allclose(g["mean"][okm], ref["mean"][okm], rtol=1e-12, atol=1e-15)
    oks = ~np.isnan(ref["sd"])
    np.testing.assert_allclose(g["sd"][oks], ref["sd"][oks], rtol=1e-12)


@pytest.mark.parametrize("nbins", [1, 10, 100])
def test_normalize_ihs_on_gpu(sg, chr22, nbins):
    hap, pos, gmap = sg.to_device(chr22.rows, chr22.pos, chr22.gmap)
    o = sg.selscan_ihs(hap, 204, pos, gmap)
    got = sg.selscan_normalize(o["lnratio"], o["status"], o["n1"], 204, nbins)
    r = to_np(o)
    ref = oracle.normalize(r["lnratio"], r["status"], r["n1"], 204, nbins)
    _norm_equal(got, ref)
    # deterministic reduction: a second call gives the same bits
    again = sg.selscan_normalize(o["lnratio"], o["status"], o["n1"], 204, nbins)
    assert torch.equal(again["score"].nan_to_num(0.0), got["score"].nan_to_num(0.0))


def test_normalize_xpehh_genome_wide_on_gpu(sg, xp):
    hap, pos, gmap = sg.to_device(xp.rows, xp.pos, xp.gmap)
    o = sg.selscan_xpehh(hap, 204, 210, pos, gmap)
    got = sg.selscan_normalize(o["lnratio"], o["status"], o["n1"], 414, 1)
    r = to_np(o)
    _norm_equal(got, oracle.normalize(r["lnratio"], r["status"], r["n1"], 414, 1))


def test_normalize_edge_cases_on_gpu(sg):
    dev = torch.device("cuda")
    # 128 bins and fewer: per-thread accumulators, one read of the markers; more: per-bin CTAs
    for m, n, nbins in ((1, 10, 1), (7, 10, 4), (3000, 500, 1024), (200_000, 5000, 128),
                        (200_000, 5000, 129), (1_000_000, 5000, 100)):
        rng = np.random.default_rng(m)
        score = rng.normal(size=m)
        st = rng.choice(np.array([0, 0, 0, 1, 2, 3, 4], dtype=np.int8), size=m)
        n1 = rng.integers(0, n + 1, size=m).astype(np.int32)
        got = sg.selscan_normalize(torch.from_numpy(score).to(dev), torch.from_numpy(st).to(dev),
                                   torch.from_numpy(n1).to(dev), n, nbins)
        _norm_equal(got, oracle.normalize(score, st, n1, n, nbins))
    with pytest.raises(sg.SelscanError):
        sg.selscan_normalize(torch.zeros(5, dtype=torch.float64, device=dev),
                             torch.zeros(5, dtype=torch.int8, device=dev),
                             torch.zeros(5, dtype=torch.int32, device=dev), 10, 2000)


def test_xpehh_small_and_maf_flag(sg):
    for nA, nB in ((2, 2), (5, 64), (64, 65), (100, 31)):
        hap, pos, gmap = synth.tiny_mosaic(nA + nB, 35, nA * 31 + nB, founders=3, switch=0.1,
                                           flip=0.03)
        rows = np.concatenate([synth.pack(hap[:, :nA]), synth.pack(hap[:, nA:])], 1)
        for flag in (0, 1):
            ref = oracle.xpehh(rows, nA, nB, pos, gmap, p=oracle.params(xpehh_maf_filter=flag))
            got = run_xpehh(sg, rows, nA, nB, pos, gmap,
                            params=sg.selscan_default_params(xpehh_maf_filter=flag))
            assert_xpehh_equal(got, ref)


def test_golden_worked_examples_on_gpu(sg):
    import json
    import os
    gd = os.path.join(os.path.dirname(__file__), "golden")
    g = json.load(open(os.path.join(gd, "worked_example_ihs.json")))
    rows = synth.pack(np.array(g["hap"], dtype=np.uint8))
    got = run_ihs(sg, rows, 6, np.array(g["pos"]), np.array(g["gmap"]))
    c, e = g["core"], g["expect_ihs"]
    assert got["status"][c] == e["status"] and got["stop"][c].tolist() == e["stop"]
    assert got["digest"][c].tolist() == e["digest"]
    assert got["lnratio"][c] == pytest.approx(e["lnratio"], abs=1e-12)
    g = json.load(open(os.path.join(gd, "worked_example_xpehh.json")))
    hap = np.array(g["hap"], dtype=np.uint8)
    rows = np.concatenate([synth.pack(hap[:, :4]), synth.pack(hap[:, 4:])], 1)
    got = run_xpehh(sg, rows, 4, 4, np.array(g["pos"]), np.array(g["gmap"]))
    e = g["expect"]
    assert got["digest"][c].tolist() == e["digest"] and got["stop"][c].tolist() == e["stop"]
    assert got["lnratio"][c] == pytest.approx(e["lnratio"], abs=1e-12)


def test_ehh_trace_matches_oracle(sg, chr22):
    hap, p, g = sg.to_device(chr22.rows, chr22.pos, chr22.gmap)
    ref_all = oracle.ihs(chr22.rows, 204, chr22.pos, chr22.gmap)
    core = int(np.argmin(np.abs(chr22.pos - 17_500_000)))
    loci = [0, 1, 5000, core, core + 3, 22146] + list(np.flatnonzero(ref_all["status"] == 4)[:2])
    for locus in loci:
        for cap in (4, 4096):
            out = sg.selscan_ehh(hap, 204, p, g, int(locus), cap)
            sg.check(out)
            got = to_np(out)
            ref = oracle.ehh(chr22.rows, 204, chr22.pos, chr22.gmap, int(locus), cap)
            assert np.array_equal(got["len"], ref["len"]), locus
            assert np.array_equal(got["stop"], ref["stop"])
            assert np.array_equal(got["status"], ref["status"])
            assert np.array_equal(got["denom"], ref["denom"])
            for w in range(3):
                for d in range(2):
                    k = min(int(ref["len"][w, d]), cap)
                    assert np.array_equal(got["S"][w, d, :k], ref["S"][w, d, :k])
            np.testing.assert_allclose(got["ihh"], ref["ihh"], rtol=1e-12, atol=0)


def test_pack_matches_reference_packing(sg):
    for n, m in ((1, 3), (64, 5), (100, 17), (333, 40)):
        h = synth.tiny_random(n, m, n + m)[0]
        want = synth.pack(h, ld=(n + 63) // 64 + 1)
        t = torch.from_numpy(h).cuda()
        got = sg.selscan_pack(t, n, ld=want.shape[1]).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want)
        t2 = torch.from_numpy(np.ascontiguousarray(h.T)).cuda()
        got2 = sg.selscan_pack(t2, n, hap_major=True, ld=want.shape[1]).cpu().numpy().view(np.uint64)
        assert np.array_equal(got2, want)


def test_pack_any_byte_values_and_both_load_paths(sg):
    """Only bit 0 of each byte counts; marker counts that are multiples of 16
    take the haplotype-major kernel's 16-byte loads (with a ragged last block
    of markers), the others its byte loads; row strides with pad words."""
    rng = np.random.default_rng(7)
    for n, m in ((130, 128), (70, 200), (64, 64), (65, 1024), (1000, 4096 + 16), (5, 80),
                 (2049, 336)):
        h = rng.integers(0, 256, size=(m, n), dtype=np.uint8)
        for ld in ((n + 63) // 64, (n + 63) // 64 + 3):
            want = synth.pack(h, ld=ld)
            got = sg.selscan_pack(torch.from_numpy(h).cuda(), n, ld=ld)
            assert np.array_equal(got.cpu().numpy().view(np.uint64), want), (n, m, ld, "mm")
            hm = torch.from_numpy(np.ascontiguousarray(h.T)).cuda()
            got2 = sg.selscan_pack(hm, n, hap_major=True, ld=ld)
            assert np.array_equal(got2.cpu().numpy().view(np.uint64), want), (n, m, ld, "hm")


def test_pack_matches_reference_packing_at_full_size(sg):
    """Device packing of the bench's 5,000 x 1,000,000 matrix from 0/1 bytes
    (5 GB), marker-major and haplotype-major, equals the generator's packing
    bit for bit (pad bits 0)."""
    d = synth.generate(synth.spec("ihs1m"))
    want = torch.from_numpy(d.rows.view(np.int64)).cuda()
    hap01 = torch.from_numpy(synth.unpack(d.rows, 5000)).cuda()       # [m, n]
    got = sg.selscan_pack(hap01, 5000)
    assert torch.equal(got, want)
    del got
    hm = hap01.t().contiguous()                                        # [n, m]
    del hap01
    got2 = sg.selscan_pack(hm, 5000, hap_major=True)
    assert torch.equal(got2, want)


def test_unsorted_input_sets_device_error(sg, plain):
    pos = plain.pos.copy()
    pos[100], pos[101] = pos[101], pos[100]
    hap, p, g = sg.to_device(plain.rows, pos, plain.gmap)
    out = sg.selscan_ihs(hap, 100, p, g)
    with pytest.raises(sg.SelscanError) as e:
        sg.check(out)
    assert e.value.code == sg.ERR_UNSORTED


def longest_walk_cores(got, k):
    """The k walked cores with the largest sum of stop indices on the GPU (the
    selection uses the GPU's output; the comparison is element by element)."""
    walked = np.flatnonzero(got["status"] != 1)
    tot = got["stop"][walked].astype(np.int64).sum(1)
    return walked[np.argsort(-tot, kind="stable")[:k]]


def sweep_region_cores(d, m, half=8):
    """Every planted sweep's core marker and its neighbours within +-half markers."""
    c = synth.sweep_cores(d)
    near = (c[:, None] + np.arange(-half, half + 1)[None, :]).ravel()
    return near[(near >= 0) & (near < m)]


def test_1m_sampled_cores_and_invariants(sg):
    """The bench's workload at full size (5,000 x 1,000,000, 20 planted
    sweeps) in the default launch (the sorted sweep): 48 random cores, every
    sweep centre with its +-8 neighbours (the long EHH tails the statistic is
    about) and the 128 cores with the longest walks on the GPU match the
    oracle element by element; properties hold at every core."""
    d = synth.generate(synth.spec("ihs1m"))
    got = run_ihs(sg, d.rows, 5000, d.pos, d.gmap)
    rng = np.random.default_rng(0)
    cores = np.unique(np.concatenate([rng.choice(d.spec.m, 48, replace=False),
                                      sweep_region_cores(d, d.spec.m),
                                      longest_walk_cores(got, 128)]))
    ref = oracle.ihs(d.rows, 5000, d.pos, d.gmap, cores=cores)
    assert_ihs_equal(got, ref, idx=cores)
    # the sweep centres walk hundreds of steps each way
    centres = np.searchsorted(cores, synth.sweep_cores(d))
    assert np.all(ref["stop"][centres, :2].min(1) > 100)
    # properties at every core
    st = got["status"]
    assert set(np.unique(st)) <= {0, 1, 2, 3, 4}
    walked = st != 1
    assert np.all(got["ihh1"][walked] >= 0) and np.all(got["ihh0"][walked] >= 0)
    assert np.array_equal(np.isfinite(got["lnratio"]), st == 0)
    idx = np.arange(d.spec.m)
    assert np.all(got["stop"][walked, 0] <= idx[walked] + 1)
    assert np.all(got["stop"][walked, 1] <= d.spec.m - idx[walked])
    n1 = synth.unpack(d.rows[:2000], 5000).sum(1)
    assert np.array_equal(got["n1"][:2000], n1)


@pytest.mark.parametrize("schedule", ["default", "in_order"])
def test_200k_every_sweep_centre(sg, schedule):
    """1,000 haplotypes x 200,000 SNPs on 50 Mb with four planted sweeps (an
    iHS analogue of the 200k XPEHH case): every sweep centre with its +-16
    neighbours, 64 random cores and the 64 longest GPU walks match the oracle
    in the default launch (the sorted sweep) and in the per-step schedule."""
    d = synth.generate(synth.spec("ihs200k"))
    L = None if schedule == "default" else sg.make_launch(sg.SCHED_IN_ORDER)
    got = run_ihs(sg, d.rows, 1000, d.pos, d.gmap, launch=L)
    rng = np.random.default_rng(3)
    cores = np.unique(np.concatenate([rng.choice(d.spec.m, 64, replace=False),
                                      sweep_region_cores(d, d.spec.m, half=16),
                                      longest_walk_cores(got, 64)]))
    ref = oracle.ihs(d.rows, 1000, d.pos, d.gmap, cores=cores)
    assert_ihs_equal(got, ref, idx=cores)
    centres = np.searchsorted(cores, synth.sweep_cores(d))
    assert np.all(ref["status"][centres] == 0)
    assert np.all(ref["stop"][centres, :2].min(1) > 100)
