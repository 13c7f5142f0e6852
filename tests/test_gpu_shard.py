"""Core-range scans (one scan split over GPUs, paper Section 3) on one GPU.

The ranges of a split run one after another here; their concatenation must
equal the whole scan bit for bit (status, n1, stops, digests, iHH, ln ratio),
in every schedule, including ranges too short for the sorted sweep next to
ones that take it, and sweeps whose walks are handed to the second pass.
The normalisation steps (per-bin sums per shard, totals, statistics, scores)
must agree with the one-call standardisation."""
import numpy as np
import pytest
import torch

import synth
from parity_util import assert_bitwise_equal, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg
    return sg


def scan(sg, mode, d, hap, pos, gmap, k0=None, k1=None, launch=None):
    nA = d.spec.pops[0].n
    m = d.spec.m
    k0 = 0 if k0 is None else k0
    k1 = m if k1 is None else k1
    if mode == "ihs":
        out = sg.selscan_ihs_range(hap, nA, pos, gmap, k0, k1, launch=launch)
    else:
        out = sg.selscan_xpehh_range(hap, nA, d.spec.pops[1].n, pos, gmap, k0, k1, launch=launch)
    sg.check(out)
    return to_np(out)


def concat(parts):
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


CASES = [
    ("ihs", "chr22", [0, 7000, 7001, 22147], None),
    ("ihs", "chr22", [0, 11000, 22147], dict(schedule=3, sweep_warmup=40, sweep_stage_cores=7)),
    ("ihs", "chr22", [0, 1, 2, 22146, 22147], dict(schedule=3)),
    ("xpehh", "xpehh", [0, 5000, 22147], None),
    ("xpehh", "xpehh", [0, 9999, 22147], dict(schedule=3, sweep_warmup=64)),
    ("ihs", "ihs200k", [0, 20000, 133000, 200000], None),       # per-step, sweep, sweep
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_ranges_concatenate_to_the_whole_scan(sg, case):
    mode, name, cuts, lk = CASES[case]
    d = synth.generate(synth.spec(name))
    hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
    launch = sg.make_launch(**lk) if lk else None
    whole = scan(sg, mode, d, hap, pos, gmap, launch=launch)
    parts = [scan(sg, mode, d, hap, pos, gmap, a, b, launch=launch) for a, b in zip(cuts, cuts[1:])]
    assert_bitwise_equal(whole, concat(parts))


def test_partitioned_ranges_of_the_1m_scan(sg):
    """The bench's 1M workload split into the ranges of four ranks
    (shard.partition), run one after another: bit-identical to the whole."""
    from paper_1403_6854_gb300 import shard
    d = synth.generate(synth.spec("ihs1m"))
    hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
    whole = scan(sg, "ihs", d, hap, pos, gmap)
    ranges = shard.partition(d.spec.m, 4)
    parts = [scan(sg, "ihs", d, hap, pos, gmap, a, b) for a, b in ranges]
    assert_bitwise_equal(whole, concat(parts))


def test_range_arguments_rejected(sg):
    d = synth.generate(synth.spec("plain"))
    hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
    for k0, k1 in ((5, 5), (10, 3), (-1, 4), (0, 2001)):
        with pytest.raises(sg.SelscanError) as e:
            sg.selscan_ihs_range(hap, 100, pos, gmap, k0, k1)
        assert e.value.code == sg.ERR_INVALID_ARG


@pytest.mark.parametrize("nbins,cuts", [(100, [0, 7000, 22147]), (10, [0, 1, 15000, 22147]),
                                        (1, [0, 11073, 22147])])
def test_normalisation_steps_over_shards(sg, nbins, cuts):
    """Per-shard bin sums, totals summed over the shards (what the all-reduce
    does across GPUs), bin statistics and scores agree with selscan_normalize
    on the whole scan: counts exactly, the rest to rounding."""
    d = synth.generate(synth.spec("chr22"))
    hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
    o = sg.selscan_ihs(hap, 204, pos, gmap)
    want = sg.selscan_normalize(o["lnratio"], o["status"], o["n1"], 204, nbins)
    sh = [(o["lnratio"][a:b], o["status"][a:b], o["n1"][a:b]) for a, b in zip(cuts, cuts[1:])]
    cnt = torch.zeros(nbins, dtype=torch.int64, device=hap.device)
    tot = torch.zeros(nbins, dtype=torch.float64, device=hap.device)
    for s, st, n1 in sh:
        c, t = sg.selscan_normalize_bin_sums(s, st, n1, 204, nbins, 0)
        cnt += c
        tot += t
    mean = sg.selscan_normalize_finish(nbins, 0, cnt, tot)
    sq = torch.zeros(nbins, dtype=torch.float64, device=hap.device)
    for s, st, n1 in sh:
        sq += sg.selscan_normalize_bin_sums(s, st, n1, 204, nbins, 1, mean)[1]
    sd = sg.selscan_normalize_finish(nbins, 1, cnt, sq)
    z = torch.cat([sg.selscan_normalize_apply(s, st, n1, 204, nbins, cnt, mean, sd)
                   for s, st, n1 in sh])
    assert torch.equal(cnt, want["count"])
    for got, ref in ((mean, want["mean"]), (sd, want["sd"])):
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.array_equal(np.isnan(g), np.isnan(r))
        ok = ~np.isnan(r)
        np.testing.assert_allclose(g[ok], r[ok], rtol=1e-12, atol=1e-15)
    g, r = z.cpu().numpy(), want["score"].cpu().numpy()
    assert np.array_equal(np.isnan(g), np.isnan(r))
    ok = ~np.isnan(r)
    np.testing.assert_allclose(g[ok], r[ok], rtol=0, atol=1e-9)
