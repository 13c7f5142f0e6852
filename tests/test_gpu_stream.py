"""Scans of host-resident data sets through paper_1403_6854_gb300.stream.

Each data set's results through the stream (upload of the next data set
overlapped with the current scan, results read back on their own stream) must
equal, bit for bit, those of the same library call on device-resident inputs,
for both schedules, for marker counts that change within the stream, and for
XPEHH.  A device-side error is raised at the result of the scan that caused it.
"""
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


def host(rows, pos, gmap):
    return (torch.from_numpy(np.ascontiguousarray(rows).view(np.int64)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(pos, dtype=np.int64)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(gmap, dtype=np.float64)).pin_memory())


def device_result(sg, mode, n, nB, rows, pos, gmap, launch, fields):
    hap, p, g = sg.to_device(rows, pos, gmap)
    if mode == sg.MODE_IHS:
        out = sg.selscan_ihs(hap, n, p, g, launch=launch)
    else:
        out = sg.selscan_xpehh(hap, n, nB, p, g, launch=launch)
    sg.check(out)
    r = to_np(out)
    return {f: r[f] for f in fields}


def chr22_sets():
    sets = []
    for seed, m in ((0, 22147), (1, 15000), (2, 22147), (3, 9000)):
        d = synth.generate(synth.spec("chr22", seed=seed))
        sets.append((d.rows[:m], d.pos[:m], d.gmap[:m]))
    return sets


@pytest.mark.parametrize("schedule", [-1, 3])
def test_ihs_stream_equals_device_calls(sg, schedule):
    from paper_1403_6854_gb300.stream import IHS_FIELDS, scan_host_stream
    sets = chr22_sets()
    launch = sg.make_launch(schedule) if schedule >= 0 else None
    got = [{f: v.numpy().copy() for f, v in r.items()}
           for r in scan_host_stream([host(*s) for s in sets], sg.MODE_IHS, 204, max_m=22147,
                                     launch=launch)]
    assert len(got) == len(sets)
    for g, s in zip(got, sets):
        want = device_result(sg, sg.MODE_IHS, 204, 0, *s, launch, IHS_FIELDS)
        assert g["status"].shape[0] == s[0].shape[0]
        assert_bitwise_equal(g, want)


def test_stream_growing_marker_counts(sg):
    """Data sets in increasing size: the workspace sized for the first is
    replaced when a later one needs more (sorted sweep, stages by size)."""
    from paper_1403_6854_gb300.stream import IHS_FIELDS, scan_host_stream
    sets = list(reversed(sorted(chr22_sets(), key=lambda t: -t[0].shape[0])))
    assert sets[0][0].shape[0] < sets[-1][0].shape[0]
    launch = sg.make_launch(sg.SCHED_SWEEP)
    got = [{f: v.numpy().copy() for f, v in r.items()}
           for r in scan_host_stream([host(*s) for s in sets], sg.MODE_IHS, 204, max_m=22147,
                                     launch=launch)]
    for g, s in zip(got, sets):
        assert_bitwise_equal(g, device_result(sg, sg.MODE_IHS, 204, 0, *s, launch, IHS_FIELDS))


def test_xpehh_stream_equals_device_calls(sg):
    from paper_1403_6854_gb300.stream import XPEHH_FIELDS, scan_host_stream
    sets = []
    for seed in (0, 1, 2):
        d = synth.generate(synth.spec("xpehh", seed=seed))
        sets.append((d.rows, d.pos, d.gmap))
    got = [{f: v.numpy().copy() for f, v in r.items()}
           for r in scan_host_stream([host(*s) for s in sets], sg.MODE_XPEHH, 204, 210)]
    for g, s in zip(got, sets):
        assert_bitwise_equal(g, device_result(sg, sg.MODE_XPEHH, 204, 210, *s, None, XPEHH_FIELDS))


def test_stream_raises_at_the_failing_scan(sg):
    from paper_1403_6854_gb300.stream import scan_host_stream
    d = synth.generate(synth.spec("plain"))
    bad = d.pos.copy()
    bad[100], bad[101] = bad[101], bad[100]
    stream = scan_host_stream([host(d.rows, d.pos, d.gmap), host(d.rows, bad, d.gmap),
                               host(d.rows, d.pos, d.gmap)], sg.MODE_IHS, 100)
    first = next(stream)
    assert (first["status"].numpy() != sg.LOCUS_UNDEFINED).any()
    with pytest.raises(sg.SelscanError) as e:
        next(stream)
    assert e.value.code == sg.ERR_UNSORTED
    # the library stays usable after the failed stream
    hap, p, g = sg.to_device(d.rows, d.pos, d.gmap)
    sg.check(sg.selscan_ihs(hap, 100, p, g))


def test_stream_closed_early_then_reused(sg):
    from paper_1403_6854_gb300.stream import scan_host_stream
    d = synth.generate(synth.spec("plain"))
    h = host(d.rows, d.pos, d.gmap)
    want = device_result(sg, sg.MODE_IHS, 100, 0, d.rows, d.pos, d.gmap, None, ("lnratio", "stop"))
    for r in scan_host_stream([h] * 5, sg.MODE_IHS, 100, fields=("lnratio", "stop")):
        assert_bitwise_equal({f: v.numpy() for f, v in r.items()}, want)
        break
    r = list(scan_host_stream([h], sg.MODE_IHS, 100, fields=("lnratio", "stop")))
    assert len(r) == 1
    assert_bitwise_equal({f: v.numpy() for f, v in r[0].items()}, want)


@pytest.mark.parametrize("layout", ["hap_major", "marker_major"])
def test_ihs_stream_of_unpacked_bytes(sg, layout):
    """0/1 bytes uploaded and packed on the device inside the stream: every
    result equals the scan of the generator's packed rows."""
    from paper_1403_6854_gb300.stream import IHS_FIELDS, scan_host_stream
    sets = chr22_sets()
    items = []
    for rows, pos, gmap in sets:
        mm = synth.unpack(np.ascontiguousarray(rows), 204)            # [m, n] bytes
        b = np.ascontiguousarray(mm.T) if layout == "hap_major" else mm
        items.append((torch.from_numpy(b).pin_memory(),) + host(rows, pos, gmap)[1:])
    got = [{f: v.numpy().copy() for f, v in r.items()}
           for r in scan_host_stream(items, sg.MODE_IHS, 204, max_m=22147, layout=layout)]
    assert len(got) == len(sets)
    for g, s in zip(got, sets):
        assert_bitwise_equal(g, device_result(sg, sg.MODE_IHS, 204, 0, *s, None, IHS_FIELDS))


def test_stream_passes_parameters(sg):
    """Non-default parameters (physical map, the crossing term, a 1/4 cutoff)
    reach every scan of the stream."""
    from paper_1403_6854_gb300.stream import IHS_FIELDS, XPEHH_FIELDS, scan_host_stream
    p = sg.selscan_default_params(use_physical_map=1, include_crossing_term=1, ehh_cut=(1, 4))
    sets = chr22_sets()[:2]
    got = [{f: v.numpy().copy() for f, v in r.items()}
           for r in scan_host_stream([host(*s) for s in sets], sg.MODE_IHS, 204, max_m=22147,
                                     params=p)]
    for g, (rows, pos, gmap) in zip(got, sets):
        hap, dp, dg = sg.to_device(rows, pos, gmap)
        want = sg.selscan_ihs(hap, 204, dp, dg, params=p)
        sg.check(want)
        w = to_np(want)
        assert_bitwise_equal(g, {f: w[f] for f in IHS_FIELDS})
    d = synth.generate(synth.spec("xpehh"))
    r = next(scan_host_stream([host(d.rows, d.pos, d.gmap)], sg.MODE_XPEHH, 204, 210, params=p))
    hap, dp, dg = sg.to_device(d.rows, d.pos, d.gmap)
    want = sg.selscan_xpehh(hap, 204, 210, dp, dg, params=p)
    sg.check(want)
    w = to_np(want)
    assert_bitwise_equal({f: v.numpy() for f, v in r.items()}, {f: w[f] for f in XPEHH_FIELDS})
