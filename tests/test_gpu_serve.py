"""Serving on the GPU: every result of a continuous-batching run (scans of
different modes and sizes sharing ticks) equals the result of the same scan
run alone through selscan_ihs / selscan_xpehh."""
import numpy as np
import pytest

import synth
from parity_util import IHH_RTOL, LN_ATOL, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg
    return sg


def make_requests():
    from paper_1403_6854_gb300.serve import Request
    out = []
    shapes = [("ihs", 100, 0, 3000), ("xpehh", 70, 130, 2500), ("ihs", 513, 0, 4000),
              ("ihs", 64, 0, 1500), ("xpehh", 200, 64, 3500), ("ihs", 1000, 0, 2000)]
    for i, (mode, nA, nB, m) in enumerate(shapes):
        pops = [synth.PopSpec(nA, 20)] + ([synth.PopSpec(nB, 30)] if mode == "xpehh" else [])
        spec = synth.ScanSpec(f"s{i}", mode, m, 250 * m, 500 + i, pops)
        d = synth.generate(spec)
        out.append(Request(i, mode, d.rows, d.pos, d.gmap, nA, nB, arrival=0.0))
    return out


def alone(sg, r):
    hap, pos, gmap = sg.to_device(r.rows, r.pos, r.gmap)
    if r.mode == "ihs":
        o = to_np(sg.selscan_ihs(hap, r.nA, pos, gmap))
        return {"status": o["status"], "n1": o["n1"], "ihh_a": o["ihh1"], "ihh_b": o["ihh0"],
                "lnratio": o["lnratio"], "stop": o["stop"], "digest": o["digest"]}
    o = to_np(sg.selscan_xpehh(hap, r.nA, r.nB, pos, gmap))
    return {"status": o["status"], "n1": o["n1"], "ihh_a": o["ihhA"], "ihh_b": o["ihhB"],
            "lnratio": o["lnratio"], "stop": o["stop"], "digest": o["digest"]}


def test_served_results_equal_alone(sg):
    from paper_1403_6854_gb300.serve import GpuExecutor, footprint, serve
    reqs = make_requests()
    budget = sum(footprint(r) for r in reqs[:3])      # at most ~3 resident: admission matters
    res, lat, mk = serve(reqs, GpuExecutor(), budget, tick_cores=700, realtime=False)
    assert sorted(res) == [r.rid for r in reqs]
    for r in reqs:
        got, ref = res[r.rid], alone(sg, r)
        for f in ("status", "n1", "stop", "digest"):
            assert np.array_equal(got[f], ref[f]), (r.rid, f)
        for f in ("ihh_a", "ihh_b"):
            np.testing.assert_allclose(got[f], ref[f], rtol=IHH_RTOL, atol=0)
        ok = ~np.isnan(ref["lnratio"])
        assert np.array_equal(np.isnan(got["lnratio"]), ~ok)
        np.testing.assert_allclose(got["lnratio"][ok], ref["lnratio"][ok], rtol=0, atol=LN_ATOL)


def test_whole_scans_next_to_ticks_equal_alone(sg):
    """Requests above the whole-scan threshold run as one sorted-sweep call on a
    side stream while the others take ticks; every result equals the scan alone."""
    from paper_1403_6854_gb300.serve import GpuExecutor, serve
    reqs = make_requests()
    ex = GpuExecutor(whole_min_markers=2600, whole_stage_cores=37)
    assert {r.rid for r in reqs if ex.is_whole(r)} == {0, 2, 4}
    budget = sum(ex.footprint(r) for r in reqs)
    res, lat, mk = serve(reqs, ex, budget, tick_cores=700, realtime=False)
    for r in reqs:
        got, ref = res[r.rid], alone(sg, r)
        for f in ("status", "n1", "stop", "digest"):
            assert np.array_equal(got[f], ref[f]), (r.rid, f)
        np.testing.assert_allclose(got["ihh_a"], ref["ihh_a"], rtol=IHH_RTOL, atol=0)
        np.testing.assert_allclose(got["ihh_b"], ref["ihh_b"], rtol=IHH_RTOL, atol=0)


def test_server_futures_equal_alone(sg):
    """The online form: futures resolve to the same results; a cancelled
    resident scan frees its memory and the rest complete."""
    from paper_1403_6854_gb300.serve import GpuExecutor, Server, footprint
    reqs = make_requests()
    srv = Server(GpuExecutor(), sum(footprint(r) for r in reqs[:2]), tick_cores=500,
                 policy="srpt")
    futs = {r.rid: srv.submit(r) for r in reqs}
    srv.cancel(4)
    for r in reqs:
        if r.rid == 4:
            continue
        got, ref = futs[r.rid].result(timeout=300), alone(sg, r)
        for f in ("status", "n1", "stop", "digest"):
            assert np.array_equal(got[f], ref[f]), (r.rid, f)
        np.testing.assert_allclose(got["ihh_a"], ref["ihh_a"], rtol=IHH_RTOL, atol=0)
    assert futs[4].cancelled() or futs[4].done()
    import time
    t = time.time()
    while srv._loop.busy() and time.time() - t < 60:
        time.sleep(0.01)
    srv.close()
    assert srv._loop.sch.used == 0


@pytest.mark.parametrize("schedule", [None, -1])
def test_plain_runner_equals_alone(sg, schedule):
    """Both comparison arms of the served bench (plain launches, and the
    library's default launch one request at a time) give the scan alone."""
    from paper_1403_6854_gb300.serve import run_plain
    reqs = make_requests()[:3]
    res, lat, mk = run_plain(reqs, realtime=False, schedule=schedule)
    for r in reqs:
        ref = alone(sg, r)
        assert np.array_equal(res[r.rid]["stop"], ref["stop"])
        assert np.array_equal(res[r.rid]["digest"].view(np.uint64), ref["digest"])
