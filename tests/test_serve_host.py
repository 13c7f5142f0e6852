"""Serving policy on the host (no GPU): admission by HBM footprint in arrival
order, tick composition that walks every core of every scan exactly once,
and the serving loop driven by a fake executor."""
import numpy as np
import pytest

from paper_1403_6854_gb300.serve import Request, Scheduler, footprint, serve, summarize


def req(rid, m=1000, n=100, mode="ihs", arrival=0.0):
    W = (n + 63) // 64
    return Request(rid, mode, np.zeros((m, W if mode == "ihs" else 2 * W), np.uint64),
                   np.arange(m, dtype=np.int64), np.zeros(m), n, n if mode == "xpehh" else 0,
                   arrival)


def test_admission_respects_budget_and_order():
    a, b, c = req(0, m=1000), req(1, m=5000), req(2, m=1000)
    sch = Scheduler(hbm_budget=footprint(a) + footprint(b) - 1)
    for r in (a, b, c):
        sch.submit(r)
    adm = sch.admit()
    # b does not fit next to a; c must wait behind b (arrival order is kept)
    assert [x.req.rid for x in adm] == [0]
    sch.release(adm[0])
    assert [x.req.rid for x in sch.admit()] == [1]


def test_oversized_request_rejected():
    with pytest.raises(ValueError):
        Scheduler(hbm_budget=100).submit(req(0))


def test_ticks_cover_every_core_once_smallest_first():
    sch = Scheduler(hbm_budget=1 << 40, tick_cores=1000, unit_cores=64)
    rs = [req(i, m=m) for i, m in enumerate((700, 2500, 90))]
    for r in rs:
        sch.submit(r)
    sch.admit()
    seen = {r.rid: np.zeros(r.m, int) for r in rs}
    ticks = 0
    while True:
        live, units = sch.compose_tick()
        if not len(units):
            break
        ticks += 1
        per = {}
        for i, c0, c1 in units.tolist():
            assert 0 <= c0 < c1 <= live[i].req.m and c1 - c0 <= 64
            seen[live[i].req.rid][c0:c1] += 1
            per[i] = per.get(i, 0) + c1 - c0
        # the tick budget is respected and the smallest remaining scan comes first
        assert sum(per.values()) <= 1000
        assert live == sorted(live, key=lambda a: a.remaining + per.get(live.index(a), 0))
        for a in sch.finished():
            sch.release(a)
    assert all((v == 1).all() for v in seen.values())
    assert ticks >= 3 and sch.used == 0


class FakeExecutor:
    def __init__(self):
        self.ticks = []

    def upload(self, r):
        return {"cores": np.zeros(r.m, int)}

    def run_tick(self, live, units):
        self.ticks.append(len({live[int(u[0])].req.rid for u in units}))
        for i, c0, c1 in units:
            live[int(i)].handle["cores"][c0:c1] += 1

    def finish(self, a):
        return a.handle["cores"].copy()


def test_serve_loop_completes_everything_and_overlaps_scans():
    rs = [req(i, m=300 + 97 * i, mode="ihs" if i % 3 else "xpehh", arrival=0.0) for i in range(9)]
    ex = FakeExecutor()
    res, lat, mk = serve(rs, ex, hbm_budget=sum(footprint(r) for r in rs[:4]), tick_cores=256,
                         unit_cores=32, realtime=False)
    assert sorted(res) == list(range(9))
    assert all((v == 1).all() for v in res.values())
    assert all(t >= 0 for t in lat.values())
    assert max(ex.ticks) > 1          # several scans shared a tick
    s = summarize(lat, cores=sum(r.m for r in rs), makespan=mk)
    assert s["requests"] == 9 and s["p99_ms"] >= s["p50_ms"]
