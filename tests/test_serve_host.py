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


@pytest.mark.parametrize("policy", ["fifo", "srpt", "ps"])
def test_ticks_cover_every_core_once(policy):
    sch = Scheduler(hbm_budget=1 << 40, tick_cores=1000, policy=policy)
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
        # one contiguous range per scan and tick, in the order of `live`
        assert units[:, 0].tolist() == list(range(len(live)))
        for i, c0, c1 in units.tolist():
            assert 0 <= c0 < c1 <= live[i].req.m
            assert c0 == live[i].next_core - (c1 - c0)
            seen[live[i].req.rid][c0:c1] += 1
            per[i] = per.get(i, 0) + c1 - c0
        # the tick budget is respected; the policy decides who goes first
        assert sum(per.values()) <= 1000
        if policy == "srpt":
            assert live == sorted(live, key=lambda a: a.remaining + per.get(live.index(a), 0))
        if policy == "fifo":
            assert [a.req.rid for a in live] == sorted(a.req.rid for a in live)
            assert per[0] == min(1000, live[0].req.m - (live[0].next_core - per[0]))
        if policy == "ps":
            assert max(per.values()) <= 1000 // len(live)
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
                         realtime=False)
    assert sorted(res) == list(range(9))
    assert all((v == 1).all() for v in res.values())
    assert all(t >= 0 for t in lat.values())
    assert max(ex.ticks) > 1          # several scans shared a tick
    s = summarize(lat, cores=sum(r.m for r in rs), makespan=mk)
    assert s["requests"] == 9 and s["p99_ms"] >= s["p50_ms"]


def test_scheduler_cancel_waiting_only():
    sch = Scheduler(hbm_budget=footprint(req(0)))
    for r in (req(0), req(1)):
        sch.submit(r)
    sch.admit()
    assert not sch.cancel(0)          # resident: not the scheduler's to drop
    assert sch.cancel(1) and not sch.waiting
    assert not sch.cancel(7)


class SlowExecutor(FakeExecutor):
    """Fake executor whose ticks take wall time, so that requests stay open."""

    def __init__(self, tick_s=0.002):
        import threading
        super().__init__()
        self.tick_s = tick_s
        self.uploaded = {}
        self.lock = threading.Lock()

    def upload(self, r):
        import threading
        with self.lock:
            self.uploaded.setdefault(r.rid, threading.Event()).set()
        return super().upload(r)

    def seen(self, rid):
        import threading
        with self.lock:
            return self.uploaded.setdefault(rid, threading.Event())

    def run_tick(self, live, units):
        import time
        time.sleep(self.tick_s)
        super().run_tick(live, units)


def test_server_futures_resolve_with_results():
    from paper_1403_6854_gb300.serve import Server
    rs = [req(i, m=200 + 50 * i, mode="ihs" if i % 2 else "xpehh") for i in range(6)]
    srv = Server(FakeExecutor(), hbm_budget=sum(footprint(r) for r in rs[:2]), tick_cores=128)
    futs = [srv.submit(r) for r in rs]
    outs = [f.result(timeout=30) for f in futs]
    srv.close()
    assert all(o.shape == (r.m,) and (o == 1).all() for o, r in zip(outs, rs))


def test_server_cancel_waiting_and_resident():
    from paper_1403_6854_gb300.serve import Server
    big = [req(i, m=20000) for i in range(3)]
    # one scan resident at a time: 1 waits behind 0, 2 behind 1
    ex = SlowExecutor()
    srv = Server(ex, hbm_budget=footprint(big[0]), tick_cores=100)
    f0, f1, f2 = (srv.submit(r) for r in big)
    srv.cancel(1)                          # waiting
    assert ex.seen(0).wait(30)
    srv.cancel(0)                          # resident: 200 ticks of 2 ms are far from done
    assert f2.result(timeout=60).shape == (20000,)
    assert not ex.seen(1).is_set()         # never uploaded
    assert f1.cancelled() and f0.cancelled()
    srv.close()
    assert srv._loop.sch.used == 0 and not srv._loop.sch.active


def test_server_rejects_oversized_and_duplicate():
    from paper_1403_6854_gb300.serve import Server
    srv = Server(SlowExecutor(0.01), hbm_budget=footprint(req(0, m=5000)))
    with pytest.raises(ValueError):
        srv.submit(req(0, m=100000))
    f = srv.submit(req(3, m=5000))
    with pytest.raises(ValueError):
        srv.submit(req(3, m=10))
    f.result(timeout=30)
    srv.close()
