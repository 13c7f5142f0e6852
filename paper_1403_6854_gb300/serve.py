"""Continuous-batching server for iHS / XPEHH scans on one GPU.

Requests (scans of any mode and size) arrive over time.  The server keeps the
packed matrices of admitted scans resident in HBM, admits waiting requests in
arrival order as soon as their HBM footprint fits the budget, and runs
"ticks": one persistent walk launch (selscan_batch_run) over core ranges of
the resident scans in policy order, so requests that arrive while others run
join the very next tick and their walks share the GPU.  A scan whose cores
are all walked is finalised, its results are copied to the host and its
memory is released.  Latency = result on the host - arrival.

`Scheduler` holds the host-side policy (admission, tick composition) and is
independent of the GPU; `GpuExecutor` runs it on the device through the
C ABI; `serve` replays a list of timed requests, `Server` is the online form
(submit -> Future, cancel); `run_plain` is the comparison: each request
alone, in arrival order, with one plain launch (one CTA per core).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np


@dataclass
class Request:
    rid: int
    mode: str                     # "ihs" or "xpehh"
    rows: np.ndarray              # packed uint64 [m, ld]
    pos: np.ndarray               # int64 [m]
    gmap: np.ndarray              # float64 [m]
    nA: int
    nB: int = 0
    arrival: float = 0.0          # seconds after the start of the run
    params: Dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.rows.shape[0]

    @property
    def ld(self) -> int:
        return self.rows.shape[1]

    @property
    def n_total(self) -> int:
        return self.nA + (self.nB if self.mode == "xpehh" else 0)


OUT_BYTES_PER_MARKER = {"ihs": 1 + 4 + 8 * 3 + 4 * 4 + 8 * 4, "xpehh": 1 + 4 + 8 * 3 + 4 * 2 + 8 * 6}
ITEM_BYTES_PER_MARKER = {"ihs": 4 * (1 + 8), "xpehh": 2 * (1 + 16)}


def footprint(req: Request) -> int:
    """Device bytes a resident scan holds: inputs, outputs, per-walk results."""
    return int(req.rows.nbytes + req.pos.nbytes + req.gmap.nbytes +
               req.m * (OUT_BYTES_PER_MARKER[req.mode] + ITEM_BYTES_PER_MARKER[req.mode]) + 4096)


@dataclass
class Active:
    req: Request
    next_core: int = 0
    handle: object = None         # executor state
    fp: int = 0                   # HBM bytes held while resident
    whole: bool = False           # runs as one whole-scan launch instead of ticks

    @property
    def remaining(self) -> int:
        return self.req.m - self.next_core


class Scheduler:
    """Admission by HBM footprint (FIFO) and tick composition by policy."""

    POLICIES = ("fifo", "srpt", "ps")
    MAX_SCANS = 64                # scans one tick can carry (the C ABI's limit)

    def __init__(self, hbm_budget: int, tick_cores: int = 32768, max_active: int = MAX_SCANS,
                 policy: str = "fifo", footprint_fn: Optional[Callable[[Request], int]] = None):
        if policy not in self.POLICIES:
            raise ValueError(policy)
        self.policy = policy
        self.fp = footprint_fn or footprint
        self.budget = int(hbm_budget)
        self.tick_cores = int(tick_cores)
        self.max_active = min(int(max_active), self.MAX_SCANS)
        self.waiting: deque = deque()
        self.active: List[Active] = []
        self.used = 0

    def submit(self, req: Request) -> None:
        if self.fp(req) > self.budget:
            raise ValueError(f"request {req.rid} needs {self.fp(req)} B, budget {self.budget} B")
        self.waiting.append(req)

    def cancel(self, rid: int) -> bool:
        """Drop a request that has not been admitted yet; True if it was waiting."""
        for r in self.waiting:
            if r.rid == rid:
                self.waiting.remove(r)
                return True
        return False

    def admit(self) -> List[Active]:
        """Admit waiting requests, in arrival order, while they fit."""
        new = []
        while self.waiting and len(self.active) < self.max_active:
            f = self.fp(self.waiting[0])
            if self.used + f > self.budget:
                break
            req = self.waiting.popleft()
            self.used += f
            a = Active(req, fp=f)
            self.active.append(a)
            new.append(a)
        return new

    def compose_tick(self) -> Tuple[List[Active], np.ndarray]:
        """Core ranges for the next tick: one contiguous range per scan, the
        tick's core budget handed out in policy order ("fifo" oldest first,
        younger scans backfill what the oldest cannot use; "srpt" least
        remaining work first; "ps" equal shares).  The device walks the ranges
        in this order, one core per warp fetch.  Returns the tick's scans and
        an int64 array of units (index into that list, c0, c1)."""
        live = [a for a in self.active if a.remaining > 0 and not a.whole]
        if not live:
            return [], np.zeros((0, 3), np.int64)
        if self.policy == "srpt":
            live.sort(key=lambda a: a.remaining)
        share = max(1, self.tick_cores // len(live)) if self.policy == "ps" else None
        budget = self.tick_cores
        out, rows = [], []
        for a in live:
            if budget <= 0:
                break
            take = min(budget, a.remaining, share or budget)
            rows.append((len(out), a.next_core, a.next_core + take))
            out.append(a)
            a.next_core += take
            budget -= take
        return out, np.array(rows, np.int64).reshape(-1, 3)

    def has_work(self) -> bool:
        return any(a.remaining > 0 and not a.whole for a in self.active)

    def finished(self) -> List[Active]:
        done = [a for a in self.active if a.remaining == 0]
        return done

    def release(self, a: Active) -> None:
        self.active.remove(a)
        self.used -= a.fp


def summarize(latencies: Dict[int, float], cores: int, makespan: float) -> Dict:
    lat = np.array(sorted(latencies.values()))
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "requests": int(lat.size),
            "core_loci_per_s": cores / makespan if makespan > 0 else 0.0, "makespan_s": makespan}


class GpuExecutor:
    """Runs the scheduler's ticks on the GPU through the batch C ABI.  Ticks
    alternate between two streams so that one tick's tail overlaps the next
    tick's start; a scan is finalised after every tick that touched it.

    Long requests (those a default launch sorts, `selscan_default_schedule`,
    or with at least `whole_min_markers` markers when that is given, and at
    most 16383 haplotypes) do not take ticks: each runs as one whole-scan call with the
    sorted-sweep schedule on one of `whole_streams` side streams, its results
    copied to pinned host memory behind it, so it completes asynchronously
    next to the ticks.  Its footprint includes the sweep's workspace (stages
    of `whole_stage_cores` cores keep the slot buffer near 1 GiB)."""

    WHOLE_MAX_N = 16383

    def __init__(self, device="cuda", whole_min_markers: Optional[int] = None, whole_streams: int = 3,
                 whole_stage_cores: int = 256):
        import torch
        import paper_1403_6854_gb300 as sg
        self.torch, self.sg = torch, sg
        self.device = torch.device(device)
        self.whole_min = None if whole_min_markers is None else int(whole_min_markers)
        self.whole_stage = int(whole_stage_cores)
        self.wstreams = [torch.cuda.Stream(self.device) for _ in range(max(1, whole_streams))]
        self.wk = 0
        self.streams = [torch.cuda.Stream(self.device), torch.cuda.Stream(self.device)]
        self.events = [None, None]
        self.ws = [None, None]
        self._ws_raw = [None, None]
        self.k = 0
        self.last_tick = {}

    # ------------------------------------------------------------ whole scans
    def is_whole(self, req: Request) -> bool:
        if req.n_total > self.WHOLE_MAX_N:
            return False
        if self.whole_min is None:
            mode = self.sg.MODE_IHS if req.mode == "ihs" else self.sg.MODE_XPEHH
            return self.sg.selscan_default_schedule(req.n_total, req.m, mode) == self.sg.SCHED_SWEEP
        return self.whole_min > 0 and req.m >= self.whole_min

    def _whole_launch(self):
        return self.sg.make_launch(self.sg.SCHED_SWEEP, sweep_stage_cores=self.whole_stage)

    def footprint(self, req: Request) -> int:
        f = footprint(req)
        if self.is_whole(req):
            mode = self.sg.MODE_IHS if req.mode == "ihs" else self.sg.MODE_XPEHH
            f += self.sg.selscan_workspace_bytes(req.n_total, req.m, mode, self._whole_launch())
        return f

    def start_whole(self, a: Active):
        """Queue the whole scan and the copy of its results; returns a handle
        for poll_finish."""
        torch, sg = self.torch, self.sg
        req = a.req
        st = self.wstreams[self.wk % len(self.wstreams)]
        self.wk += 1
        p = sg.selscan_default_params(**req.params)
        L = self._whole_launch()
        with torch.cuda.stream(st):
            hap, pos, gmap = sg.to_device(req.rows, req.pos, req.gmap, self.device)
            if req.mode == "ihs":
                o = sg.selscan_ihs(hap, req.nA, pos, gmap, params=p, launch=L, stream=st)
                o["ihh_a"], o["ihh_b"] = o["ihh1"], o["ihh0"]
            else:
                o = sg.selscan_xpehh(hap, req.nA, req.nB, pos, gmap, params=p, launch=L, stream=st)
                o["ihh_a"], o["ihh_b"] = o["ihhA"], o["ihhB"]
            host = {}
            for f in self.FIELDS:
                h = torch.empty(o[f].shape, dtype=o[f].dtype, pin_memory=True)
                h.copy_(o[f], non_blocking=True)
                host[f] = h
        done = torch.cuda.Event()
        done.record(st)
        return (done, host, (o, hap, pos, gmap))

    # ------------------------------------------------------------ ticks
    def upload(self, req: Request):
        torch, sg = self.torch, self.sg
        dev = self.device
        mode = sg.MODE_IHS if req.mode == "ihs" else sg.MODE_XPEHH
        m = req.m
        ipc = 4 if req.mode == "ihs" else 2
        ndig = 4 if req.mode == "ihs" else 6
        st = self.streams[self.k % 2]
        with torch.cuda.stream(st):
            t = dict(hap=torch.from_numpy(np.ascontiguousarray(req.rows).view(np.int64)).to(dev),
                     pos=torch.from_numpy(np.ascontiguousarray(req.pos)).to(dev),
                     gmap=torch.from_numpy(np.ascontiguousarray(req.gmap)).to(dev),
                     status=torch.empty(m, dtype=torch.int8, device=dev),
                     n1=torch.empty(m, dtype=torch.int32, device=dev),
                     ihh_a=torch.empty(m, dtype=torch.float64, device=dev),
                     ihh_b=torch.empty(m, dtype=torch.float64, device=dev),
                     lnratio=torch.empty(m, dtype=torch.float64, device=dev),
                     stop=torch.empty((m, ipc), dtype=torch.int32, device=dev),
                     digest=torch.empty((m, ndig), dtype=torch.int64, device=dev),
                     error=torch.zeros(1, dtype=torch.int32, device=dev))
            nb = sg.selscan_batch_item_bytes(m, mode)
            raw = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
        off = (-raw.data_ptr()) % 256
        t["items"] = raw[off:off + nb]
        t["_raw"] = raw
        p = sg.selscan_default_params(**req.params)
        s = sg.selscan_scan()
        s.mode, s.nA, s.nB, s.m, s.ld = mode, req.nA, req.nB if req.mode == "xpehh" else 0, m, req.ld
        s.params = p
        s.hap, s.pos_bp, s.gmap = t["hap"].data_ptr(), t["pos"].data_ptr(), t["gmap"].data_ptr()
        for f in ("status", "n1", "ihh_a", "ihh_b", "lnratio", "stop", "digest", "error", "items"):
            setattr(s, f, t[f].data_ptr())
        sg.selscan_batch_prepare(s, st)
        # both streams must see the prepared scan before any tick uses it
        ev = torch.cuda.Event()
        ev.record(st)
        self.streams[(self.k + 1) % 2].wait_event(ev)
        return (s, t)

    def wait_slot(self) -> None:
        """Block until the stream the next tick goes to has finished its
        previous tick, so that no more than two ticks are ever queued."""
        ev = self.events[self.k % 2]
        if ev is not None:
            ev.synchronize()

    def run_tick(self, live: List[Active], units) -> None:
        sg, torch = self.sg, self.torch
        i = self.k % 2
        st = self.streams[i]
        scans = [a.handle[0] for a in live]
        max_n = max(a.req.n_total for a in live)
        max_ld = max(a.req.ld for a in live)
        need = sg.selscan_batch_workspace_bytes(max_n, max_ld, len(scans), max(1, len(units)))
        if self.ws[i] is None or self.ws[i].numel() < need:
            with torch.cuda.stream(st):
                raw = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
            off = (-raw.data_ptr()) % 256
            self.ws[i] = raw[off:off + need]
            self._ws_raw[i] = raw
        sg.selscan_batch_run(scans, units[:, 0], units[:, 1], units[:, 2], max_n, max_ld,
                             self.ws[i], st)
        ev = torch.cuda.Event()
        ev.record(st)
        self.events[i] = ev
        for a in live:
            self.last_tick[a.req.rid] = self.k
        self.k += 1

    FIELDS = ("status", "n1", "ihh_a", "ihh_b", "lnratio", "stop", "digest", "error")

    def start_finish(self, a: Active):
        """Queue finalisation and the copy of the results to pinned host memory
        on the completion stream, after every tick issued so far; returns a
        handle for poll_finish."""
        torch = self.torch
        s, t = a.handle
        if not hasattr(self, "fstream"):
            self.fstream = torch.cuda.Stream(self.device)
        fs = self.fstream
        for ev in self.events:
            if ev is not None:
                fs.wait_event(ev)
        self.sg.selscan_batch_finalize(s, fs)
        host = {}
        with torch.cuda.stream(fs):
            for f in self.FIELDS:
                h = torch.empty(t[f].shape, dtype=t[f].dtype, pin_memory=True)
                h.copy_(t[f], non_blocking=True)
                host[f] = h
        done = torch.cuda.Event()
        done.record(fs)
        self.last_tick.pop(a.req.rid, None)
        return (done, host, t)

    def poll_finish(self, handle, block: bool = False):
        """Results of a queued finalisation once they are on the host, else None."""
        done, host, _ = handle
        if block:
            done.synchronize()
        elif not done.query():
            return None
        out = {f: host[f].numpy() for f in self.FIELDS}
        out["digest"] = out["digest"].view(np.uint64)
        if int(out["error"][0]) != 0:
            # a device error ends the serving loop and fails every open request:
            # a TIMEOUT voids the whole tick it happened in, including the other
            # scans' walks of that tick, so no result of it may be returned
            raise self.sg.SelscanError(int(out["error"][0]), "served scan")
        return out

    def finish(self, a: Active) -> Dict[str, np.ndarray]:
        return self.poll_finish(self.start_finish(a), block=True)


class _Loop:
    """One pass of the serving loop: admit, launch the next tick, queue the
    finalisation of scans whose cores are all walked, collect finished ones.
    The host never waits for the GPU unless told to (nothing left to launch)."""

    def __init__(self, sch: Scheduler, executor):
        self.sch, self.ex = sch, executor
        self.finishing: List[Tuple[Active, object]] = []
        self.cancelled = set()
        self.async_finish = hasattr(executor, "start_finish")
        self.whole = hasattr(executor, "start_whole")

    def busy(self) -> bool:
        return bool(self.sch.waiting or self.sch.active or self.finishing)

    def cancel(self, rid: int) -> bool:
        """Cancel a waiting or resident scan.  A resident scan stops receiving
        ticks; its memory is released once the ticks already issued for it
        are done."""
        if self.sch.cancel(rid):
            return True
        for a in self.sch.active:
            if a.req.rid == rid:
                self.cancelled.add(rid)
                a.next_core = a.req.m
                return True
        return False

    def step(self, may_block: bool) -> Tuple[List[Tuple[Active, Optional[Dict]]], bool]:
        """Returns (done, idle): scans completed in this pass with their results
        (None for a cancelled scan) and whether no tick was launched."""
        sch, ex = self.sch, self.ex
        done = []
        for a in sch.admit():
            if self.whole and ex.is_whole(a.req):
                a.whole = True
                a.next_core = a.req.m
                self.finishing.append((a, ex.start_whole(a)))
            else:
                a.handle = ex.upload(a.req)
        if sch.has_work() and hasattr(ex, "wait_slot"):
            ex.wait_slot()      # at most two ticks in flight: new scans join the next one
        live, units = sch.compose_tick()
        if len(units):
            ex.run_tick(live, units)
        queued = {id(f[0]) for f in self.finishing}
        for a in sch.finished():
            if id(a) in queued:
                continue
            if self.async_finish:
                self.finishing.append((a, ex.start_finish(a)))
            else:
                done.append((a, ex.finish(a)))
                sch.release(a)
        idle = not len(units)
        still = []
        for a, h in self.finishing:
            out = ex.poll_finish(h, block=idle and may_block)
            if out is None:
                still.append((a, h))
                continue
            done.append((a, out))
            sch.release(a)
        self.finishing = still
        for i, (a, out) in enumerate(done):
            if a.req.rid in self.cancelled:
                self.cancelled.discard(a.req.rid)
                done[i] = (a, None)
        return done, idle


def serve(requests: List[Request], executor, hbm_budget: int, tick_cores: int = 32768,
          clock: Callable[[], float] = time.perf_counter,
          realtime: bool = True, policy: str = "fifo") -> Tuple[Dict[int, Dict], Dict[int, float], float]:
    """Replay requests (by arrival time; realtime=False submits all at once).
    Returns results, latencies (result on the host - arrival), makespan."""
    loop = _Loop(Scheduler(hbm_budget, tick_cores, policy=policy,
                           footprint_fn=getattr(executor, "footprint", None)), executor)
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    results, latency = {}, {}
    t0 = clock()
    while pending or loop.busy():
        now = clock() - t0
        while pending and (pending[0].arrival <= now or not realtime):
            loop.sch.submit(pending.popleft())
        done, idle = loop.step(may_block=not (pending and realtime))
        for a, out in done:
            results[a.req.rid] = out
            latency[a.req.rid] = (clock() - t0) - a.req.arrival
        if idle and not loop.finishing and pending and realtime:
            wait = pending[0].arrival - (clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.002))
    return results, latency, clock() - t0


class Server:
    """Online form of the loop: submit() (from any thread) returns a Future
    that resolves to the scan's results; cancel() drops a waiting or resident
    scan (its Future is cancelled).  A background thread runs the loop and
    owns the executor; close() drains nothing, it stops after the current
    pass and cancels whatever is still open."""

    def __init__(self, executor, hbm_budget: int, tick_cores: int = 32768, policy: str = "fifo",
                 idle_wait: float = 0.002):
        import threading
        self._loop = _Loop(Scheduler(hbm_budget, tick_cores, policy=policy,
                                     footprint_fn=getattr(executor, "footprint", None)), executor)
        self._lock = threading.Lock()
        self._inbox: deque = deque()
        self._cancels: deque = deque()
        self._futures: Dict[int, "Future"] = {}
        self._wake = threading.Event()
        self._stop = False
        self._idle_wait = idle_wait
        self._error: Optional[BaseException] = None
        self._thread = threading.Thread(target=self._run, name="selscan-serve", daemon=True)
        self._thread.start()

    def submit(self, req: Request):
        from concurrent.futures import Future
        need = self._loop.sch.fp(req)
        if need > self._loop.sch.budget:
            raise ValueError(f"request {req.rid} needs {need} B, budget {self._loop.sch.budget} B")
        fut = Future()
        with self._lock:
            if self._stop:
                raise RuntimeError("server closed")
            if req.rid in self._futures:
                raise ValueError(f"request id {req.rid} is open")
            self._futures[req.rid] = fut
            self._inbox.append(req)
        self._wake.set()
        return fut

    def cancel(self, rid: int) -> None:
        with self._lock:
            self._cancels.append(rid)
        self._wake.set()

    def close(self, timeout: Optional[float] = None) -> None:
        with self._lock:
            self._stop = True
        self._wake.set()
        self._thread.join(timeout)
        with self._lock:
            for f in self._futures.values():
                f.cancel()
            self._futures.clear()
        if self._error is not None:
            raise self._error

    def _resolve(self, rid: int, out) -> None:
        with self._lock:
            fut = self._futures.pop(rid, None)
        if fut is None:
            return
        if out is None:
            fut.cancel()
        elif fut.set_running_or_notify_cancel():
            fut.set_result(out)

    def _run(self) -> None:
        loop = self._loop
        try:
            while True:
                with self._lock:
                    if self._stop:
                        return
                    while self._inbox:
                        loop.sch.submit(self._inbox.popleft())
                    cancels = list(self._cancels)
                    self._cancels.clear()
                for rid in cancels:
                    waiting = any(r.rid == rid for r in loop.sch.waiting)
                    if loop.cancel(rid) and waiting:
                        self._resolve(rid, None)
                if not loop.busy():
                    self._wake.wait(self._idle_wait)
                    self._wake.clear()
                    continue
                done, idle = loop.step(may_block=False)
                for a, out in done:
                    self._resolve(a.req.rid, out)
                if idle and loop.finishing:
                    time.sleep(self._idle_wait / 4)
        except BaseException as e:          # surfaced to every open Future and by close()
            self._error = e
            with self._lock:
                futs = list(self._futures.values())
                self._futures.clear()
            for f in futs:
                if f.set_running_or_notify_cancel():
                    f.set_exception(e)


def run_plain(requests: List[Request], device="cuda", clock: Callable[[], float] = time.perf_counter,
              realtime: bool = True, schedule: Optional[int] = None
              ) -> Tuple[Dict[int, Dict], Dict[int, float], float]:
    """Comparison: each request alone, in arrival order, one call per request.
    schedule None: plain launches (one CTA per core, no persistence); a
    schedule number (SCHED_DEFAULT: the library's own choice, the sorted sweep
    for long chromosomes and the persistent per-step walk otherwise) isolates
    what serving adds over running the same algorithm one request at a time."""
    import torch
    import paper_1403_6854_gb300 as sg
    results, latency = {}, {}
    L = sg.make_launch(sg.SCHED_PLAIN if schedule is None else schedule)
    t0 = clock()
    for req in sorted(requests, key=lambda r: r.arrival):
        if realtime:
            wait = req.arrival - (clock() - t0)
            if wait > 0:
                time.sleep(wait)
        hap, pos, gmap = sg.to_device(req.rows, req.pos, req.gmap, device)
        p = sg.selscan_default_params(**req.params)
        if req.mode == "ihs":
            o = sg.selscan_ihs(hap, req.nA, pos, gmap, params=p, launch=L)
        else:
            o = sg.selscan_xpehh(hap, req.nA, req.nB, pos, gmap, params=p, launch=L)
        out = {k: v.cpu().numpy() for k, v in o.items() if not k.startswith("_")}
        results[req.rid] = out
        latency[req.rid] = (clock() - t0) - req.arrival
        del o
    torch.cuda.synchronize()
    return results, latency, clock() - t0
