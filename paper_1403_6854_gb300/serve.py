"""Continuous-batching server for iHS / XPEHH scans on one GPU.

Requests (scans of any mode and size) arrive over time.  The server keeps the
packed matrices of admitted scans resident in HBM, admits waiting requests in
arrival order as soon as their HBM footprint fits the budget, and runs
"ticks": one persistent walk launch (selscan_batch_run) over core ranges taken
round-robin from every resident scan, so requests that arrive while others
run join the very next tick and their walks share the GPU.  A scan whose cores
are all walked is finalised, its results are copied to the host and its
memory is released.  Latency = result on the host - arrival.

`Scheduler` holds the host-side policy (admission, tick composition) and is
independent of the GPU; `GpuExecutor` runs it on the device through the
C ABI; `run_plain` is the comparison: each request alone, in arrival order,
with one plain launch (one CTA per core).
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

    @property
    def remaining(self) -> int:
        return self.req.m - self.next_core


class Scheduler:
    """Admission by HBM footprint (FIFO) and round-robin tick composition."""

    def __init__(self, hbm_budget: int, tick_cores: int = 32768, unit_cores: int = 4,
                 max_active: int = 64):
        self.budget = int(hbm_budget)
        self.tick_cores = int(tick_cores)
        self.unit_cores = int(unit_cores)
        self.max_active = int(max_active)
        self.waiting: deque = deque()
        self.active: List[Active] = []
        self.used = 0

    def submit(self, req: Request) -> None:
        if footprint(req) > self.budget:
            raise ValueError(f"request {req.rid} needs {footprint(req)} B, budget {self.budget} B")
        self.waiting.append(req)

    def admit(self) -> List[Active]:
        """Admit waiting requests, in arrival order, while they fit."""
        new = []
        while self.waiting and len(self.active) < self.max_active:
            f = footprint(self.waiting[0])
            if self.used + f > self.budget:
                break
            req = self.waiting.popleft()
            self.used += f
            a = Active(req)
            self.active.append(a)
            new.append(a)
        return new

    def compose_tick(self) -> Tuple[List[Active], np.ndarray]:
        """Core ranges for the next tick.  The tick's core budget goes to the
        resident scans with the least remaining work first (shortest remaining
        work first: a small request finishes within a tick or two of its
        admission), split into units of unit_cores cores that are interleaved
        across scans.  Returns the tick's scans and an int64 array of units
        (index into that list, c0, c1)."""
        live = sorted((a for a in self.active if a.remaining > 0), key=lambda a: a.remaining)
        if not live:
            return [], np.zeros((0, 3), np.int64)
        budget = self.tick_cores
        parts = []
        for i, a in enumerate(live):
            if budget <= 0:
                live = live[:i]
                break
            take = min(budget, a.remaining)
            c0 = np.arange(a.next_core, a.next_core + take, self.unit_cores, dtype=np.int64)
            c1 = np.minimum(c0 + self.unit_cores, a.next_core + take)
            k = np.arange(c0.size, dtype=np.int64)
            parts.append(np.stack([k, np.full(c0.size, i, np.int64), c0, c1], 1))
            a.next_core += take
            budget -= take
        u = np.concatenate(parts)
        u = u[np.lexsort((u[:, 1], u[:, 0]))]      # interleave: unit k of every scan, then k + 1
        return live, u[:, 1:]

    def finished(self) -> List[Active]:
        done = [a for a in self.active if a.remaining == 0]
        return done

    def release(self, a: Active) -> None:
        self.active.remove(a)
        self.used -= footprint(a.req)


def summarize(latencies: Dict[int, float], cores: int, makespan: float) -> Dict:
    lat = np.array(sorted(latencies.values()))
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "requests": int(lat.size),
            "core_loci_per_s": cores / makespan if makespan > 0 else 0.0, "makespan_s": makespan}


class GpuExecutor:
    """Runs the scheduler's ticks on the GPU through the batch C ABI.  Ticks
    alternate between two streams so that one tick's tail overlaps the next
    tick's start; a scan is finalised after every tick that touched it."""

    def __init__(self, device="cuda"):
        import torch
        import paper_1403_6854_gb300 as sg
        self.torch, self.sg = torch, sg
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(self.device), torch.cuda.Stream(self.device)]
        self.events = [None, None]
        self.ws = [None, None]
        self._ws_raw = [None, None]
        self.k = 0
        self.last_tick = {}

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

    def finish(self, a: Active) -> Dict[str, np.ndarray]:
        torch = self.torch
        s, t = a.handle
        st = self.streams[self.last_tick.get(a.req.rid, self.k) % 2]
        other = self.events[(self.last_tick.get(a.req.rid, self.k) + 1) % 2]
        if other is not None:
            st.wait_event(other)
        self.sg.selscan_batch_finalize(s, st)
        st.synchronize()
        out = {f: t[f].cpu().numpy() for f in ("status", "n1", "ihh_a", "ihh_b", "lnratio", "stop",
                                               "digest", "error")}
        out["digest"] = out["digest"].view(np.uint64)
        if int(out["error"][0]) != 0:
            raise self.sg.SelscanError(int(out["error"][0]), f"request {a.req.rid}")
        self.last_tick.pop(a.req.rid, None)
        return out


def serve(requests: List[Request], executor, hbm_budget: int, tick_cores: int = 32768,
          unit_cores: int = 4, clock: Callable[[], float] = time.perf_counter,
          realtime: bool = True) -> Tuple[Dict[int, Dict], Dict[int, float], float]:
    """Serve requests (sorted by arrival).  Returns results, latencies, makespan."""
    sch = Scheduler(hbm_budget, tick_cores, unit_cores)
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    results, latency = {}, {}
    t0 = clock()
    while pending or sch.waiting or sch.active:
        now = clock() - t0
        while pending and (pending[0].arrival <= now or not realtime):
            sch.submit(pending.popleft())
        for a in sch.admit():
            a.handle = executor.upload(a.req)
        live, units = sch.compose_tick()
        if len(units):
            executor.run_tick(live, units)
        for a in sch.finished():
            results[a.req.rid] = executor.finish(a)
            latency[a.req.rid] = (clock() - t0) - a.req.arrival
            sch.release(a)
        if not len(units) and not sch.finished() and pending and realtime:
            wait = pending[0].arrival - (clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    return results, latency, clock() - t0


def run_plain(requests: List[Request], device="cuda", clock: Callable[[], float] = time.perf_counter,
              realtime: bool = True) -> Tuple[Dict[int, Dict], Dict[int, float], float]:
    """Comparison: each request alone, in arrival order, one plain launch (one CTA per core)."""
    import torch
    import paper_1403_6854_gb300 as sg
    results, latency = {}, {}
    L = sg.make_launch(sg.SCHED_PLAIN)
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
