"""Benchmark: iHS core loci/s on one GB300 (and N GPUs under torchrun).

Workload (default): batched iHS at scale, 5,000 haplotypes x 1,000,000 SNPs on
250 Mb, 200-founder mosaic, 20 planted sweeps (synth.spec("ihs1m")).  One step
is one whole scan through the C ABI (core selection, every EHH walk, iHH and
ln ratios) with the packed matrix already resident in HBM.  The matrix
(632 MB) is larger than L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "ihs1m": "batched iHS at scale: 5,000 haplotypes x 1,000,000 SNPs on 250 Mb, 200-founder "
             "mosaic, 20 planted sweeps of 50-500 kb at 30-90% carrier frequency",
    "ihs250k": "profiling case: the ihs1m recipe on 5,000 haplotypes x 250,000 SNPs on 62.5 Mb, "
               "5 planted sweeps",
    "chr22": "iHS chr22-shaped: 204 haplotypes x 22,147 SNPs on 35 Mb, 30 founders, planted 400 kb sweep",
    "plain": "iHS plain: 100 haplotypes x 2,000 SNPs on 2 Mb, 10 founders",
}
METRIC = "iHS/XPEHH core loci/s on 1 GB300; served p50/p99 scan latency vs plain launches"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def walk_lengths(stop, pos, max_gap_bp, ipc=4, k0=0):
    """Steps computed by each walk (S values, i = 0 .. last), from its stop index
    (stop holds the cores k0, k0 + 1, ... of a chromosome whose positions are pos)."""
    m = pos.shape[0]
    j = (k0 + np.arange(stop.shape[0]))[:, None].repeat(ipc, 1)
    d = (np.arange(ipc) & 1)[None, :].repeat(stop.shape[0], 0)
    s = stop.astype(np.int64)
    edge = np.where(d == 0, s == j + 1, s == m - j)
    x = np.where(d == 0, j - s, j + s)
    xp = np.where(d == 0, x + 1, x - 1)
    xc = np.clip(x, 0, m - 1)
    xpc = np.clip(xp, 0, m - 1)
    gap = (~edge) & (s > 0) & (np.abs(pos[xc] - pos[xpc]) > max_gap_bp)
    ln = np.where(s == 0, 0, np.where(edge | gap, s, s + 1))
    return ln


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(data, budget_s=20.0, seed=1234):
    """Time the CPU oracle, as it stands, on a bounded stratified sample of
    cores: the markers inside the planted sweep windows (whose long walks cost
    the string-enumeration oracle the most) and the rest, each sampled at
    random; the scan's oracle time is estimated stratum by stratum (a
    stratum's sampled time x its markers / sampled markers), so neither kind of
    core is over-represented."""
    import oracle
    d = data
    n = d.spec.pops[0].n
    rng = np.random.default_rng(seed)
    inside = np.zeros(d.spec.m, bool)
    for c, w, _ in d.spec.pops[0].sweeps:
        inside |= np.abs(d.pos - c) <= w / 2
    strata = {"sweep windows": np.flatnonzero(inside), "elsewhere": np.flatnonzero(~inside)}
    # the sweep windows get half of the budget (when they exist): their few
    # cores carry most of the oracle's time and of the estimate's variance
    budgets = {"sweep windows": budget_s / 2 if strata["sweep windows"].size else 0.0}
    budgets["elsewhere"] = budget_s - budgets["sweep windows"]
    threads = os.cpu_count() or 1
    est_time, walked_all, parts = 0.0, 0, []
    for name, pool in strata.items():
        if pool.size == 0 or budgets[name] <= 0:
            continue
        order = rng.permutation(pool)
        done, walked, t, k = 0, 0, 0.0, 0
        chunk = 2 * threads if name == "sweep windows" else 8 * threads
        while t < budgets[name] and k < len(order):
            cores = np.sort(order[k:k + chunk])
            k += chunk
            t0 = time.perf_counter()
            r = oracle.ihs(d.rows, n, d.pos, d.gmap, cores=cores, threads=threads)
            t += time.perf_counter() - t0
            done += len(cores)
            walked += int((r["status"] != oracle.MAF_FILTERED).sum())
        est_time += t * pool.size / done
        walked_all += walked * pool.size / done
        parts.append(f"{name}: {done} of {pool.size} markers ({walked} MAF-passing), {t:.1f} s")
    return {"value": walked_all / est_time, "unit": "core loci/s", "cores": threads,
            "kind": "oracle",
            "sample": "stratified random sample of the same matrix, the oracle's time for the "
                      "whole scan estimated per stratum (" + "; ".join(parts) +
                      f"; {threads} host threads)"}


def rank_spec(workload: str, rank: int, scaling: str = "weak"):
    """Weak scaling: rank r scans its own chromosome (seed r) of the same shape;
    strong scaling: every rank holds the same chromosome (seed 0) and scans its
    share of the cores."""
    import synth
    return synth.spec(workload, seed=rank if scaling == "weak" else 0)


def aggregate(ms: float, cores: int, world: int, device):
    """Whole-job numbers: the slowest rank's time and the core loci of all ranks
    (one all-reduce of two scalars; nothing on the data path is exchanged)."""
    if world <= 1:
        return ms, float(cores)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, float(cores)], dtype=torch.float64, device=device)
    a, b = t[:1].clone(), t[1:].clone()
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a[0]), float(b[0])


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    d = synth.generate(synth.spec(args.workload))
    for _ in range(args.warmup):
        cpu_baseline(d, budget_s=2.0)
    vals, t0 = [], time.perf_counter()
    for s in range(args.steps):
        cb = cpu_baseline(d, budget_s=args.ref_budget, seed=100 + s)
        vals.append(cb["value"])
    dt = time.perf_counter() - t0
    v = float(np.mean(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "core loci/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "sample": cb["sample"]},
        "cpu_baseline": dict(cb, value=v),
        "e2e": {"value": v, "unit": "core loci/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


SWEEP_DRAM_BYTES_PER_CORE = 4.6139e9 / 125020
# ncu capture of the 250k case (5,000 x 250,000, default sweep shape; summarised
# in profiles/sweep_split_walk_ihs250k_full.md): sweep_kernel alone read + wrote
# 3.489 GB (125,020 core loci) and issued 7.164e9 warp instructions over
# 997,618 marker passes of 5,120 elements, i.e. 44.88 thread instructions per
# sorted element and marker pass, 19.80 of them on the ALU pipe
# (sm__inst_executed_pipe_alu 3.161e9 warp instructions)
SORT_DRAM_BYTES_PER_CORE = 3.4889e9 / 125020
SORT_INSTR_PER_ELEMENT_PASS = 44.88
SORT_ALU_OPS_PER_ELEMENT_PASS = 19.80


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ihs1m", choices=list(WORKLOADS))
    ap.add_argument("--schedule", type=int, default=-1,
                    help="-1: autotuned launch shape; 0/1/2/3: fixed schedule with defaults")
    ap.add_argument("--stage-cores", type=int, default=0,
                    help="with --schedule 3: cores per chunk and sweep stage (0: the default "
                         "single stage); smaller stages need less workspace")
    ap.add_argument("--tune-cache", action="store_true")
    ap.add_argument("--served", type=int, default=200, help="requests in the served mix (0: skip)")
    ap.add_argument("--load", type=float, default=0.7, help="served arrival rate / capacity")
    ap.add_argument("--overload", type=float, default=2.0,
                    help="second served run at this arrival rate / capacity (0: skip)")
    ap.add_argument("--policy", default="fifo", choices=["fifo", "srpt", "ps"],
                    help="served tick composition")
    ap.add_argument("--tick-cores", type=int, default=32768, help="served cores per tick")
    ap.add_argument("--scaling", default="strong", choices=["strong", "weak"],
                    help="N > 1: strong = one chromosome, its cores split into contiguous ranges "
                         "(one per rank, whole matrix on every GPU), results gathered and the "
                         "standardisation's bin sums all-reduced; weak = one chromosome per rank")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--complexity", action="store_true",
                    help="sample-size and SNP-density sweeps of both exact forms, with log-log slopes")
    ap.add_argument("--tables", action="store_true",
                    help="instead of the main line: the paper's runtime-table workloads "
                         "(stand-ins) timed on the GPU and, on a bounded sample, the oracle")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.tables:
        run_tables(args)
        return
    if args.complexity:
        run_complexity(args)
        return

    import torch
    import torch.distributed as dist
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    spec = rank_spec(args.workload, rank, args.scaling)
    d = synth.generate(spec)
    from paper_1403_6854_gb300 import shard
    if args.scaling == "strong":
        ranges = shard.partition(spec.m, world)
        k0, k1 = ranges[rank]
    else:
        ranges, (k0, k1) = None, (0, spec.m)
    n = spec.pops[0].n
    W = spec.W
    hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap, dev)
    params = sg.selscan_default_params()
    K, Wm = args.steps, args.warmup
    from paper_1403_6854_gb300.tune import Autotuner
    if args.schedule >= 0:
        launch_fields, shape = dict(schedule=args.schedule), {"schedule": args.schedule,
                                                              "source": "--schedule"}
        if args.stage_cores > 0:
            launch_fields["sweep_stage_cores"] = args.stage_cores
            shape["sweep_stage_cores"] = args.stage_cores
    else:
        tuner = Autotuner(cache_path=os.path.join(ROOT, "_build_tune.json") if args.tune_cache else None)
        _, shape = tuner.launch_for(hap, pos, gmap, "ihs", n)
        from paper_1403_6854_gb300.tune import SHAPE_FIELDS
        launch_fields = {f: shape.get(f, 0) for f in SHAPE_FIELDS}
        shape = dict(shape, source=("autotuner, sorted-sweep candidates timed on the whole scan"
                                    if shape.get("schedule") == 3 else
                                    "autotuner on the first 65,536 markers"))
    # per step: before the first walk kernel, after it the sort of the first
    # stage (sweep schedule), after the last walk kernel
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(K)]
    for trio in ev:                      # create the events before handing them out
        for e_ in trio:
            e_.record()
    torch.cuda.synchronize()
    ws = None
    out = None
    for _ in range(Wm):
        out = sg.selscan_ihs_range(hap, n, pos, gmap, k0, k1, params=params,
                                   launch=sg.make_launch(**launch_fields), workspace=ws, out=out)
        ws = out["_workspace"]
    torch.cuda.synchronize()
    sg.check(out)

    gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
    gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    launches_per_step = sg.selscan_launch_count(n, k1 - k0, sg.MODE_IHS, sg.make_launch(**launch_fields))
    with ClockSampler(gpu_id) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for k in range(K):
            out = sg.selscan_ihs_range(hap, n, pos, gmap, k0, k1, params=params,
                                       launch=sg.make_launch(events=ev[k], **launch_fields),
                                       workspace=ws, out=out)
        t1.record()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    sg.check(out)
    ms = t0.elapsed_time(t1)
    walk_ms = float(np.mean([a.elapsed_time(b) for a, b, _ in ev]))
    sort_ms = float(np.mean([a.elapsed_time(c) for a, _, c in ev]))
    status = out["status"].cpu().numpy()
    stop = out["stop"].cpu().numpy()
    cores = int((status != sg.LOCUS_MAF_FILTERED).sum())
    lens = walk_lengths(stop, d.pos, params.max_gap_bp, k0=k0)
    lens[status == sg.LOCUS_MAF_FILTERED] = 0
    steps_total = int(lens.sum())
    walk_bytes = steps_total * 8 * W + int(np.maximum(lens - 1, 0).sum()) * 16

    ms_max, cores_all = aggregate(ms, cores, world, dev)
    value = cores_all * K / (ms_max / 1e3)

    # the exchange of a split scan, once after the timed steps: gather of the
    # per-core results and the two all-reduces of the standardisation's bin sums
    exchange = None
    if world > 1 and args.scaling == "strong":
        mine = {f: out[f] for f in ("status", "n1", "ihh1", "ihh0", "lnratio", "stop", "digest")}
        torch.cuda.synchronize()
        dist.barrier()
        a0 = time.perf_counter()
        full = shard.gather(mine, ranges)
        z, cnt, mean, sd = shard.normalize(shard.DeviceOps(sg), out["lnratio"], out["status"],
                                           out["n1"], n, 100)
        torch.cuda.synchronize()
        exchange = {"what": "all-gather of the per-core results and the Eq. 7 bin-sum all-reduces "
                            "(100 frequency bins), once after the timed steps",
                    "ms": (time.perf_counter() - a0) * 1e3,
                    "gathered_cores": int(full["status"].numel()),
                    "bins_with_scores": int((cnt > 0).sum())}

    # end to end: host buffers, H2D of the inputs and D2H of the scores every step
    e2e, e2e_bufs = None, None
    if rank == 0 and world == 1 and not args.no_extras:
        from paper_1403_6854_gb300.stream import scan_host_stream
        h_rows = torch.from_numpy(d.rows.view(np.int64)).pin_memory()
        h_pos = torch.from_numpy(d.pos).pin_memory()
        h_gmap = torch.from_numpy(d.gmap).pin_memory()
        e2e_fields = ("status", "lnratio", "ihh1", "ihh0")
        h2d_b = int(d.rows.nbytes + d.pos.nbytes + d.gmap.nbytes)
        d2h_b = int(sum(out[f].numel() * out[f].element_size() for f in e2e_fields))

        def e2e_stream(steps):
            # the public streaming call: upload of step k + 1 overlapped with scan k,
            # scores of step k read back behind it; the last result is on the host
            # before the clock stops
            last = None
            for r in scan_host_stream([(h_rows, h_pos, h_gmap)] * steps, sg.MODE_IHS, n,
                                      params=params, launch=sg.make_launch(**launch_fields),
                                      fields=e2e_fields, workspace=ws):
                last = r
            return last

        e2e_stream(2)                     # untimed: the stream's buffers come from the caches
        torch.cuda.synchronize()
        steps_e2e = K
        a0 = time.perf_counter()
        last = e2e_stream(steps_e2e)
        e2e_s = (time.perf_counter() - a0) / steps_e2e
        assert int((last["status"].numpy() != sg.LOCUS_MAF_FILTERED).sum()) == cores
        # one call at a time (no overlap), each step split into its parts by events
        res = {f: torch.empty(out[f].shape, dtype=out[f].dtype).pin_memory() for f in e2e_fields}
        dh, dp, dg = torch.empty_like(hap), torch.empty_like(pos), torch.empty_like(gmap)
        steps_ser = max(2, min(K, 3))
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps_ser)]
        torch.cuda.synchronize()
        a0 = time.perf_counter()
        for st in range(steps_ser):
            evs[st][0].record()
            dh.copy_(h_rows, non_blocking=True)
            dp.copy_(h_pos, non_blocking=True)
            dg.copy_(h_gmap, non_blocking=True)
            evs[st][1].record()
            o2 = sg.selscan_ihs(dh, n, dp, dg, params=params, workspace=ws,
                                launch=sg.make_launch(**launch_fields))
            evs[st][2].record()
            for f in res:
                res[f].copy_(o2[f], non_blocking=True)
            evs[st][3].record()
            torch.cuda.synchronize()
        ser_s = (time.perf_counter() - a0) / steps_ser
        h2d_ms = float(np.median([e[0].elapsed_time(e[1]) for e in evs]))
        e2e = {"value": cores / e2e_s, "unit": "core loci/s",
               "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
               "ms_per_step": e2e_s * 1e3, "steps": steps_e2e,
               "how": "paper_1403_6854_gb300.stream.scan_host_stream over the steps: pinned host "
                      "matrix, positions and map uploaded every step (overlapped with the "
                      "previous step's scan), scores read back to pinned host memory every "
                      "step; host clock from the first upload to the last result on the host",
               "serial": {"ms_per_step": ser_s * 1e3, "steps": steps_ser,
                          "what": "one call at a time: H2D, scan, D2H, synchronise",
                          "parts_ms": {"h2d": h2d_ms,
                                       "scan": float(np.median([e[1].elapsed_time(e[2])
                                                                for e in evs])),
                                       "d2h": float(np.median([e[2].elapsed_time(e[3])
                                                               for e in evs]))},
                          "h2d_gbs": h2d_b / (h2d_ms / 1e3) / 1e9}}
        e2e_bufs = (h_rows, h_pos, h_gmap, res, dh, dp, dg, o2, last)

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras = run_extras(sg, torch, synth, d, hap, pos, gmap, n, ws)
        # standardisation (Eq. 7) of this scan's scores in 100 frequency bins
        nz = sg.selscan_normalize(out["lnratio"], out["status"], out["n1"], n, 100)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(5):
            nz = sg.selscan_normalize(out["lnratio"], out["status"], out["n1"], n, 100)
        b.record()
        torch.cuda.synchronize()
        nms = a.elapsed_time(b) / 5
        extras["normalize"] = {"what": "Eq. 7 standardisation, 100 derived-frequency bins, "
                                       "deterministic two-pass reduction",
                               "ms": nms, "value": spec.m / (nms / 1e3), "unit": "markers/s",
                               "bins_with_scores": int((nz["count"] > 0).sum())}

    if rank == 0 and world == 1 and not args.no_extras:
        del e2e_bufs
        extras["ingest"] = run_ingest(sg, torch, d, n, params, launch_fields)

    if rank == 0 and world == 1 and args.served > 0 and not args.no_extras:
        extras["served"] = run_served(args, torch, synth)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(d)

    if rank == 0:
        hbm, src = peaks()
        achieved = walk_bytes / (walk_ms / 1e3) / 1e9
        path = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "walk_ms": walk_ms, "walk_bytes": walk_bytes,
                "what": "algorithmic row bytes of every walk step (sum of L x 8W + 16 (L - 1)) "
                        "over the time of all walk kernels",
                "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)"}
        work = sg.selscan_sweep_work(n, k1 - k0, sg.MODE_IHS, sg.make_launch(**launch_fields))
        if work is not None:
            # the dominant kernel, the sort, against the integer issue peak measured here:
            # four warp instructions per SM cycle (128 thread operations), which the
            # IADD3 / IMNMX chains of libselscan_peak reach; beside it the ALU pipe alone
            # (LOP3 / PRMT / funnel shift: 64 per SM cycle)
            from paper_1403_6854_gb300 import peak as int_peak
            pk = int_peak.measure()
            issue_peak = float(np.median([pk[o]["ops_per_s"] for o in ("IADD3", "IMNMX")]))
            alu_peak = float(np.median([pk[o]["ops_per_s"] for o in ("LOP3", "PRMT", "SHF")]))
            element_passes = work[0] * work[1]
            ops = element_passes * SORT_INSTR_PER_ELEMENT_PASS / (sort_ms / 1e3)
            alu = element_passes * SORT_ALU_OPS_PER_ELEMENT_PASS / (sort_ms / 1e3)
            roofline = {"bound": "alu", "kernel": "sweep_kernel (the sort; first stage)",
                        "achieved": ops / 1e9, "peak": issue_peak / 1e9, "unit": "Gop/s",
                        "frac": ops / issue_peak,
                        "traffic": cores * SORT_DRAM_BYTES_PER_CORE,
                        "traffic_note": "ncu capture of the 250k case (3.489 GB of sweep_kernel "
                                        "DRAM traffic over 125,020 core loci), scaled by core loci",
                        "kernel_ms": sort_ms, "split_walk_ms": walk_ms - sort_ms,
                        "element_passes": element_passes, "marker_passes": work[0],
                        "ops_per_element_pass": SORT_INSTR_PER_ELEMENT_PASS,
                        "ops_note": "integer thread instructions (all pipes) per sorted element and "
                                    "marker pass from the ncu capture of the 250k case, times the "
                                    "passes of this launch",
                        "peak_source": "integer issue rate (IADD3 / IMNMX chains: 128 thread "
                                       "operations = 4 warp instructions per SM cycle) measured "
                                       "in this run by libselscan_peak",
                        "alu_pipe": {"achieved": alu / 1e9, "peak": alu_peak / 1e9,
                                     "frac": alu / alu_peak,
                                     "ops_per_element_pass": SORT_ALU_OPS_PER_ELEMENT_PASS,
                                     "peak_source": "LOP3 / PRMT / funnel shift chains: 64 "
                                                    "lanes per SM cycle"},
                        "int_peaks_ops_per_sm_per_cycle": {k: round(v["ops_per_sm_per_cycle"], 2)
                                                           for k, v in pk.items()},
                        "path": path}
            if args.stage_cores > 0:
                # several stages: the timed sort is the first stage's, the passes are every
                # stage's, so no fraction is formed from them
                for r in (roofline, roofline["alu_pipe"]):
                    r["achieved"] = None
                    r["frac"] = None
                roofline["note"] = "several sweep stages (--stage-cores): no sort fraction"
        else:
            roofline = dict(path, kernel="walk_persistent_kernel (both passes)", traffic=None)
        line = {
            "metric": METRIC, "value": value, "unit": "core loci/s", "n_gpus": world,
            "steps": K, "warmup": Wm, "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": args.scaling if world > 1 else "strong", "vs_baseline": None,
            "dtype": "u64+f64",
            "data": "synthetic (seeded Li-Stephens mosaic; stands in for the paper's ms and "
                    "1000 Genomes inputs)",
            "config": {"workload": WORKLOADS[args.workload], "n_haplotypes": n, "n_snps": spec.m,
                       "core_loci_per_gpu": cores, "walk_steps_per_scan": steps_total,
                       "schedule": ["persistent longest-first", "persistent in-order",
                                    "plain one-CTA-per-core", "sorted sweep + split walk"][
                                        launch_fields.get("schedule", 1)],
                       "launch_shape": shape,
                       "l2": "inputs larger than L2 (packed matrix 632 MB), no flush",
                       "parallelism": (f"strong: one chromosome, cores split into {world} "
                                       f"contiguous ranges (rank 0: [{k0}, {k1}))"
                                       if args.scaling == "strong" else
                                       f"weak: one chromosome (seed = rank) per GPU x{world}")},
            "roofline": roofline,
            "gpu_launches": launches_per_step * K,
            "clocks": clk.summary(),
        }
        if e2e:
            line["e2e"] = e2e
        if exchange:
            line["exchange"] = exchange
        if cpu:
            line["cpu_baseline"] = cpu
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# the paper's 16-thread selscan times (s) of its runtime tables, as context
PAPER_16_THREADS_S = {"IHS250": 58, "IHS500": 150, "IHS1000": 380, "IHS2000": 752, "CEU22": 33,
                      "XP250": 25, "XP500": 67, "XP1000": 180, "XP2000": 493, "CEUYRI22": 52}


def run_tables(args):
    """One JSON line: per runtime-table workload (stand-ins of the same shape),
    the GPU scan time with the default launch and the oracle's rate on a random
    sample of cores (about 3 s of host time), extrapolated to the whole scan."""
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg
    import oracle
    rows_out = []
    names = ["IHS250", "IHS500", "IHS1000", "IHS2000", "CEU22",
             "XP250", "XP500", "XP1000", "XP2000", "CEUYRI22"]
    threads = os.cpu_count() or 1
    for name in names:
        sp = synth.spec({"CEU22": "chr22", "CEUYRI22": "xpehh"}.get(name, name))
        d = synth.generate(sp)
        hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
        nA = sp.pops[0].n
        nB = sp.pops[1].n if sp.mode == "xpehh" else 0

        def call(o):
            kw = dict(workspace=None if o is None else o["_workspace"], out=o)
            if sp.mode == "ihs":
                return sg.selscan_ihs(hap, nA, pos, gmap, **kw)
            return sg.selscan_xpehh(hap, nA, nB, pos, gmap, **kw)
        o = call(None)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            o = call(o)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        st = o["status"].cpu().numpy()
        cores = int((st != sg.LOCUS_MAF_FILTERED).sum())
        # oracle on a random sample, growing until ~3 s of host time
        rng = np.random.default_rng(7)
        walked = np.flatnonzero(st != sg.LOCUS_MAF_FILTERED)
        k, spent, done = 16, 0.0, 0
        while spent < 3.0 and done < walked.size:
            pick = np.sort(rng.choice(walked, size=min(k, walked.size), replace=False))
            t0 = time.perf_counter()
            if sp.mode == "ihs":
                oracle.ihs(d.rows, nA, d.pos, d.gmap, cores=pick, threads=threads)
            else:
                oracle.xpehh(d.rows, nA, nB, d.pos, d.gmap, cores=pick, threads=threads)
            spent = time.perf_counter() - t0
            done = pick.size
            k *= 2
        orate = done / spent if spent > 0 else 0.0
        rows_out.append({"dataset": name, "shape": f"{nA}{'+' + str(nB) if nB else ''} x {sp.m}",
                         "gpu_ms": best, "core_loci": cores,
                         "gpu_core_loci_per_s": cores / (best / 1e3),
                         "oracle_core_loci_per_s": orate, "oracle_threads": threads,
                         "oracle_sample_cores": done,
                         "paper_selscan_16_threads_s": PAPER_16_THREADS_S[name]})
    print(json.dumps({"tables": rows_out, "data": "seeded stand-ins of the same shapes (mosaic of "
                      "100 founders on 4 Mbp; chr22-shaped configs for CEU22 / CEUYRI22)",
                      "note": "the paper's times are on its 12-core Xeon and are context only"}),
          flush=True)


def loglog_slope(x, y) -> float:
    """Least-squares slope of log y against log x."""
    lx, ly = np.log(np.asarray(x, dtype=np.float64)), np.log(np.asarray(y, dtype=np.float64))
    return float(np.polyfit(lx, ly, 1)[0])


COMPLEXITY_N = (250, 500, 1000, 2000, 5000)          # at 5,000 SNPs / Mb
COMPLEXITY_D = (1250, 2500, 5000, 10000, 20000)      # SNPs / Mb, at n = 1,000


def run_complexity(args):
    """One JSON line: GPU scan time of both exact forms (per-step partition
    refinement, sorted sweep) and the walk steps over a sample-size sweep and
    a SNP-density sweep on a 20 Mb neutral region, with log-log slopes (the
    paper reports O(N D^2) for its per-step algorithm)."""
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1403_6854_gb300 as sg
    shapes = [("per_step", sg.make_launch(sg.SCHED_IN_ORDER)), ("sorted_sweep", sg.make_launch(sg.SCHED_SWEEP))]

    def point(n, dens):
        sp = synth.complexity_spec(n, dens)
        d = synth.generate(sp)
        hap, pos, gmap = sg.to_device(d.rows, d.pos, d.gmap)
        row = {"n": n, "snps_per_mb": dens, "m": sp.m}
        for name, L in shapes:
            o = sg.selscan_ihs(hap, n, pos, gmap, launch=L)
            torch.cuda.synchronize()
            best = 1e30
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                o = sg.selscan_ihs(hap, n, pos, gmap, launch=L, workspace=o["_workspace"], out=o)
                b.record()
                torch.cuda.synchronize()
                best = min(best, a.elapsed_time(b))
            row[name + "_ms"] = best
        st = o["status"].cpu().numpy()
        walked = st != sg.LOCUS_MAF_FILTERED
        row["core_loci"] = int(walked.sum())
        row["walk_steps"] = int(o["stop"].cpu().numpy()[walked].astype(np.int64).sum())
        del o, hap, pos, gmap
        return row

    n_pts = [point(n, 5000) for n in COMPLEXITY_N]
    d_pts = [point(1000, dd) for dd in COMPLEXITY_D]
    fits = {}
    for key, pts, xk in (("vs_n", n_pts, "n"), ("vs_density", d_pts, "snps_per_mb")):
        xs = [p[xk] for p in pts]
        fits[key] = {f: loglog_slope(xs, [p[f] for p in pts])
                     for f in ("per_step_ms", "sorted_sweep_ms", "walk_steps", "core_loci")}
    print(json.dumps({"complexity": {"n_sweep": n_pts, "density_sweep": d_pts, "loglog_slopes": fits},
                      "data": "seeded neutral mosaics (100 founders, 20 Mbp, 1 cM/Mb)",
                      "note": "the paper reports O(N D^2) for selscan (N haploid samples, D SNP "
                              "density); slopes are d log(y) / d log(x)"}), flush=True)


def run_extras(sg, torch, synth, d, hap, pos, gmap, n, ws):
    """XPEHH throughput and the per-step comparisons (persistent in-order,
    plain launches) on the same GPU and matrix."""
    ex = {}
    L = sg.make_launch(sg.SCHED_IN_ORDER, warps_per_cta=4)
    o = sg.selscan_ihs(hap, n, pos, gmap, launch=L)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    o = sg.selscan_ihs(hap, n, pos, gmap, launch=L, workspace=o["_workspace"], out=o)
    b.record()
    torch.cuda.synchronize()
    cores = int((o["status"] != sg.LOCUS_MAF_FILTERED).sum())
    ex["per_step_in_order"] = {"value": cores / (a.elapsed_time(b) / 1e3), "unit": "core loci/s",
                               "ms_per_scan": a.elapsed_time(b)}
    del o
    # plain launches (one CTA per core) on the same matrix
    L = sg.make_launch(sg.SCHED_PLAIN)
    o = sg.selscan_ihs(hap, n, pos, gmap, launch=L)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    o = sg.selscan_ihs(hap, n, pos, gmap, launch=L, workspace=o["_workspace"], out=o)
    b.record()
    torch.cuda.synchronize()
    cores = int((o["status"] != sg.LOCUS_MAF_FILTERED).sum())
    ex["plain_launch"] = {"value": cores / (a.elapsed_time(b) / 1e3), "unit": "core loci/s",
                          "ms_per_scan": a.elapsed_time(b)}
    # XPEHH on the CEUYRI22-shaped pair
    x = synth.generate(synth.spec("xpehh"))
    xh, xp, xg = sg.to_device(x.rows, x.pos, x.gmap)
    o = sg.selscan_xpehh(xh, 204, 210, xp, xg)
    torch.cuda.synchronize()
    a.record()
    reps = 5
    for _ in range(reps):
        o = sg.selscan_xpehh(xh, 204, 210, xp, xg, workspace=o["_workspace"], out=o)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    # XPEHH at scale (sorted sweep): 2,500 + 2,500 haplotypes x 1,000,000 SNPs
    x1 = synth.generate(synth.spec("xpehh1m"))
    xh1, xp1, xg1 = sg.to_device(x1.rows, x1.pos, x1.gmap)
    o1 = sg.selscan_xpehh(xh1, 2500, 2500, xp1, xg1)
    for _ in range(2):                   # warm-up calls on the allocated workspace
        o1 = sg.selscan_xpehh(xh1, 2500, 2500, xp1, xg1, workspace=o1["_workspace"], out=o1)
    torch.cuda.synchronize()
    reps1 = []
    for _ in range(3):
        a1, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a1.record()
        o1 = sg.selscan_xpehh(xh1, 2500, 2500, xp1, xg1, workspace=o1["_workspace"], out=o1)
        b1.record()
        torch.cuda.synchronize()
        reps1.append(a1.elapsed_time(b1))
    sg.check(o1)
    ms1 = float(np.median(reps1))
    ex["xpehh_1m"] = {"workload": "XPEHH at scale: pop A 2,500 (200 founders, 20 planted sweeps) / "
                                  "pop B 2,500 (150 founders) haplotypes x 1,000,000 SNPs",
                      "value": x1.spec.m / (ms1 / 1e3), "unit": "core loci/s", "ms_per_scan": ms1,
                      "ok_loci": int((o1["status"] == 0).sum())}
    del o1, xh1, xp1, xg1
    ex["xpehh"] = {"workload": "XPEHH: pop A 204 / pop B 210 haplotypes x 22,147 SNPs",
                   "value": x.spec.m / (ms / 1e3), "unit": "core loci/s", "ms_per_scan": ms}
    return ex


def hap_major_bytes(rows, n):
    """uint8 [n, m] 0/1 matrix (one row per haplotype) from packed marker-major
    rows: the input layout of a phased haplotype file read haplotype by
    haplotype.  Built 64 haplotypes (one row word) at a time."""
    m = rows.shape[0]
    out = np.empty((n, m), dtype=np.uint8)
    for w in range((n + 63) // 64):
        bits = np.unpackbits(np.ascontiguousarray(rows[:, w]).view(np.uint8).reshape(m, 8), axis=1,
                             bitorder="little")                      # [m, 64]
        h = min(64, n - 64 * w)
        out[64 * w:64 * w + h] = bits[:, :h].T
    return out


def run_ingest(sg, torch, d, n, params, launch_fields, reps=3, streamed_steps=5):
    """Timed ingest of the bench's matrix: haplotype-major 0/1 bytes in pinned
    host memory -> H2D -> selscan_pack (device) -> the scan, per call; events
    split the three parts.  The packed rows equal the generator's."""
    host = torch.from_numpy(hap_major_bytes(d.rows, n)).pin_memory()       # [n, m] uint8
    h_pos = torch.from_numpy(d.pos).pin_memory()
    h_gmap = torch.from_numpy(d.gmap).pin_memory()
    dev = torch.device("cuda")
    dbytes = torch.empty(host.shape, dtype=torch.uint8, device=dev)
    dp, dg = torch.empty_like(h_pos, device=dev), torch.empty_like(h_gmap, device=dev)
    out, ws = None, None
    times = []
    for r in range(reps + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record()
        dbytes.copy_(host, non_blocking=True)
        dp.copy_(h_pos, non_blocking=True)
        dg.copy_(h_gmap, non_blocking=True)
        ev[1].record()
        rows = sg.selscan_pack(dbytes, n, hap_major=True)
        ev[2].record()
        out = sg.selscan_ihs(rows, n, dp, dg, params=params, workspace=ws, out=out,
                             launch=sg.make_launch(**launch_fields))
        ws = out["_workspace"]
        ev[3].record()
        torch.cuda.synchronize()
        if r > 0:
            times.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                          ev[2].elapsed_time(ev[3])])
    sg.check(out)
    same = bool(torch.equal(rows, torch.from_numpy(d.rows.view(np.int64)).to(dev)))
    t = np.mean(np.array(times), axis=0)
    cores = int((out["status"] != sg.LOCUS_MAF_FILTERED).sum())
    del dbytes, rows
    # the same data sets streamed: upload and packing of data set k + 1 beside scan k
    from paper_1403_6854_gb300.stream import scan_host_stream

    def stream(steps):
        last = None
        for res in scan_host_stream([(host, h_pos, h_gmap)] * steps, sg.MODE_IHS, n,
                                    params=params, launch=sg.make_launch(**launch_fields),
                                    fields=("status", "lnratio"), workspace=ws,
                                    layout="hap_major"):
            last = res
        return last

    stream(2)                                   # untimed: buffers from the caches
    torch.cuda.synchronize()
    a0 = time.perf_counter()
    last = stream(streamed_steps)
    st_s = (time.perf_counter() - a0) / streamed_steps
    assert int((last["status"].numpy() != sg.LOCUS_MAF_FILTERED).sum()) == cores
    return {"what": "haplotype-major 0/1 bytes in pinned host memory -> H2D -> selscan_pack -> "
                    "selscan_ihs, per call (CUDA events)",
            "h2d_bytes": int(host.numel() + h_pos.numel() * 8 + h_gmap.numel() * 8),
            "h2d_ms": float(t[0]), "pack_ms": float(t[1]), "scan_ms": float(t[2]),
            "total_ms": float(t.sum()), "value": cores / (float(t.sum()) / 1e3),
            "unit": "core loci/s", "pack_equals_generator": same,
            "streamed": {"what": "stream.scan_host_stream(layout='hap_major') over the same "
                                 "data set: bytes uploaded and packed beside the previous scan, "
                                 "scores read back; host clock to the last result",
                         "steps": streamed_steps, "ms_per_scan": st_s * 1e3,
                         "value": cores / st_s, "unit": "core loci/s"}}


def run_served(args, torch, synth):
    """Served mix: Poisson arrivals at `load` x the server's measured capacity;
    continuous batching vs one plain launch per scan, same arrivals."""
    from paper_1403_6854_gb300.serve import GpuExecutor, Request, run_plain, serve, summarize
    t_gen = time.perf_counter()
    reqs = []
    for i in range(args.served):
        sp = synth.served_request(i)
        d = synth.generate(sp)
        reqs.append(Request(i, sp.mode, d.rows, d.pos, d.gmap, sp.pops[0].n,
                            sp.pops[1].n if sp.mode == "xpehh" else 0))
    t_gen = time.perf_counter() - t_gen
    total_cores = sum(r.m for r in reqs)
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(0.5 * free, 64 << 30))
    ex = GpuExecutor()
    # capacity: the whole mix with every request present at t = 0
    serve(reqs[:8], ex, budget, tick_cores=args.tick_cores, realtime=False)      # warm-up
    _, _, mk = serve(reqs, ex, budget, tick_cores=args.tick_cores, policy=args.policy,
                     realtime=False)
    capacity = total_cores / mk                              # markers per second
    rate = args.load * capacity / (total_cores / len(reqs))  # requests per second
    rng = np.random.Generator(np.random.PCG64(2024))
    gaps = rng.exponential(1.0, size=len(reqs))              # unit-rate Poisson gaps

    def at_rate(rps):
        for r, a in zip(reqs, np.cumsum(gaps / rps)):
            r.arrival = float(a)
        _, lat_s, mk_s = serve(reqs, ex, budget, tick_cores=args.tick_cores, policy=args.policy)
        _, lat_p, mk_p = run_plain(reqs)
        _, lat_d, mk_d = run_plain(reqs, schedule=-1)
        return {"arrival_rate_per_s": rps,
                "continuous_batching": summarize(lat_s, total_cores, mk_s),
                "plain_launches": summarize(lat_p, total_cores, mk_p),
                "sequential_default_launches": summarize(lat_d, total_cores, mk_d)}

    out = {"requests": len(reqs), "mix": "70% iHS / 30% XPEHH, haplotypes log-U(100, 5000), "
                                         "SNPs log-U(10k, 500k), seed 1000 + i",
           "policy": args.policy, "tick_cores": args.tick_cores, "load": args.load,
           "capacity_markers_per_s": capacity, "hbm_budget_bytes": budget,
           "generation_s": t_gen}
    out.update(at_rate(rate))
    if args.overload > 0:
        out["overload"] = dict(load=args.overload, **at_rate(args.overload * rate / args.load))
    out["note"] = ("latency = results on host - arrival; core_loci_per_s counts every marker "
                   "(MAF-filtered cores included) over the makespan; capacity = the whole mix "
                   "present at t = 0 through the server; every arm sees the same arrivals; "
                   "plain_launches: one request at a time, one CTA per core; "
                   "sequential_default_launches: one request at a time with the library's "
                   "default launch (the same walk algorithms the server uses), so the gap to "
                   "continuous_batching is what batching and overlap add")
    return out


if __name__ == "__main__":
    main()
