"""Autotuner for the walk kernels' launch shape.

The shape changes how the walks run, never their results.  Samples of up to
16383 haplotypes use the sorted sweep: its cost depends on the chromosome's
length (chunking, warm-up, walks that outrun a chunk's history), so its few
candidates are timed on the whole scan.  Larger samples use the per-step
schedules (warps per CTA, on-chip group words per warp, rows per TMA window
buffer, cores per queue fetch), timed on a prefix of the scan (the first
`sample_markers` markers, a view, no copy).  Timing is CUDA events around
the walk kernels; the fastest shape is cached under a key built from the
scan's shape (mode, haplotype count bucket, marker count bucket for the
sweep, row stride), in memory and optionally in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, List, Optional

SHAPE_FIELDS = ("schedule", "warps_per_cta", "smem_entries", "window_rows", "cores_per_fetch",
                "probe_steps", "min_ctas_per_sm", "big_group_entries", "sweep_warmup",
                "sweep_stage_cores", "sweep_threads", "sweep_split_tile")

SWEEP_MAX_N = 16383
SWEEP_CANDIDATES: List[Dict] = [
    dict(schedule=1, warps_per_cta=4),          # per-step in-order, for short chromosomes
    dict(schedule=3),
    dict(schedule=3, sweep_warmup=2048),        # longer histories: fewer walks handed to
    dict(schedule=3, sweep_warmup=4096),        # the per-step second pass
    dict(schedule=3, sweep_threads=512),
]

DEFAULT_CANDIDATES: List[Dict] = [
    dict(schedule=1, warps_per_cta=8, smem_entries=512, window_rows=0, cores_per_fetch=1),
    dict(schedule=1, warps_per_cta=8, smem_entries=256, window_rows=0, cores_per_fetch=1),
    dict(schedule=1, warps_per_cta=8, smem_entries=1024, window_rows=0, cores_per_fetch=1),
    dict(schedule=1, warps_per_cta=4, smem_entries=512, window_rows=0, cores_per_fetch=1),
    dict(schedule=1, warps_per_cta=8, smem_entries=512, window_rows=4, cores_per_fetch=1),
    dict(schedule=1, warps_per_cta=8, smem_entries=512, window_rows=16, cores_per_fetch=1),
    dict(schedule=1, warps_per_cta=8, smem_entries=512, window_rows=0, cores_per_fetch=4),
    dict(schedule=1, warps_per_cta=8, smem_entries=512, window_rows=0, cores_per_fetch=16),
    dict(schedule=1, warps_per_cta=8, smem_entries=256, window_rows=4, cores_per_fetch=1,
         min_ctas_per_sm=3),
    dict(schedule=1, warps_per_cta=8, smem_entries=384, window_rows=0, cores_per_fetch=1,
         min_ctas_per_sm=3),
    dict(schedule=0, warps_per_cta=8, smem_entries=512, window_rows=0, cores_per_fetch=1,
         probe_steps=64),
]


def shape_key(mode: str, n_total: int, ld: int, m: int = 0) -> str:
    """Cache key: mode, haplotype count rounded to a power-of-two bucket, row
    stride, and (sweep) the marker count rounded to a power-of-two bucket."""
    b = 1 << max(0, math.ceil(math.log2(max(n_total, 2))))
    key = f"{mode}:n{b}:ld{ld}"
    if m > 0:
        key += f":m{1 << max(0, math.ceil(math.log2(m)))}"
    return key


class Autotuner:
    def __init__(self, cache_path: Optional[str] = None,
                 candidates: Optional[List[Dict]] = None, sample_markers: int = 65536,
                 reps: int = 2, sweep_candidates: Optional[List[Dict]] = None):
        self.cache_path = cache_path
        self.candidates = candidates or DEFAULT_CANDIDATES
        self.sweep_candidates = sweep_candidates or SWEEP_CANDIDATES
        self.sample_markers = sample_markers
        self.reps = reps
        self.cache: Dict[str, Dict] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def _save(self):
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def choose(self, key: str, timer: Callable[[Dict], float],
               candidates: Optional[List[Dict]] = None) -> Dict:
        """Best candidate for `key` (cached), timing each candidate with `timer`
        (milliseconds; the minimum over `reps` calls is kept)."""
        if key in self.cache:
            return self.cache[key]["shape"]
        results = []
        for cand in (candidates or self.candidates):
            t = min(timer(cand) for _ in range(self.reps))
            results.append((t, cand))
        best_t, best = min(results, key=lambda x: x[0])
        self.cache[key] = {"shape": best, "ms": best_t,
                           "tried": [{"shape": c, "ms": t} for t, c in results]}
        self._save()
        return best

    # ---------------------------------------------------------------- GPU
    def launch_for(self, hap, pos, gmap, mode: str, nA: int, nB: int = 0):
        """selscan_launch tuned for this scan's shape: (launch, shape dict)."""
        import torch
        import paper_1403_6854_gb300 as sg
        m, ld = hap.shape
        sweep = nA + nB <= SWEEP_MAX_N
        k = m if sweep else min(m, self.sample_markers)
        h, p, g = hap[:k], pos[:k], gmap[:k]
        ws = {}

        def timer(cand: Dict) -> float:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            e1.record()
            torch.cuda.synchronize()
            L = sg.make_launch(events=(e0, e1), **{f: cand.get(f, 0) for f in SHAPE_FIELDS})
            key = tuple(sorted(cand.items()))
            if mode == "ihs":
                o = sg.selscan_ihs(h, nA, p, g, launch=L, workspace=ws.get(key))
            else:
                o = sg.selscan_xpehh(h, nA, nB, p, g, launch=L, workspace=ws.get(key))
            torch.cuda.synchronize()
            ws[key] = o["_workspace"]
            return e0.elapsed_time(e1)

        if sweep:
            shape = self.choose(shape_key(mode, nA + nB, ld, m), timer, self.sweep_candidates)
        else:
            shape = self.choose(shape_key(mode, nA + nB, ld), timer)
        return sg.make_launch(**{f: shape.get(f, 0) for f in SHAPE_FIELDS}), shape
