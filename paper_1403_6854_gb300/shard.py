"""One scan split over several GPUs, one process per GPU.

The sites of a scan are independent and every walk may read the whole data
set (the paper's program splits the sites of one data set over threads that
all see it, Section 3), so the GPU form is:

* every rank holds the whole packed matrix, positions and map (a 1M-marker,
  5,000-haplotype chromosome is 632 MB);
* the cores are split into contiguous ranges of near-equal predicted work
  (``partition``), and each rank scans its range with ``selscan_ihs_range`` /
  ``selscan_xpehh_range``: no data moves while the walks run, and each core's
  results equal those of the whole scan bit for bit;
* the per-core results are gathered (``gather``: an all-gather of the
  structure-of-arrays outputs);
* standardisation (Eq. 7 per derived-frequency bin for iHS, Eq. 11 genome
  wide for XPEHH) needs each bin's mean and standard deviation over all
  ranks: two all-reduces of per-bin sums (``normalize``), the count and sum
  first, then the sum of squared deviations about the mean.

The collective calls go through ``torch.distributed`` (NCCL on GPUs, gloo on
CPU).  The per-rank compute is reached through an ``ops`` object, so that the
host logic (partition, gather, the order of the all-reduces) runs the same
with the library's kernels (``DeviceOps``) and, in tests, with any other
implementation of the same four calls.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

Range = Tuple[int, int]


def partition(m: int, world: int, weights: Optional[Sequence[float]] = None) -> List[Range]:
    """Split cores [0, m) into `world` contiguous ranges of near-equal
    predicted work.  `weights[k]` is core k's predicted cost (default: one unit
    per marker, the cost model of the sorted sweep, whose per-marker sort is
    the same for every marker).  Every range is non-empty when world <= m; the
    boundaries are where the running total crosses r / world of the sum."""
    if world < 1 or m < 1:
        raise ValueError("partition: world >= 1 and m >= 1")
    if world > m:
        raise ValueError("partition: more ranks than cores")
    if weights is None:
        cuts = [(m * r) // world for r in range(world + 1)]
    else:
        w = np.asarray(weights, dtype=np.float64)
        if w.shape != (m,) or np.any(w < 0):
            raise ValueError("partition: weights must be m non-negative values")
        cum = np.concatenate([[0.0], np.cumsum(w)])
        total = cum[-1]
        cuts = [0]
        for r in range(1, world):
            k = int(np.searchsorted(cum, total * r / world, side="left"))
            # keep every range non-empty
            k = max(k, cuts[-1] + 1)
            k = min(k, m - (world - r))
            cuts.append(k)
        cuts.append(m)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


class DeviceOps:
    """The per-rank calls of a sharded scan, on this rank's GPU through the
    library (``paper_1403_6854_gb300``)."""

    def __init__(self, sg, params=None, launch=None):
        self.sg, self.params, self.launch = sg, params, launch

    def scan_range(self, mode: str, hap, nA: int, nB: int, pos, gmap, k0: int, k1: int):
        if mode == "ihs":
            out = self.sg.selscan_ihs_range(hap, nA, pos, gmap, k0, k1, params=self.params,
                                            launch=self.launch)
        else:
            out = self.sg.selscan_xpehh_range(hap, nA, nB, pos, gmap, k0, k1, params=self.params,
                                              launch=self.launch)
        self.sg.check(out)
        return {k: v for k, v in out.items() if not k.startswith("_") and k != "error"}

    def bin_sums(self, score, status, n1, n: int, nbins: int, pass_: int, mean=None):
        return self.sg.selscan_normalize_bin_sums(score, status, n1, n, nbins, pass_, mean)

    def finish(self, nbins: int, pass_: int, count, total):
        return self.sg.selscan_normalize_finish(nbins, pass_, count, total)

    def apply(self, score, status, n1, n: int, nbins: int, count, mean, sd):
        return self.sg.selscan_normalize_apply(score, status, n1, n, nbins, count, mean, sd)


def scan(ops, mode: str, hap, nA: int, nB: int, pos, gmap, rank: int, world: int,
         weights=None) -> Tuple[Range, Dict[str, torch.Tensor]]:
    """This rank's share of one scan: its core range and its outputs."""
    m = int(pos.shape[0])
    k0, k1 = partition(m, world, weights)[rank]
    return (k0, k1), ops.scan_range(mode, hap, nA, nB, pos, gmap, k0, k1)


def gather(local: Dict[str, torch.Tensor], ranges: Sequence[Range], group=None
           ) -> Dict[str, torch.Tensor]:
    """All-gather of every rank's per-core outputs into whole-scan arrays, in
    core order (each rank passes its own range's outputs)."""
    import torch.distributed as dist
    world = len(ranges)
    longest = max(k1 - k0 for k0, k1 in ranges)
    out = {}
    for f in sorted(local):
        t = local[f]
        pad = torch.zeros((longest,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[:t.shape[0]] = t
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        out[f] = torch.cat([p[:k1 - k0] for p, (k0, k1) in zip(parts, ranges)])
    return out


def normalize(ops, score, status, n1, n: int, nbins: int, group=None):
    """Standardised scores of this rank's cores with the bin statistics of all
    ranks (Eq. 7 / Eq. 11): returns (scores, count, mean, sd).  One all-reduce
    of (count, sum) per bin, then one of the sums of squared deviations."""
    import torch.distributed as dist
    count, total = ops.bin_sums(score, status, n1, n, nbins, 0)
    dist.all_reduce(count, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
    mean = ops.finish(nbins, 0, count, total)
    _, sq = ops.bin_sums(score, status, n1, n, nbins, 1, mean)
    dist.all_reduce(sq, op=dist.ReduceOp.SUM, group=group)
    sd = ops.finish(nbins, 1, count, sq)
    return ops.apply(score, status, n1, n, nbins, count, mean, sd), count, mean, sd
