"""One scan split over ranks (paper Section 3: sites split, data set shared),
on CPU: the partition of the cores, the all-gather of the per-core results
and the two all-reduces of the per-bin sums that standardisation (Eq. 7,
Eq. 11) needs, run by two and three gloo ranks.  The per-rank compute comes
from the CPU oracle (scan of a core range) and numpy (bin sums), so the host
logic of ``paper_1403_6854_gb300.shard`` is checked without a GPU against a
single-rank oracle run."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1403_6854_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleOps:
    """The four per-rank calls of a sharded scan on the CPU: the oracle for a
    core range, numpy for the per-bin sums (the bins of Eq. 7: n1 / n in nbins
    equal bins, decided in integers; one bin for Eq. 11)."""

    def __init__(self, data):
        self.d = data

    def scan_range(self, mode, hap, nA, nB, pos, gmap, k0, k1):
        import oracle
        cores = np.arange(k0, k1)
        if mode == "ihs":
            r = oracle.ihs(self.d.rows, nA, self.d.pos, self.d.gmap, cores=cores, threads=2)
        else:
            r = oracle.xpehh(self.d.rows, nA, nB, self.d.pos, self.d.gmap, cores=cores, threads=2)
        return {k: torch.from_numpy(np.ascontiguousarray(v).view(np.int64) if v.dtype == np.uint64
                                    else np.ascontiguousarray(v)) for k, v in r.items()}

    @staticmethod
    def _bins(n1, n, nbins):
        n1 = n1.numpy().astype(np.int64)
        return np.zeros(n1.size, np.int64) if nbins == 1 else np.minimum(nbins - 1, n1 * nbins // n)

    def bin_sums(self, score, status, n1, n, nbins, pass_, mean=None):
        b = self._bins(n1, n, nbins)
        ok = status.numpy() == 0
        x = score.numpy()
        cnt = np.bincount(b[ok], minlength=nbins).astype(np.int64)
        if pass_ == 0:
            s = np.bincount(b[ok], weights=x[ok], minlength=nbins)
        else:
            d = x[ok] - mean.numpy()[b[ok]]
            s = np.bincount(b[ok], weights=d * d, minlength=nbins)
        return torch.from_numpy(cnt), torch.from_numpy(s.astype(np.float64))

    def finish(self, nbins, pass_, count, total):
        c = count.numpy().astype(np.float64)
        t = total.numpy()
        with np.errstate(invalid="ignore", divide="ignore"):
            if pass_ == 0:
                return torch.from_numpy(np.where(c > 0, t / np.maximum(c, 1), np.nan))
            return torch.from_numpy(np.where(c > 1, np.sqrt(t / np.maximum(c - 1, 1)), np.nan))

    def apply(self, score, status, n1, n, nbins, count, mean, sd):
        b = self._bins(n1, n, nbins)
        ok = status.numpy() == 0
        c, mu, s = count.numpy()[b], mean.numpy()[b], sd.numpy()[b]
        good = ok & (c >= 2) & (s > 0)
        out = np.full(score.numel(), np.nan)
        out[good] = (score.numpy()[good] - mu[good]) / s[good]
        return torch.from_numpy(out)


def _worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synth
        d = synth.generate(synth.spec("plain" if mode == "ihs" else "xpehh"))
        nA = d.spec.pops[0].n
        nB = d.spec.pops[1].n if mode == "xpehh" else 0
        m = d.spec.m if mode == "ihs" else 3000          # XPEHH: the first 3,000 markers
        if mode == "xpehh":
            d = synth.ScanData(d.spec, d.rows[:m], d.pos[:m], d.gmap[:m])
        ops = OracleOps(d)
        ranges = shard.partition(m, world)
        (k0, k1), local = shard.scan(ops, mode, None, nA, nB, torch.from_numpy(d.pos), None, rank,
                                     world)
        assert (k0, k1) == ranges[rank]
        full = shard.gather(local, ranges)
        nbins = 10 if mode == "ihs" else 1
        z, count, mean, sd = shard.normalize(ops, local["lnratio"], local["status"], local["n1"],
                                             nA + nB, nbins)
        zs = [torch.empty(max(b - a for a, b in ranges), dtype=torch.float64) for _ in ranges]
        pad = torch.full((zs[0].numel(),), float("nan"), dtype=torch.float64)
        pad[:z.numel()] = z
        dist.all_gather(zs, pad)
        zfull = torch.cat([t[:b - a] for t, (a, b) in zip(zs, ranges)])
        if rank == 0:
            q.put({"full": {k: v.numpy() for k, v in full.items()}, "z": zfull.numpy(),
                   "count": count.numpy(), "mean": mean.numpy(), "sd": sd.numpy(),
                   "ranges": ranges})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(world, mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = q.get(timeout=200)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world,mode", [(2, "ihs"), (3, "ihs"), (2, "xpehh")])
def test_sharded_scan_gather_and_normalisation(world, mode):
    import oracle
    import synth
    res = _run(world, mode)
    d = synth.generate(synth.spec("plain" if mode == "ihs" else "xpehh"))
    if mode == "ihs":
        ref = oracle.ihs(d.rows, 100, d.pos, d.gmap)
        n, nbins = 100, 10
    else:
        m = 3000
        ref = oracle.xpehh(d.rows[:m], 204, 210, d.pos[:m], d.gmap[:m])
        n, nbins = 414, 1
    got = res["full"]
    # the gathered ranges are the single-rank scan, field by field
    for f, v in ref.items():
        g = got[f].view(np.uint64) if v.dtype == np.uint64 else got[f]
        assert np.array_equal(g, v, equal_nan=v.dtype.kind == "f"), f
    # the bin statistics summed over ranks equal those of one rank's whole scan
    want = oracle.normalize(ref["lnratio"], ref["status"], ref["n1"], n, nbins)
    assert np.array_equal(res["count"], want["count"])
    ok = ~np.isnan(want["mean"])
    np.testing.assert_allclose(res["mean"][ok], want["mean"][ok], rtol=1e-12, atol=1e-15)
    ok = ~np.isnan(want["sd"])
    np.testing.assert_allclose(res["sd"][ok], want["sd"][ok], rtol=1e-12)
    assert np.array_equal(np.isnan(res["z"]), np.isnan(want["score"]))
    ok = ~np.isnan(want["score"])
    np.testing.assert_allclose(res["z"][ok], want["score"][ok], rtol=0, atol=1e-9)


def test_partition_ranges():
    assert shard.partition(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert shard.partition(5, 5) == [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)]
    assert shard.partition(7, 1) == [(0, 7)]
    # weighted: the cut sits where the running load first reaches half of it
    w = np.r_[np.full(50, 4.0), np.ones(50)]
    r = shard.partition(100, 2, w)
    assert r == [(0, 32), (32, 100)]          # loads 128 and 122 of 250
    loads = [w[a:b].sum() for a, b in shard.partition(100, 4, w)]
    assert max(loads) - min(loads) <= 4.0
    # every range non-empty even with zero weights at the ends
    w = np.zeros(10)
    w[5] = 1.0
    r = shard.partition(10, 4, w)
    assert all(b > a for a, b in r) and r[0][0] == 0 and r[-1][1] == 10
    for a, b in zip(r, r[1:]):
        assert a[1] == b[0]
    with pytest.raises(ValueError):
        shard.partition(3, 4)
    with pytest.raises(ValueError):
        shard.partition(5, 2, np.ones(4))
