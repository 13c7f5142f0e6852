"""The N-GPU bench path on CPU: two gloo ranks, each with its own chromosome
(weak scaling), combine into whole-job numbers (max time, summed core loci)
with no data-path collective."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    spec = bench.rank_spec("plain", rank)
    ms = 10.0 * (rank + 1)
    cores = 1000 + rank
    got = bench.aggregate(ms, cores, world, torch.device("cpu"))
    dist.barrier()
    q.put((rank, spec.seed, spec.m, spec.n, got))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=100) for _ in ps)
    for p in ps:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, s0, m0, n0, g0), (r1, s1, m1, n1, g1) = res
    assert (s0, s1) == (0, 1)                    # one chromosome per rank
    assert (m0, n0) == (m1, n1)                  # same shape: weak scaling
    assert g0 == g1 == (20.0, 2001.0)            # slowest rank, all core loci


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(12.5, 77, 1, None) == (12.5, 77.0)
