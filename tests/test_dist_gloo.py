"""The N > 1 path of bench.py on CPU: two gloo ranks, each advancing its
own replicas (no collective on the data path), timing reduced by max."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = {}
    for name in ("large", "batched", "uneven"):
        seeds[name] = [r.seed for r in bench.rank_requests(bench.WORKLOADS[name], rank)]
    t = bench.max_over_ranks(1.0 + rank)
    out.put((rank, seeds, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_run_disjoint_replicas_and_reduce_time_by_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (s, t)) for r, s, t in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for name in ("large", "batched", "uneven"):
        a, b = set(res[0][0][name]), set(res[1][0][name])
        assert len(a) == len(res[0][0][name]) and not (a & b)   # disjoint replicas
        assert len(res[0][0][name]) == len(res[1][0][name])      # same work per rank (weak)
    assert res[0][1] == res[1][1] == 2.0
