"""Replica path of bench.py on CPU: two gloo ranks draw disjoint noise streams and
report the slowest rank's time (no data-path collective exists)."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = torch.tensor([bench.rank_seed(s, rank) for s in range(-3, 8)], dtype=torch.int64)
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    t = bench.max_over_ranks(10.0 + rank, world, device="cpu")
    q.put((rank, [g.tolist() for g in gathered], t))
    dist.destroy_process_group()


def test_two_replicas_disjoint_noise_and_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t in res:
        assert t == pytest.approx(11.0)
        flat = [s for g in gathered for s in g]
        assert len(set(flat)) == len(flat)
