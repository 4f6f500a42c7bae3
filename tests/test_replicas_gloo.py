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


def _store_worker(rank, world, port, q, tmpdir):
    """Each replica keeps its own noise vectors' loops in a base-2 store; rank 0 combines the
    stores after a barrier (files instead of a data-path collective)."""
    import numpy as np
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import paper_1309_2256_gb300 as dl

    def sources(r):
        return np.random.default_rng(bench.rank_seed(5, r)).normal(size=(11, 20))

    st = dl.dl_store_open(os.path.join(tmpdir, f"rank{rank}"), 20)
    dl.dl_store_add(st, sources(rank))
    dl.dl_store_close(st)
    dist.barrier()
    worst = 0.0
    try:
        if rank == 0:
            # 11 sources per replica: complete files 1, 2, 4 (sets of up to 7), 4 in .partial
            for n in range(1, 8):
                got = sum(dl.dl_store_load(os.path.join(tmpdir, f"rank{r}"), 20, n) for r in range(world))
                ref = sum(sources(r)[dl.dl_store_sources(n)].sum(0) for r in range(world))
                worst = max(worst, float(np.abs(got - ref).max()))
    except Exception as e:  # report instead of leaving the queue empty
        worst = repr(e)
    q.put((rank, worst))
    dist.destroy_process_group()


def test_replica_loop_stores_combine(tmp_path):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_store_worker, args=(r, world, port, q, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert isinstance(res[0], float) and res[0] < 1e-13, res[0]
    assert sorted(os.listdir(tmp_path)) == sorted(f"rank{r}.{s}" for r in range(world)
                                                  for s in ("1", "2", "4", "partial"))
