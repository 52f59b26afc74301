"""The multi-rank paths of bench.py, run as two gloo ranks on the CPU: the
reduction (max time, summed work) and the sharding of the batched and served
workloads (independent meshes and requests, no data exchanged)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, updates = bench.reduce_over_ranks(10.0 + rank, 1000.0 * (rank + 1))
    out[rank] = (ms, updates)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (11.0, 3000.0)


def test_reduce_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(5.0, 7.0) == (5.0, 7.0)


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import meshgen
    k = 6
    mine = bench.shard(meshgen.batch_specs(k * world), rank, world)
    seeds = torch.tensor([s[3] for s in mine], dtype=torch.int64)
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    reqs = bench.shard(meshgen.serve_requests(40 * world, rate=2000.0 * world, hi=4096), rank, world)
    flag = bench.reduce_flag(rank == 0)
    out[rank] = ([g.tolist() for g in gathered], len(mine), len(reqs), reqs[-1][0], flag)
    dist.barrier()
    dist.destroy_process_group()


def test_batched_and_served_workloads_shard_across_two_gloo_ranks():
    # weak scaling: each rank gets its own k meshes (every world-th of a
    # world x k list) and its own request stream at the configured rate; no
    # mesh is on two ranks and none is missing
    import meshgen
    world, k = 2, 6
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
    all_seeds = [s[3] for s in meshgen.batch_specs(k * world)]
    gathered, n0, r0, last0, flag0 = out[0]
    assert gathered == out[1][0]
    flat = sorted(x for g in gathered for x in g)
    assert flat == sorted(all_seeds) and len(set(flat)) == k * world
    assert n0 == out[1][1] == k
    assert r0 == out[1][2] == 40
    # 40 arrivals of a 4,000/s stream split in two: about 20 ms each
    assert 0.01 < last0 < 0.04
    assert flag0 is False and out[1][4] is False
