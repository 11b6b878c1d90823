"""Multi-rank path of bench.py on CPU with the gloo backend (world size 2): each rank owns a full
replica of the workload, and the only collective is the max-over-ranks timing reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    plan = bench.replica_plan(world, rank, (1e-2, 1e-6))
    ms = bench.max_over_ranks(10.0 * (rank + 1), world, device="cpu")
    cnt = torch.tensor([len(plan)], dtype=torch.int64)
    dist.all_reduce(cnt)
    out[rank] = (ms, int(cnt.item()), [r for r, _ in plan])
    dist.destroy_process_group()


def test_two_rank_replicas_and_timing_reduction():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        ms, total, owners = out[rank]
        assert ms == 20.0                       # the max over ranks
        assert total == 4                       # 2 solves per rank, weak scaling
        assert owners == [rank, rank]
