"""The N > 1 path of bench.py runs independent replicas; its only collectives are a barrier and
a max-reduction of the step time.  Exercise that logic with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 1.0 + rank                      # rank 1 is the slow one
    dist.barrier()
    t = bench.max_over_ranks(t_local, world, torch.device("cpu"))
    ws, r, _ = bench.dist_info()
    out[rank] = (t, ws, r)
    dist.destroy_process_group()


def test_two_rank_max_over_ranks_on_gloo():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (2.0, 2, 0) and out[1] == (2.0, 2, 1)
