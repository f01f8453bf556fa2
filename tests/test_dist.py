"""Host logic of the multi-GPU benchmark with two gloo ranks on the CPU: every rank gets its
own seeded batch (weak scaling, no data-path collective) and the reported time is the
maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    specs, _ = W.batch(4, seed=bench.rank_seed(rank))
    ms = 10.0 + 5.0 * rank
    out[rank] = (bench.reduce_max(ms, world, device="cpu"), [s.ni for s in specs], sum(s.ncells for s in specs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_host_logic():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    t0, ni0, c0 = out[0]
    t1, ni1, c1 = out[1]
    assert t0 == t1 == 15.0                 # both ranks report the slowest rank's time
    assert ni0 != ni1                       # independent batches per rank
    import bench
    v = bench.weak_value(c0, world, 10, t0)
    assert v == pytest.approx(c0 * 2 * 3 * 10 / 15e-3 / 1e9)
