"""Host-side logic of bench.py's multi-GPU replicas path on CPU: two gloo
ranks with different step times and sizes; the job value uses the slowest
rank's time and the sum of all ranks' dofs."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, dofs, value = bench.aggregate(10.0 + 5.0 * rank, 1000 * (rank + 1),
                                      dist)
    q.put((rank, ms, dofs, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, dofs, value in out:
        assert ms == 15.0 and dofs == 3000.0
        assert abs(value - 3000.0 / 15e-3) < 1e-6


def test_single_process_aggregate():
    import bench
    ms, dofs, value = bench.aggregate(20.0, 500)
    assert (ms, dofs) == (20.0, 500) and abs(value - 25000.0) < 1e-9
