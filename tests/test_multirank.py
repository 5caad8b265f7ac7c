"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica; the job time is the maximum over ranks and the work the sum.  The
solver path itself has no collective (runs are independent replicas)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    t = bench.reduce_max(1.5 + rank, w)      # rank-dependent time
    u = bench.reduce_sum(100.0 * (rank + 1), w)
    bench.barrier(w)
    out[rank] = (r, w, lr, t, u)
    dist.destroy_process_group()


def test_two_rank_reductions():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        r, w, lr, t, u = out[rank]
        assert (r, w, lr) == (rank, world, rank)
        assert t == 2.5 and u == 300.0


def test_reference_arm_other_ranks_exit(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""
