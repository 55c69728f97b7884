"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
solves its own batch (different seeds, no data exchanged) and the job's time
is the slowest rank's, its verified count the sum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank
    local_ok = 1000 + rank
    ms, ok = bench.aggregate_ranks(local_ms, local_ok, dist, "cpu")
    q.put((rank, ms, ok, bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    for rank, ms, ok, seed in res:
        assert ms == 150.0 and ok == 2001.0
    assert res[0][3] != res[1][3]


def test_rank_batches_differ():
    import bench
    from paper_2007_11208_gb300 import synth
    a = synth.batch_specs(64, bench.rank_seed(0))
    b = synth.batch_specs(64, bench.rank_seed(1))
    assert a != b
