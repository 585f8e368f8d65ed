"""Multi-rank host logic on CPU (gloo, world size 2): replica seeding and the
max-over-ranks throughput reduction used by bench.py under torchrun."""
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
    import torch.distributed as dist
    from paper_1707_02162_gb300.replicas import aggregate_throughput, replica_seed
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [2.0, 5.0][rank]                      # rank 1 is the slow one
    value, slowest = aggregate_throughput(1000.0, local)
    out[rank] = (value, slowest, replica_seed(1, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_same_aggregate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    v0, s0, seed0 = out[0]
    v1, s1, seed1 = out[1]
    assert s0 == s1 == 5.0                        # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 1000.0 / 5.0)
    assert seed0 == 1 and seed1 != seed0          # distinct replica batches


def test_single_process_falls_back_to_local_numbers():
    from paper_1707_02162_gb300.replicas import aggregate_throughput
    assert aggregate_throughput(10.0, 2.0) == (5.0, 2.0)
