"""Host logic of the multi-GPU bench path, run as two gloo ranks on the CPU.

The path shards into independent instances (one per rank, no exchange of spins): the ranks
must simulate different instances, agree on the slowest rank's time, and report the whole-job
throughput over all ranks.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    ms = bench.max_over_ranks(10.0 + rank)            # rank 1 is the slowest
    value = bench.job_value(1000, 5, ws, ms)
    rp, col, _ = bench.instance(rank, n=2000)
    out[rank] = (ws, r, ms, value, bench.graph_seed(rank), int(col.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_time_and_shard_instances():
    world = 2
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    a, b = out[0], out[1]
    assert a[0] == b[0] == 2 and (a[1], b[1]) == (0, 1)
    assert a[2] == b[2] == 11.0                       # max over ranks
    assert a[3] == b[3] == pytest.approx(2 * 1000 * 5 / (11.0 * 1e6))
    assert a[4] != b[4] and a[5] != b[5]              # independent instances per rank
