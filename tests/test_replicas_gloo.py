"""The N > 1 host logic of bench.py on CPU: replicas with a gloo process group, world size 2.  Each
rank reports its own step time; the job time is the maximum over ranks and the whole-job throughput
is the sum of all ranks' units over that time (no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, vals = bench.aggregate_ranks([10.0 + rank, 20.0 - rank], [1e6, 2e6], world, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, vals))


def test_aggregate_ranks_max_time_sum_units():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, vals in out:
        assert ms == [11.0, 20.0]                       # the slowest rank decides each time
        assert vals == pytest.approx([2 * 1e6 / 11e-3, 2 * 2e6 / 20e-3])


def test_aggregate_single_rank_is_identity():
    import bench
    ms, vals = bench.aggregate_ranks([5.0], [1e6], 1, None)
    assert ms == [5.0] and vals == pytest.approx([1e6 / 5e-3])
