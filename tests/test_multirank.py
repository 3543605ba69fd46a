"""The N > 1 path of bench.py on CPU: two gloo ranks (independent replicas,
no collective on the data path) agree on the slowest rank's time and the
whole-job rate, and draw different node sets (rank 0's is the one-GPU set)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 1.0 + rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, world, "cpu")
        rate = bench.whole_job_rate(world, bench.N_NODES, ms)
        _, nodes = bench.build_inputs(rank)
        out[rank] = (ms, rate, nodes[:50])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    import bench
    assert res[0][0] == res[1][0] == 2.0
    assert res[0][1] == res[1][1] == world * bench.N_NODES / 0.002
    assert res[0][2] != res[1][2]
    assert res[0][2] == bench.build_inputs(0)[1][:50]
