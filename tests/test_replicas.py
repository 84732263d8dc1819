"""The multi-GPU path of bench.py is replicas only: each rank runs its own copy of the
workload, the process group carries only the barrier and the max-over-ranks time, and the
reported value is the units of all ranks over the slowest rank's time.  Checked here with
world_size-2 gloo process groups on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    got_ws, got_rank, local = bench.dist_setup()
    assert (got_ws, got_rank, local) == (ws, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(ws)
    # rank r "took" 1 + r seconds for 10 units of work
    t_max = bench.allreduce_max(ws, 1.0 + rank, local)
    out[rank] = (t_max, bench.whole_job_rate(ws, 10.0, t_max))
    bench.barrier(ws)
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_replicas_take_the_slowest_rank(ws):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == list(range(ws))
    for r in range(ws):
        t_max, value = res[r]
        assert t_max == float(ws)  # the slowest rank's time, on every rank
        assert value == ws * 10.0 / ws  # all ranks' units over that time


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_setup() == (1, 0, 0)
        assert bench.allreduce_max(1, 3.5, 0) == 3.5
        assert bench.whole_job_rate(1, 7.0, 2.0) == 3.5
    finally:
        os.environ.update(env)
