"""The multi-GPU form of the benchmark is replicas only: every rank solves its own copy of the workload
and the ranks exchange only the step time (its maximum). Checked here with world_size-2 gloo process
groups on the CPU (no GPU involved)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, q):
    import sys
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(values[rank], dist, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("values", [[3.5, 1.25], [2.0, 9.0]])
def test_step_time_is_the_maximum_over_two_ranks(values):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out == {0: max(values), 1: max(values)}


def test_single_process_keeps_its_own_time():
    import bench
    assert bench.max_over_ranks(4.25) == 4.25


def _straggler(rank, world, port, q):
    import sys
    import time
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t0 = time.perf_counter()
        time.sleep(0.05 if rank == 0 else 0.2)  # rank 1 is the slow replica
        dt = time.perf_counter() - t0
        q.put((rank, bench.max_over_ranks(dt, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_a_slow_replica_sets_the_step_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_straggler, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] and out[0] >= 0.2
