"""Multi-GPU runs are independent replicas (the path does not shard; no
collective on the data path).  bench.py's only cross-rank step is the
max-over-ranks time; check it with two gloo processes on the CPU."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, dist)          # rank 1 is slower
    v = bench.replica_value(1000.0, t, world)
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in out:
        assert t == 2.5                 # both ranks see the slowest time
        assert v == 2 * 1000.0 / 2.5    # whole-job throughput of both replicas


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.replica_value(10.0, 2.0, 1) == 5.0
