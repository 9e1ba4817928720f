"""The N > 1 path of bench.py on CPU: world_size-2 gloo process groups (one process
per rank, 127.0.0.1 rendezvous). Replicas do no data-path collective; the only
cross-rank steps are the barrier around the timed region and the aggregation of
time (max) and work (sum), tested here without a GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, works, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t, w = bench.aggregate(times[rank], works[rank], dist, "cpu")
        out.put((rank, t, w))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    times, works = [1.25, 2.5], [1.0e9, 3.0e9]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, works, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, w in res:
        assert t == 2.5          # the slowest rank's time
        assert w == 4.0e9        # all ranks' work
    # whole-job throughput = summed work over the slowest time
    assert res[0][2] / res[0][1] == 1.6e9


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate(0.5, 7.0, None, "cpu") == (0.5, 7.0)


def test_dist_setup_reads_torchrun_environment(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("RANK", "2")
    monkeypatch.setenv("LOCAL_RANK", "2")
    assert bench.dist_setup() == (4, 2, 2)
