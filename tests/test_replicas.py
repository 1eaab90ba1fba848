"""Multi-GPU mode is independent replicas (one problem and seed per rank, no
data-path collective); the host-side aggregation of the benchmark -- slowest
rank's step time, every rank's units -- runs here as two gloo ranks on CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: step of 100 + 50 r ms over 1e9 (r + 1) units
        res = bench.replica_throughput(100.0 + 50.0 * rank, 1e9 * (rank + 1), world)
        out.put((rank, res))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    for r in range(2):
        ms_max, units, rate = got[r]
        assert ms_max == 150.0                       # the slowest rank
        assert units == 3e9                          # both ranks' units
        assert rate == pytest.approx(3e9 / 0.150)


def test_replica_aggregation_single_rank():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    ms_max, units, rate = bench.replica_throughput(200.0, 4e9, 1)
    assert (ms_max, units) == (200.0, 4e9) and rate == pytest.approx(2e10)
