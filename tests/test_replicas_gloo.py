"""Multi-rank host logic of the benchmark on CPU (world size 2, gloo): the
case does not shard, so N GPUs run N independent replicas and the job's
throughput is N x steps over the slowest rank's time."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.replica_throughput(ms[rank], 5, world, "cpu")))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ms = [400.0, 500.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        t_max, value = out[r]
        assert t_max == 500.0
        assert abs(value - 2 * 5 / 0.5) < 1e-12      # 10 replica-steps in 0.5 s


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(250.0, 5, 1) == (250.0, 20.0)
