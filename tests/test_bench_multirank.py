"""The multi-GPU path of the benchmark is replicas only: each rank times its own copy of the
workload and the job time is the slowest rank's.  Its host logic runs here with two gloo
ranks on the CPU (no GPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = 100.0 + 50.0 * rank                  # the second rank is slower
    t = bench.job_time_ms(local, dist, "cpu")
    q.put((rank, t, bench.job_value(world, 1000, 10, t)))
    dist.destroy_process_group()


def test_job_time_is_slowest_rank_and_value_counts_all_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 150.0                                  # max over ranks
        assert abs(v - 2 * 1000 * 10 / 0.150 / 1e6) < 1e-12
