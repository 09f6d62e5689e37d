"""The multi-GPU path of bench.py is replicas: each rank runs its own queries, and the job's time is the
slowest rank's. Two gloo ranks on the CPU check the max-over-ranks rate and the disjoint query ids."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed 10 queries in 100 * (r + 1) ms
        rate, ms = bench.whole_job_rate(100.0 * (rank + 1), 10, world)
        out.put((rank, rate, ms, [bench.replica_query_id(rank, i) for i in range(100)]))
    finally:
        dist.destroy_process_group()


def test_replica_rate_is_the_slowest_rank_and_ids_are_disjoint():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms, _ in res:
        assert ms == 200.0  # the slower rank's time
        assert abs(rate - 2 * 10 / 0.2) < 1e-9  # 20 queries in 0.2 s
    assert not set(res[0][3]) & set(res[1][3])


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms = bench.whole_job_rate(500.0, 10, 1)
    assert ms == 500.0 and abs(rate - 20.0) < 1e-12
