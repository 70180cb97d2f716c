"""The bench's multi-process path on the CPU.  Under torchrun every rank runs
its own independently seeded grid (replicas: groups are independent until
the final sum, so nothing is exchanged on the data path); the line reports
the slowest rank's time and the whole job's rate.  Here two ranks over gloo
take that reduction and read their ranks from the launcher's environment."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_env()
        ms = bench.max_over_ranks(2.0 + 1.5 * rank, dist, "cpu")
        q.put((rank, w, r, loc, ms, bench.job_rate(1000, w, ms / 1e3)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_the_whole_job():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1]
    for rank, w, r, loc, ms, rate in res:
        assert (w, r, loc) == (2, rank, rank)
        assert ms == 3.5                        # the slower rank's time, on both
        assert rate == pytest.approx(2 * 1000 / 3.5e-3)


def test_one_process_keeps_its_own_time():
    import bench
    assert bench.max_over_ranks(4.25, None, "cpu") == 4.25
    assert bench.job_rate(10, 1, 2.0) == 5.0
    cfg = bench.workload_config(type("P", (), dict(n=4, n_groups=2, n_out=11, n_src=3))(), 2)
    assert cfg["parallelism"] == "replicas"
