"""The multi-rank path of bench.py on CPU: world_size-2 gloo ranks (one
process each, rendezvous on 127.0.0.1) agree on the slowest rank's time and
report the whole job's rate; every rank is an independent replica (no
data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from tests.conftest import ROOT  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        worst = bench.max_over_ranks(ms, world, "cpu")
        rate = bench.whole_job_rate(2.0e9, 4, world, worst)
        dist.barrier()
        out.put((rank, worst, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_the_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, worst, rate in res:
        assert worst == 15.0
        # 2 ranks x 4 steps x 2e9 units in 15 ms
        assert rate == pytest.approx(2 * 4 * 2.0e9 / 15e-3)


def test_one_rank_is_its_own_time():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_rate(3.0, 10, 1, 30.0) == pytest.approx(1000.0)
