"""The bench's multi-rank arithmetic on CPU: two gloo ranks, as torchrun
launches them (one process each).  Every rank gets the slowest rank's time,
and the whole-job throughput counts every rank's units over that time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        seconds = [0.5, 2.0][rank]                       # rank 1 is the slow one
        t = bench.max_over_ranks(seconds)
        v = bench.job_throughput(10, world, t)
        tdist.barrier()
        out.put((rank, t, v))
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_with_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, t, v in res:
        assert t == 2.0                                  # the slowest rank's time on both
        assert v == pytest.approx(10 * 2 / 2.0)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.job_throughput(16, 1, 0.5) == 32.0
