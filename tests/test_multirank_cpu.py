"""The multi-GPU path of bench.py on the host: two processes joined by a gloo
process group (127.0.0.1), as torchrun launches them.  Each rank works on its own
data; the group carries only barriers and the timing reduction, which must give
every rank the slowest rank's times, from which the whole job's rate follows."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.ranks_from_env()
    dist = bench.init_ranks(w, "gloo")
    try:
        dist.barrier()
        # rank 0 is slower on the first timing, rank 1 on the second
        got = bench.max_over_ranks([10.0 * (2 - rank), 5.0 + 3.0 * rank], dist, "cpu")
        dist.barrier()
        q.put((r, w, local, got, bench.whole_job_rate(w, 240, got[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_their_timings_to_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, (r, w, local, got, rate) in enumerate(out):
        assert (r, w, local) == (rank, 2, rank)
        assert got == [20.0, 8.0]                       # each timing's maximum over the two ranks
        assert rate == pytest.approx(2 * 240 / 0.020)   # all ranks' units over the slowest rank's time


def test_one_process_needs_no_group():
    import bench
    assert bench.init_ranks(1, "gloo") is None
    assert bench.max_over_ranks([3.0, 4.0], None, "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(1, 100, 50.0) == pytest.approx(2000.0)
