"""The multi-rank path of bench.py on the CPU (no GPU): two gloo ranks, as
torchrun launches them on 127.0.0.1, reduce their timings with the bench's
own max_over_ranks (the slowest rank sets the job's time), and job_value
turns one rank's flops into the whole job's throughput (replicas, weak
scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as td
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        td.barrier()
        # rank 0 is slower in the first quantity, rank 1 in the second
        out = bench.max_over_ranks([10.0 - 3.0 * rank, 2.0 + 5.0 * rank], td, "cpu")
        q.put((rank, out))
        td.barrier()
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == [10.0, 7.0]


def test_job_value_counts_every_replica():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    # two replicas of 3e12 flops each, slowest rank 2 s: 3 TFLOP/s
    assert bench.job_value(2, 3e12, 2.0) == pytest.approx(3.0)
    assert bench.job_value(1, 3e12, 2.0) == pytest.approx(1.5)
