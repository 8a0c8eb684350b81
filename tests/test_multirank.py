"""Multi-process (world_size 2, gloo, CPU) checks of the N > 1 path of bench.py: every rank runs
an independent replica of the workload, the job's time is the slowest rank's (all-reduce MAX),
the value counts the units of all ranks, only rank 0 prints, and the reference arm runs on
rank 0 alone."""
import io
import os
import socket
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        ms = [3.0, 5.0][rank]                      # the second rank is slower
        t = bench.max_over_ranks(ms)
        v = bench.whole_job_value(1e9, world, t)
        # the reference arm: rank 0 alone runs and prints one JSON line
        buf = io.StringIO()
        args = type("A", (), {"warmup": 0, "steps": 1, "gpus": world, "workload": "cfd128_b16_f4_fp64"})()
        spec = dict(bench.WORKLOADS["cfd128_b16_f4_fp64"])
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(args, spec, rank)
        q.put((rank, t, v, buf.getvalue()))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_reduce_to_the_slowest_and_count_all_units():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get() for _ in range(world))
    for rank, t, v, out in res:
        assert t == 5.0                              # max over ranks on every rank
        assert abs(v - 1e9 * 2 / 5e-3 / 1e9) < 1e-9  # units of both ranks over the slowest time
        if rank != 0:
            assert out == ""                         # non-zero ranks of the reference arm do no work


def test_single_process_is_the_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.25) == 4.25
    assert bench.whole_job_value(2e9, 1, 1000.0) == 2.0
