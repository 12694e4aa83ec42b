"""The multi-rank path of bench.py on the CPU: two gloo ranks (127.0.0.1), each with its own
step time; both must see the slowest rank's time and the same whole-job value; the reference
arm prints only on rank 0."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 100.0 + 50.0 * rank                          # rank 1 is slower
    t = bench.max_over_ranks(mine, world, torch.device("cpu"))
    v = bench.job_value(world, 64, 5, t)
    # the reference arm: rank 0 prints its line, the other ranks return without work
    buf = io.StringIO()
    args = bench.parse([])
    if rank != 0:
        with redirect_stdout(buf):
            bench.reference_main(args)
    q.put((rank, t, v, buf.getvalue()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_max_time_and_value():
    world = 2
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    assert out[0][2] == out[1][2] == pytest.approx(2 * 64 * 5 / 0.150)
    assert out[1][3] == ""          # rank 1 printed nothing
