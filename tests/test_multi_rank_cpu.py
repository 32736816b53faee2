"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

bench.py runs one rank per GPU (replicas: no data-path collective). What the ranks share is
the barrier, the slowest-rank time and the whole-job throughput, and only rank 0 prints; the
reference arm runs on rank 0 alone. Those host-side pieces are checked here with the gloo
backend, as the N > 1 launch runs them with NCCL."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [3.0, 7.5][rank]                   # this rank's timed region, ms
        mx = bench.max_over_ranks(local)
        value = bench.job_rate(1000.0, world, mx)  # 1000 units per rank
        dist.barrier()
        # the reference arm runs and prints on rank 0 only
        buf = io.StringIO()
        args = type("A", (), {"workload": "none-such", "gpus": world, "steps": 1, "warmup": 0})()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(args)
        q.put((rank, mx, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time_and_rank0_reports():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, value, printed in out:
        assert mx == 7.5                            # every rank sees the slowest rank
        assert value == pytest.approx(2 * 1000.0 / 7.5e-3)
        if rank != 0:
            assert printed == ""                    # only rank 0 prints


def test_single_process_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.25) == 4.25
    assert bench.job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
