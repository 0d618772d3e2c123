"""The N > 1 path of the bench (replicas, no data-path collective): two gloo
ranks on CPU check the max-over-ranks timing, the whole-job throughput and
that the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + 5.0 * rank, world)            # per-rank times 10, 15 ms
        v = bench.replica_throughput(100, 4, world, t)
        # the reference arm: only rank 0 works (the others return at once)
        import io
        import contextlib
        buf = io.StringIO()
        args = bench.parse(["--impl", "reference", "--gpus", str(world), "--cpu-seconds", "0"]) if rank else None
        if rank:
            with contextlib.redirect_stdout(buf):
                bench.run_reference(args)
        q.put((rank, t, v, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, printed in out:
        assert t == 15.0                                              # the slowest rank's time on every rank
        assert v == pytest.approx(100 * 4 * 2 / 0.015)                # all ranks' iterations / that time
        if rank:
            assert printed == ""                                      # non-zero ranks print nothing
