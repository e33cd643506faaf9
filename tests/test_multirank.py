"""The N > 1 path of the benchmark on CPU (gloo, world size 2).

Fields are sharded across ranks with no data exchange; the ranks meet only
for the barrier and the max-over-ranks reduction of the elapsed time, and the
job throughput counts the bytes of every rank."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r "took" 10 + 5r ms; the job time is the slowest rank's
        t = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu", world)
        dist.barrier()
        v = bench.job_gbs(world, 1e9, 4, t * 1e-3)
        # the reference arm: only rank 0 works, the others return at once
        called = []
        bench.run_reference = lambda args: called.append(rank)
        os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
        sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world)]
        bench.main()
        q.put((rank, t, v, called))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, called in res:
        assert t == 15.0                         # max over ranks
        assert v == pytest.approx(2 * 4 / 15e-3)  # both ranks' bytes / slowest time
        assert called == ([0] if rank == 0 else [])
