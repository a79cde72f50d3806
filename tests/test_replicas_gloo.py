"""The N > 1 benchmark path (independent replicas, one per rank) on CPU with
two gloo ranks: ranks trace disjoint frames, the timed region's duration is
the maximum over ranks, and the job rate counts every rank's units."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank)
    dist.barrier()
    q.put((rank, bench.replica_frame_base(rank), t,
           bench.job_throughput(10_000 * 3, world, t)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import socket
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = mp.Queue()
    ps = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, t0, v0), (r1, b1, t1, v1) = out
    assert b0 != b1                       # disjoint frames
    assert t0 == t1 == 15.0               # max over ranks on every rank
    assert v0 == v1 == pytest.approx(2 * 30_000 / 0.015)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(100, 1, 1000.0) == 100.0
