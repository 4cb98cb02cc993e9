"""The multi-GPU bench path is replicas (one independent solve per rank, no collective on the
data path): its plumbing -- process-group set-up from the torchrun environment, the barrier
around the timed region and the max over ranks -- checked with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        impl = "reference"   # the reference arm's ranks use gloo

    w, r, local = bench.dist_init(Args())
    bench.barrier(w)
    m = bench.max_over_ranks(float(10 + r), w)
    bench.barrier(w)
    out.put((r, w, m))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_max_time():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 11.0), (1, 2, 11.0)]
