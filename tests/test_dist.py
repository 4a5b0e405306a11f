"""The benchmark's multi-process path on CPU: two gloo ranks (no GPU).

Every rank solves its own video (replicas, no data-path collective); the only
collectives are the barrier around the timed region and the max over ranks of
the elapsed time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ws, r, local = bench.dist_setup()
    assert (ws, r, local) == (world, rank, rank) and dist.get_backend() == "gloo"
    bench.barrier(ws)
    mx = bench.max_over_ranks(ws, 10.0 * (rank + 1))
    out[rank] = mx
    shapes = bench.batch_shapes()
    assert len(shapes) == 24 and shapes[0] == (240, 320, 4)
    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="CPU path (gloo)")
def test_two_gloo_ranks_barrier_and_max():
    world = 2
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == 20.0
