"""The N > 1 path of bench.py on CPU: replicas only, so the only cross-rank
steps are the barrier around the timed region and the max-over-ranks of the
timed total.  Two gloo ranks on 127.0.0.1 check both."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    # each rank timed a different total; every rank must see the slowest one
    total_ms = bench.max_over_ranks(100.0 + 50.0 * rank, world)
    steps = 4
    ms_per_step = total_ms / steps
    value = world * 1000.0 / ms_per_step       # whole-job solves/s, as run_ours computes it
    out[rank] = (total_ms, value)
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    total_ms, value = out[0]
    assert total_ms == 150.0
    assert value == pytest.approx(2 * 1000.0 / (150.0 / 4))


def test_single_rank_helpers_are_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
