"""Host logic of the multi-GPU bench path ("replicas only": one independent channel per rank,
no collective on the data path): the max-over-ranks timing reduction and the whole-job
throughput, run as two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    ms = 100.0 + 25.0 * rank                      # rank 1 is the slower one
    slowest = bench.max_over_ranks(ms, w, "cpu")
    out[rank] = (slowest, bench.replica_throughput(1000, 10, w, slowest * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    slowest, value = out[0]
    assert slowest == 125.0
    # 2 replicas x 1000 points x 10 steps in 0.125 s
    assert value == pytest.approx(2 * 1000 * 10 / 0.125 / 1e6)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_throughput(10, 2, 1, 1.0) == pytest.approx(2e-5)
