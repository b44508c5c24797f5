"""bench.py's multi-GPU plumbing ("replicas only": one apply does not shard, N ranks each run
the whole workload).  Two gloo ranks on the host check the max-over-ranks reduction and the
whole-job rate; no GPU is used."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist                      # noqa: E402
import torch.multiprocessing as mp                    # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    r, w = bench.dist_setup(0)                         # no GPUs: gloo
    assert (r, w) == (rank, world)
    ms_local = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    ms, value = bench.replica_rate(ms_local, 1000, w)
    bench.barrier(w)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_gloo_replicas():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        ms, value = out[rank]
        assert ms == pytest.approx(15.0)               # max over ranks
        assert value == pytest.approx(world * 1000 / 15e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_rate(20.0, 500, 1) == (20.0, pytest.approx(500 / 20e-3 / 1e6))
