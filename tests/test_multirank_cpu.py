"""The replica path of bench.py on two gloo ranks (CPU): the job time is the
slowest rank's and the throughput counts every rank's replica."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = [10.0, 25.0][rank]
    mx = bench.max_over_ranks(local_ms, ws, "cpu")
    dist.barrier()
    value = bench.weak_scaling_value(ws, 1000, 5, mx)
    if rank == 0:
        with open(out_path, "w") as f:
            f.write("%r %r" % (mx, value))
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r0.txt")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    mx, value = map(float, open(out).read().split())
    assert mx == 25.0
    assert value == pytest.approx(2 * 1000 * 5 / 0.025)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.weak_scaling_value(1, 10, 2, 1000.0) == pytest.approx(20.0)
