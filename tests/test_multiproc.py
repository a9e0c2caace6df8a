"""The whole-job totals of bench.py's multi-GPU path on CPU: two gloo ranks
report the slowest rank's time and the sum of the work every rank did (the
split of the job itself is tested in test_multirank.py)."""
import os
import socket
import sys
from pathlib import Path

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, str(ROOT))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, dd = bench.job_totals(1.5 + rank, 10.0 * (rank + 1), "cpu")
    out[rank] = torch.tensor([ms, dd, 0.0], dtype=torch.float64)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_totals_gloo():
    world = 2
    out = torch.zeros((world, 3), dtype=torch.float64).share_memory_()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r, 0].item() == 2.5            # the slowest rank's time
        assert out[r, 1].item() == 30.0           # all ranks' work


def test_single_process_totals_pass_through():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.job_totals(3.0, 7.0, "cpu") == (3.0, 7.0)
