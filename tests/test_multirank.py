"""The bench's multi-rank path on CPU (gloo, world size 2): each rank times its own
replica, the timed region is the maximum over ranks, and the whole-job rate counts
every rank's iterations.  No GPU and no collective on the data path."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = 100.0 + 50.0 * rank  # rank 1 is the slower replica
    got = bench.reduce_max_ms(mine, dist, torch.device("cpu"))
    rate = bench.whole_job_rate(world, 20, got)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max_ms": got, "rate": rate}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_count_all_iterations(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["max_ms"] == pytest.approx(150.0)
        assert r["rate"] == pytest.approx(2 * 20 / 0.150)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max_ms(12.5, None, None) == 12.5
    assert bench.whole_job_rate(1, 10, 500.0) == pytest.approx(20.0)
