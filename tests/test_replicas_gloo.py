"""The N > 1 path of bench.py runs independent replicas (no collective on the data path): the
host logic that joins them - a barrier, the maximum time over the ranks, the whole-job value of
all ranks' units over that time - checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 3.0 * rank                      # the ranks' own step times
        bench.barrier(world)
        worst = bench.max_over_ranks(ms, world)
        value = bench.replica_value(1000, world, worst)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{worst} {value}")
    finally:
        dist.destroy_process_group()


def test_two_replicas_join_on_the_slowest(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        worst, value = (float(x) for x in open(tmp_path / f"r{r}.txt").read().split())
        assert worst == 13.0
        assert abs(value - 2000 / 13e-3) < 1e-6 * value
