"""Multi-replica timing of bench.py on CPU: two gloo ranks stand in for two GPUs.

With N GPUs every rank runs an independent replica of the workload (the path has no exchange
step on this one-GPU-per-box setup), the ranks take the slowest rank's time, and the reported
value is the DOF x steps of all replicas over that time."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 * (rank + 1)   # rank r took 10 (r + 1) ms for its replica
        slow = bench.slowest_rank_ms(ms, world, "cpu")
        value = bench.job_value(1000, 5, world, slow)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{slow} {value}\n")
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    got = [tuple(map(float, open(tmp_path / f"rank{r}.txt").read().split())) for r in range(2)]
    for slow, value in got:
        assert slow == 20.0
        # 2 replicas x 1000 DOF x 5 steps in 20 ms
        assert value == pytest.approx(2 * 1000 * 5 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(12.5, 1, "cpu") == 12.5
    assert bench.job_value(100, 4, 1, 2.0) == pytest.approx(100 * 4 / 0.002)
