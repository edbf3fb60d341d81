"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
timing; the job time is the slowest rank's and the rate counts every rank's
replica; the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = [12.5, 40.0][rank]
    ms = bench.max_over_ranks(my_ms, dist, "cpu")
    rate = bench.whole_job_rate(1000, 10, world, ms)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{ms} {rate}")
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        ms, rate = (float(v) for v in open(tmp_path / f"rank{r}.txt").read().split())
        assert ms == 40.0
        assert abs(rate - 1000 * 10 * 2 / 0.040 / 1e6) < 1e-12


def test_single_process_rate_and_reference_rank_guard():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    # 143.9 us per step of 1,559,826 node-updates is 10,840 Mnode-updates/s
    assert abs(bench.whole_job_rate(1_559_826, 200, 1, 0.1439 * 200) - 1_559_826 / 143.9) < 1e-6

    class Args:
        steps, warmup = 1, 3
    # ranks other than 0 return before any work
    assert bench.run_reference(Args(), 1, 2) is None
