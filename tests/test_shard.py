"""Sharding the batched porous samples across ranks (no GPU).

* The balanced assignment is a partition of the samples, identical on every
  rank, and its largest load is within the greedy rule's bound of the mean.
* Two gloo ranks each take their share of a sample set, compute per-sample
  results, gather them and merge them back into sample order; the job's
  rate counts every rank's node updates over the slowest rank's time.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")

from paper_2312_14789_gb300 import inputs as I  # noqa: E402
from paper_2312_14789_gb300 import shard  # noqa: E402


def test_assignment_is_a_balanced_partition():
    w = [s["n_target"] for s in I.porous_batch_specs(64)]
    for world in (1, 2, 3, 4, 8):
        a = shard.assign_balanced(w, world)
        assert sorted(i for part in a for i in part) == list(range(64))
        assert a == shard.assign_balanced(list(w), world)
        loads = [sum(w[i] for i in part) for part in a]
        # greedy LPT: the largest load exceeds the mean by at most the largest item
        assert max(loads) - np.mean(loads) <= max(w)
        assert shard.imbalance(w, a) < 1.05 or world == 8
    assert shard.assign_balanced([5, 5, 5], 2) == [[0, 2], [1]]
    with pytest.raises(ValueError):
        shard.assign_balanced([1], 0)


def test_merge_by_sample():
    a = [[0, 3], [1, 2, 4]]
    assert shard.merge_by_sample([["a", "d"], ["b", "c", "e"]], a, 5) == ["a", "b", "c", "d", "e"]
    with pytest.raises(ValueError):
        shard.merge_by_sample([["a"], ["b", "c", "e"]], a, 5)
    with pytest.raises(ValueError):
        shard.merge_by_sample([["a", "d"], ["b", "c", "e"]], a, 6)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2312_14789_gb300 import shard as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    weights = [120, 80, 75, 60, 50, 40, 10]
    a = S.assign_balanced(weights, world)
    mine = a[rank]
    # per-sample "results" that identify the sample
    results = [1000 + i for i in mine]
    gathered = [None] * world
    dist.all_gather_object(gathered, results)
    merged = S.merge_by_sample(gathered, a, len(weights))
    my_updates = sum(weights[i] for i in mine) * 10
    total = bench.sum_over_ranks(my_updates, dist, "cpu")
    ms = bench.max_over_ranks([5.0, 8.0][rank], dist, "cpu")
    rate = bench.job_rate(total, ms)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(" ".join(str(v) for v in merged) + f"\n{total} {ms} {rate}")
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_merge(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        lines = open(tmp_path / f"rank{r}.txt").read().splitlines()
        assert [int(v) for v in lines[0].split()] == [1000 + i for i in range(7)]
        total, ms, rate = (float(v) for v in lines[1].split())
        assert total == 4350.0 and ms == 8.0
        assert abs(rate - 4350.0 / 0.008 / 1e6) < 1e-12
