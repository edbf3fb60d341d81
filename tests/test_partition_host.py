"""The partition plan of a node set (host only, no GPU) and its halo exchange
across two gloo ranks.

* The owned sets split the nodes into contiguous ranges of device positions;
  each partition's halo is exactly the set of stencil members its nodes
  reference outside the range (checked against the exported stencils), and
  halo_from counts them per owner.
* Two gloo ranks each own one partition and advance a stand-in operator
  that, like the streaming step, reads every node's stencil members only
  (x_i <- sum_j c_ij x_idx(i,j) + d_i, FP64, fixed slot order), exchanging
  halo values with send/recv after every step in the plan's order; after
  several steps every rank's owned values equal the unpartitioned
  computation bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2312_14789_gb300 import inputs as I  # noqa: E402
from paper_2312_14789_gb300 import mlbm  # noqa: E402


def _stencils(n=3000, seed=48):
    w = I.porous(seed=seed, n_target=n, porosity=0.7)
    return w, mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED)


@pytest.mark.parametrize("n_parts,bounds", [(1, None), (2, None), (3, None), (5, "uneven")])
def test_plan_halo_is_exactly_the_referenced_outside_set(n_parts, bounds):
    w, st = _stencils()
    if bounds == "uneven":
        bounds = np.array([0, 100, 101, 1500, 2000, w.n])
    plan = mlbm.partition_plan(st, n_parts, bounds)
    assert plan["n_owned"].sum() == w.n
    assert plan["first"][0] == 0 and np.all(np.diff(plan["first"]) == plan["n_owned"][:-1])
    idx = mlbm.stencils_export(st)["idx"]          # caller ids
    owner = np.empty(w.n, np.int64)
    owned_all = []
    for q in range(n_parts):
        owned, halo = mlbm.partition_nodes(st, n_parts, q, bounds)
        assert len(owned) == plan["n_owned"][q] and len(halo) == plan["n_halo"][q]
        owner[owned] = q
        owned_all.append(owned)
    assert np.array_equal(np.sort(np.concatenate(owned_all)), np.arange(w.n))
    for q in range(n_parts):
        owned, halo = mlbm.partition_nodes(st, n_parts, q, bounds)
        ref = np.setdiff1d(np.unique(idx[owned]), owned)
        assert np.array_equal(np.sort(halo), ref)
        # halo slots grouped by owner, in increasing owner order
        assert np.all(np.diff(owner[halo]) >= 0)
        for o in range(n_parts):
            assert plan["halo_from"][q, o] == np.count_nonzero(owner[halo] == o)
        assert plan["halo_from"][q, q] == 0


def test_plan_rejects_bad_bounds():
    w, st = _stencils(1500)
    for P, b in [(2, [0, 10]), (2, [1, 10, w.n]), (2, [0, 10, w.n + 1]), (3, [0, 10, 10, w.n]), (0, None)]:
        with pytest.raises((mlbm.MlbmError, ValueError)):
            mlbm.partition_plan(st, P, b)


def _coeffs(n, K, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, (n, K))
    c /= c.sum(1, keepdims=True) * 1.01
    return c, rng.uniform(-1e-3, 1e-3, n)


def _apply(x, idx, c, d, rows):
    out = np.empty(len(rows))
    for r, i in enumerate(rows):
        acc = 0.0
        for j in range(idx.shape[1]):
            acc += c[i, j] * x[idx[i, j]]
        out[r] = acc + d[i]
    return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


STEPS = 6


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = I.porous(seed=49, n_target=1200, porosity=0.7)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED)
    idx = mlbm.stencils_export(st)["idx"]
    c, d = _coeffs(w.n, 16, 5)
    x0 = np.random.default_rng(6).uniform(0.5, 1.5, w.n)
    parts = [mlbm.partition_nodes(st, world, q) for q in range(world)]
    owned, halo = parts[rank]
    # this rank's memory: owned values, then halo values
    local = {int(v): i for i, v in enumerate(np.concatenate([owned, halo]))}
    x = np.concatenate([x0[owned], x0[halo]])
    lidx = np.vectorize(local.get)(idx[owned])

    def exchange(x):
        # send to every peer the owned values in its halo, in its slot order;
        # receive into this rank's halo block of each peer
        reqs = []
        for o in range(world):
            if o == rank:
                continue
            peer_halo = parts[o][1]
            mine = peer_halo[np.isin(peer_halo, owned)]
            buf = torch.from_numpy(x[[local[int(v)] for v in mine]].copy())
            reqs.append(dist.isend(buf, dst=o))
        for o in range(world):
            if o == rank:
                continue
            theirs = halo[np.isin(halo, parts[o][0])]
            buf = torch.empty(len(theirs), dtype=torch.float64)
            dist.recv(buf, src=o)
            x[[local[int(v)] for v in theirs]] = buf.numpy()
        for r in reqs:
            r.wait()

    for _ in range(STEPS):
        new_owned = np.empty(len(owned))
        for r, i in enumerate(owned):
            acc = 0.0
            for j in range(16):
                acc += c[i, j] * x[lidx[r, j]]
            new_owned[r] = acc + d[i]
        x[:len(owned)] = new_owned
        exchange(x)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.stack([owned.astype(np.float64), x[:len(owned)]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_halos_and_match_the_unpartitioned_result(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    w = I.porous(seed=49, n_target=1200, porosity=0.7)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED)
    idx = mlbm.stencils_export(st)["idx"]
    c, d = _coeffs(w.n, 16, 5)
    x = np.random.default_rng(6).uniform(0.5, 1.5, w.n)
    for _ in range(STEPS):
        x = _apply(x, idx, c, d, np.arange(w.n))
    seen = np.zeros(w.n, bool)
    for r in range(2):
        ids, vals = np.load(tmp_path / f"rank{r}.npy")
        ids = ids.astype(np.int64)
        assert np.array_equal(vals, x[ids])       # bit for bit
        seen[ids] = True
    assert seen.all()
