"""Host-side pieces of bench.py that need no GPU: the algorithmic byte count
(the roofline's numerator) per node kind and model, the rule that ties a
committed ncu traffic record to the step kernel source, variant and node
order it was taken on (and scales a smaller capture to the bench launch),
the clock sampler's parsing, and the batched porous configuration's specs."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2312_14789_gb300 import inputs as I  # noqa: E402
from paper_2312_14789_gb300 import mlbm  # noqa: E402


def test_algorithmic_bytes_per_node_kind():
    """tau = 1: 4 (3 + 3) + 24 K + 4 K + 1 = 473 B per least-squares node at
    K = 16; BGK: 4 (9 + 9) + 24 K + 4 K + 1 = 521 B; equilibrium nodes 25 and
    53 B; Lagrange nodes 77 and 125 B."""
    info = {"n_wls": 10, "n_lagrange": 3, "n_eq": 2}
    assert bench.algorithmic_bytes(info, 16, "tau1") == 10 * 473 + 3 * 77 + 2 * 25
    assert bench.algorithmic_bytes(info, 16, "bgk") == 10 * 521 + 3 * 125 + 2 * 53
    assert bench.algorithmic_bytes(info, 12, "bgk") == 10 * 409 + 3 * 125 + 2 * 53
    w = I.porous(seed=5, n_target=3000, porosity=0.7)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED)
    i = mlbm.stencils_info(st)
    assert i["n_wls"] + i["n_lagrange"] + i["n_eq"] == w.n
    assert bench.algorithmic_bytes(i, 16, "tau1") == i["n_wls"] * 473 + i["n_lagrange"] * 77


def test_traffic_record_applies_only_to_its_kernel_and_scales(tmp_path, monkeypatch):
    rec = {"kernel_source_hash": bench.kernel_source_hash(), "kernel_variant": 26, "node_order": "hilbert",
           "dram_bytes_per_launch": 1.0e9, "node_updates_per_launch": 2_000_000}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setitem(bench.TRAFFIC, "porous_batch", str(p))
    assert bench.measured_traffic("porous_batch", 26, 0) == 1.0e9
    assert bench.measured_traffic("porous_batch", 26, 0, node_updates=6_000_000) == pytest.approx(3.0e9)
    assert bench.measured_traffic("porous_batch", 25, 0) is None
    assert bench.measured_traffic("porous_batch", 26, 1) is None
    rec["kernel_source_hash"] = "0" * 16
    p.write_text(json.dumps(rec))
    assert bench.measured_traffic("porous_batch", 26, 0) is None
    monkeypatch.setitem(bench.TRAFFIC, "porous_batch", str(tmp_path / "missing.json"))
    assert bench.measured_traffic("porous_batch", 26, 0) is None


def test_committed_traffic_records_are_consistent():
    """Each committed record names its capture and lies within a few percent
    of the algorithmic bytes of the launch it was taken on."""
    for path in bench.TRAFFIC.values():
        if not os.path.exists(path):
            continue
        rec = json.load(open(path))
        for k in ("kernel_source_hash", "kernel_variant", "node_order", "dram_bytes_per_launch",
                  "algorithmic_bytes_per_launch", "command"):
            assert k in rec, (path, k)
        assert 0.95 <= rec["dram_bytes_per_launch"] / rec["algorithmic_bytes_per_launch"] <= 1.10


def test_clock_parsing():
    out = "\n".join([
        "2070, 2070, 300.1, 0, Not Active, Not Active, Not Active, Not Active",
        "1965, 2070, 1200.5, 100, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 1210.5, 99, Not Active, Not Active, Not Active, Active",
        "2010, 2070, 1100.0, 97, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.Clocks.parse(out)
    assert c["sm_mhz"] == 1980 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 4 and c["samples_under_load"] == 3


def test_porous_batch_specs():
    a = I.porous_batch_specs(64)
    assert len(a) == 64 and a[0]["seed"] == 1000 and a[-1]["seed"] == 1063
    assert all(50_000 <= s["n_target"] < 400_000 and 0.5 <= s["porosity"] < 0.85 for s in a)
    assert [s["s"] for s in a[:4]] == [1.0, 0.5, 0.25, 1.0]
    assert [s["g"] for s in a[:3]] == [1e-6, 5e-6, 2e-5]
    # seeds decide the samples: a later rank's set continues the sequence
    b = I.porous_batch_specs(4, first_seed=1002)
    assert b[0]["n_target"] == a[2]["n_target"] and b[0]["porosity"] == a[2]["porosity"]


def test_ranks_share_the_host_cores(monkeypatch):
    monkeypatch.delenv("OMP_NUM_THREADS", raising=False)
    monkeypatch.setenv("LOCAL_WORLD_SIZE", "4")
    monkeypatch.setattr(bench.os, "cpu_count", lambda: 64)
    assert bench.share_host_cores(4) == 16
    assert bench.os.environ["OMP_NUM_THREADS"] == "16"
    monkeypatch.setenv("OMP_NUM_THREADS", "3")          # a caller's setting stays
    bench.share_host_cores(4)
    assert bench.os.environ["OMP_NUM_THREADS"] == "3"
    monkeypatch.delenv("OMP_NUM_THREADS")
    monkeypatch.setenv("LOCAL_WORLD_SIZE", "1")
    bench.share_host_cores(1)
    assert "OMP_NUM_THREADS" not in bench.os.environ


def test_strouhal_of_a_sampled_sine():
    """St = D / (period U0): a C_L series with a period of 1234.5 steps,
    sampled every 50 steps, gives its frequency back from the zero crossings."""
    import numpy as np
    every, d_lb, u0, period = 50, 80.0, 0.05, 1234.5
    t = np.arange(0, 200_000, every, dtype=np.float64)
    cl = 0.02 + 0.3 * np.sin(2 * np.pi * t / period + 0.4)
    st = bench.strouhal_of(cl, every, d_lb, u0)
    assert abs(st / (d_lb / (period * u0)) - 1) < 1e-4
    assert bench.strouhal_of(np.ones(10), every, d_lb, u0) is None


def test_karman_lattice_cells():
    import numpy as np
    cell, eqv = I.karman_lattice(80.0)
    assert cell.shape == (328, 1760)
    assert abs((cell == 1).sum() / (np.pi * 40.0 ** 2) - 1) < 0.01     # the cylinder's area
    assert np.all(cell[0] == 2) and np.all(cell[-1] == 2) and np.all(cell[:, 0] == 2) and np.all(cell[:, -1] == 2)
    # parabolic inflow with maximum U0 = 0.05 across the channel, rest on top and bottom
    h = cell.shape[0] - 1.0
    assert abs(eqv[int(h // 2), 0, 1] - 0.05 * 4 * (h // 2) * (h - h // 2) / h ** 2) < 1e-15
    assert eqv[0, 0, 1] == 0.0 and np.all(eqv[..., 0] == 1.0)
