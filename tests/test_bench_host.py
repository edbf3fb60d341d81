"""Host-side pieces of bench.py that need no GPU: the algorithmic byte count of
the benchmark workload (the roofline's numerator) against the figure recorded
in the committed ncu summary, and the rule that ties the summary's DRAM
traffic to the step kernel source, variant and node order it was taken on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2312_14789_gb300 import mlbm  # noqa: E402


def _profile_fields():
    vals = {}
    for line in open(bench.PROFILE).read().splitlines():
        line = line.strip()
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    return vals


def test_algorithmic_bytes_of_the_bench_workload_match_the_profile():
    """Per node kind: 4 (9 + 9) + 24 K + 4 K + 1 bytes for a least-squares node,
    16 + 36 + 1 for an equilibrium node; the six runs of the sweep."""
    w = bench.make_workload()
    st_by_s = {s: mlbm.build_stencils_for(w, K=16, s=s, bb_mode=mlbm.BB_SIMPLE)
               for s in sorted({s for _, s in bench.CASES})}
    infos = [mlbm.stencils_info(st_by_s[s]) for _, s in bench.CASES]
    total = sum(bench.algorithmic_bytes(i, 16) for i in infos)
    n_wls = sum(i["n_wls"] for i in infos)
    n_eq = sum(i["n_eq"] for i in infos)
    assert sum(i["n_lagrange"] for i in infos) == 0
    assert total == n_wls * 521 + n_eq * 53
    assert total == int(_profile_fields()["algorithmic_bytes_per_launch"])


def test_profile_traffic_applies_only_to_its_kernel_source_variant_and_order():
    f = _profile_fields()
    variant = int(f["kernel_variant"])
    order = bench.ORDER_NAMES.index(f["node_order"])
    if f["kernel_source_hash"] != bench.kernel_source_hash():
        pytest.skip("the step kernel source changed since the summary was taken")
    t = bench.measured_traffic(variant, order)
    assert t == float(f["dram_bytes_per_launch"])
    # within a few percent of the algorithmic bytes: nothing re-read
    assert 0.99 <= t / int(f["algorithmic_bytes_per_launch"]) <= 1.02
    assert bench.measured_traffic(variant + 1, order) is None
    assert bench.measured_traffic(variant, (order + 1) % len(bench.ORDER_NAMES)) is None
