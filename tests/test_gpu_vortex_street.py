"""Vortex-street parity with the FP64 oracle over a long run (Sec. 3.1).

Cylinder channel 22D x 4.1D, D = 40 node spacings (~260k Poisson-disk nodes,
seed 2), K = 16, simple bounce-back, BGK, Re = 100 at streaming distance
s = 1/2 (D = 80 lattice units, U0 = 0.05, tau = 0.62), 200,000 steps from
rest to periodic shedding.  The GPU path (FP32) records C_D and C_L every 50
steps; over the second half of the run its Strouhal number (upward zero
crossings of C_L) must agree with the oracle's within 0.5 % and its mean
drag coefficient within 1 % (the vortex-street tolerance of the contract).

The oracle's statistics come from tests/golden/vortex_re100_s05.json,
written by tests/golden/make_vortex_golden.py, which runs the FP64 oracle
alone (about two hours on 8 cores).  The test first checks that it has
regenerated the same node set (count and coordinate hash).
"""
import json
import os
import sys

import numpy as np
import pytest

import oracle as O
from paper_2312_14789_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_vortex_golden as G  # noqa: E402

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(HERE, "golden", "vortex_re100_s05.json")


def test_vortex_street_strouhal_and_drag_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_14789_gb300 import mlbm
    gold = json.load(open(GOLDEN))
    w = I.karman(seed=gold["seed"])
    assert w.n == gold["nodes"] and G.node_set_hash(w) == gold["node_set_hash"], \
        "the node set differs from the one the golden statistics were computed on"
    re_, s, u0, d = gold["Re"], gold["s"], gold["U0"], gold["D_spacings"]
    every, steps = gold["sample_every"], gold["steps"]
    tau = 3.0 * u0 * (d / s) / re_ + 0.5
    assert tau == gold["tau"]
    d_lb = d / s
    st = mlbm.build_stencils_for(w, K=gold["K"], s=s, bb_mode=mlbm.BB_SIMPLE)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0))
    n_samples = steps // every
    cd, cl = np.empty(n_samples), np.empty(n_samples)
    for i in range(n_samples):
        mlbm.step(ctx, every)
        _, _, cd[i], cl[i] = mlbm.drag_lift(ctx, d, u0)
    h = n_samples // 2
    st_g = O.strouhal(cl[h:], every, d_lb, u0)
    cd_g = float(np.mean(cd[h:]))
    summary = {"strouhal": (st_g, gold["strouhal"]), "cd_mean": (cd_g, gold["cd_mean"]),
               "cl_amplitude": (float(np.ptp(cl[h:]) / 2), gold["cl_amplitude"])}
    assert np.isfinite(st_g), summary
    assert abs(st_g / gold["strouhal"] - 1) <= 5e-3, summary
    assert abs(cd_g / gold["cd_mean"] - 1) <= 1e-2, summary
