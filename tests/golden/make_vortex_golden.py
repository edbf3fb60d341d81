"""Write the FP64 oracle's vortex-street statistics (Sec. 3.1, Karman vortex
street) to tests/golden/vortex_re100_s05.json.  Calls only the oracle and the
seeded node-set generator; nothing here touches the CUDA library.

Case: channel 22D x 4.1D around a cylinder of D = 40 node spacings
(Poisson-disk nodes, seed 2, ~260k nodes), K = 16 least-squares stencils,
simple bounce-back on the cylinder, BGK, Re = 100 at streaming distance
s = 1/2 (D = 80 lattice units, U0 = 0.05, tau = 3 U0 (D/s) / Re + 1/2),
200,000 steps from rest.  C_D and C_L (momentum exchange) are sampled every
50 steps; the Strouhal number (upward zero crossings of C_L), the mean C_D
and the C_L amplitude are taken over the second half of the run.

    python tests/golden/make_vortex_golden.py [--steps 200000]

The oracle needs about half an hour on 8 cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

RE, S, U0, D, SEED, K = 100, 0.5, 0.05, 40.0, 2, 16
SAMPLE = 50
OUT = os.path.join(HERE, "vortex_re100_s05.json")


def node_set_hash(w) -> str:
    """Hash of the node set (coordinates rounded to 1e-9 spacings, classes),
    so that a test can check that it regenerated the same nodes."""
    h = hashlib.sha256()
    h.update(np.round(np.asarray(w.xy, np.float64) * 1e9).astype(np.int64).tobytes())
    h.update(np.asarray(w.node_class, np.uint8).tobytes())
    return h.hexdigest()[:16]


def oracle_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("mlbm_oracle.c", "__init__.py"):
        h.update(open(os.path.join(ROOT, "oracle", f), "rb").read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=200_000)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    import oracle as O
    from paper_2312_14789_gb300 import inputs as I

    tau = 3.0 * U0 * (D / S) / RE + 0.5
    d_lb = D / S
    w = I.karman(seed=SEED)
    t0 = time.time()
    op = O.Operator(w, K=K, s=S, bb_mode=0).check()
    t_build = time.time() - t0
    n_samples = args.steps // SAMPLE
    f = O.equilibrium(np.ones(w.n), 0.0, 0.0)
    cd, cl = np.empty(n_samples), np.empty(n_samples)
    t0 = time.time()
    for i in range(n_samples):
        f = O.run_bgk(op, f, tau, (0.0, 0.0), SAMPLE)
        fx, fy = O.force_bgk(op, f)
        cd[i] = 2.0 * fx / (U0 ** 2 * d_lb)
        cl[i] = 2.0 * fy / (U0 ** 2 * d_lb)
        if (i + 1) % 400 == 0:
            print(f"{(i + 1) * SAMPLE} steps, {time.time() - t0:.0f} s, C_D {cd[i]:.5f} C_L {cl[i]:.5f}",
                  file=sys.stderr, flush=True)
    t_run = time.time() - t0
    h = n_samples // 2
    out = {
        "case": "Karman vortex street, Sec. 3.1: channel 22D x 4.1D, D = 40 node spacings, Poisson-disk nodes",
        "Re": RE, "s": S, "U0": U0, "D_spacings": D, "tau": tau, "K": K, "bounce_back": "simple", "model": "BGK",
        "seed": SEED, "nodes": int(w.n), "node_set_hash": node_set_hash(w), "oracle_source_hash": oracle_source_hash(),
        "steps": args.steps, "sample_every": SAMPLE, "statistics_over": "second half of the run",
        "strouhal": O.strouhal(cl[h:], SAMPLE, d_lb, U0),
        "cd_mean": float(np.mean(cd[h:])),
        "cl_amplitude": float(np.ptp(cl[h:]) / 2),
        "cd_every_10000_steps": [float(v) for v in cd[199::200]],
        "cl_every_10000_steps": [float(v) for v in cl[199::200]],
        "oracle_seconds": {"stencils": t_build, "run": t_run},
        "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
        "written_by": "tests/golden/make_vortex_golden.py (FP64 oracle only)",
    }
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: out[k] for k in ("nodes", "strouhal", "cd_mean", "cl_amplitude")}))


if __name__ == "__main__":
    main()
