"""Run the fused step on a named workload for a few steps (for profilers).

    python -m paper_2312_14789_gb300.profile_step --workload karman --steps 3
    python -m paper_2312_14789_gb300.profile_step --workload porous --steps 3

karman: the ~260k-node cylinder channel, BGK, K = 16, s = 1/2 (one run);
karman_sweep: its six (Re, s) runs in one batched context (the benchmark case);
porous: the ~1M-node porous box, tau = 1, K = 16, s = 1/2.
No timing is reported; the process exits 0 when the steps ran.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2312_14789_gb300 import inputs as I  # noqa: E402
from paper_2312_14789_gb300 import mlbm  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="karman", choices=["karman", "karman_sweep", "porous"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--n-target", type=int, default=1_000_000)
    ap.add_argument("--variant", type=int, default=-1, help="kernel variant (-1: autotune)")
    ap.add_argument("--node-order", default="hilbert", choices=["hilbert", "morton", "rows", "input"],
                    help="device node order of the stencils")
    args = ap.parse_args()
    order = ["hilbert", "morton", "rows", "input"].index(args.node_order)
    if args.workload == "karman_sweep":
        import bench
        w = I.karman(seed=2)
        st_by_s = {s: mlbm.build_stencils_for(w, K=16, s=s, bb_mode=mlbm.BB_SIMPLE)
                   for s in sorted({s for _, s in bench.CASES})}
        for st in st_by_s.values():
            mlbm.stencils_set_order(st, order)
        ctx = mlbm.batch_init([st_by_s[s] for _, s in bench.CASES],
                              [mlbm.Params(mlbm.MODEL_BGK, bench.tau_of(re, s), 0.0, 0.0, 0.0) for re, s in bench.CASES])
    elif args.workload == "karman":
        w = I.karman(seed=2)
        st = mlbm.build_stencils_for(w, K=16, s=0.5, bb_mode=mlbm.BB_SIMPLE)
        mlbm.stencils_set_order(st, order)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, 0.62, 0.0, 0.0, 0.0))
    else:
        w = I.porous(seed=3, n_target=args.n_target)
        st = mlbm.build_stencils_for(w, K=16, s=0.5, bb_mode=mlbm.BB_INTERPOLATED)
        mlbm.stencils_set_order(st, order)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-6, 0.0))
    if args.variant >= 0:
        mlbm.set_kernel_variant(ctx, args.variant)
    else:
        mlbm.autotune(ctx, 10)
    mlbm.set_graphs(ctx, False)  # one launch per step, so a profiler can pick single launches
    mlbm.step(ctx, args.warmup + args.steps)
    rho, _ = mlbm.macroscopics(ctx)
    print(f"{args.workload}: {ctx.n} nodes, variant {mlbm.kernel_variant(ctx)}, {args.warmup + args.steps} steps, "
          f"mean rho {rho.mean():.6f}")


if __name__ == "__main__":
    main()
