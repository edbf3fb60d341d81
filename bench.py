"""Benchmark of the fused MLBM step and of the time to steady state.

Default workload (`--workload porous_batch`): the batched porous
configuration of Sec. 3.2's flow through a porous sample -- 64 independent
samples (seeds 1000..1063), each a square box of random non-overlapping
solid disks (radii U(8, 16) spacings) with node count U(50k, 400k) and
porosity U(0.5, 0.85), periodic in x with solid walls top and bottom, K = 16
least-squares stencils, interpolated bounce-back, the tau = 1 model (MLBM1:
only rho and u stored) in FP32, streaming distance cycling {1, 1/2, 1/4} and
body force {1e-6, 5e-6, 2e-5} (Darcy and inertial samples mixed); all 64 in
one batched context, one fused launch per time step replayed from captured
CUDA graphs, kernel variant picked by the library's autotuner.  One bench
"step" is one time step of every sample (~13M node updates).  The working
set (~6 GB) is far larger than L2, so steps are timed back to back without
a flush.  Graph capture and instantiation happen before the timed region.

After the timed steps (N = 1 only) the time-to-steady legs run on held-out
porous samples of the learned warm-start configuration (porosity 0.7,
~192k nodes, s = 1, g = 1e-6, seeds 20000..): cold single-instance runs,
one cold batched run, a learned warm start (network trained here, on the
GPU, on cold-solved training samples, seeds 10000..) batched and single,
each to |u(t) - u(t-1000)| / (1000 |u(t)|) < 1e-7 checked every 100 steps,
plus the paper's own criterion (Sec. 3.2: relative change of the mean
velocity over 2e4 steps per unit time below 1e-2) on the cold batch.

`--workload karman_sweep`: the vortex-street sweep (channel 22D x 4.1D, D =
40 spacings, ~260k nodes, BGK, simple bounce-back; the six runs Re in
{100, 200} x s in {1/2, 1/4, 1/8} in one batched context).

`--workload lattice_compare`: the paper's comparison with lattice LBM (Sec.
3.1), the vortex street at Re = 100: the lattice (D = 80 spacings) against
the meshless step on the scattered, hybrid and coarsened hybrid node sets
and with the paper's RBF-FD interpolant (D = 40 node spacings, s = 1/2): time
per step of each and, over --vortex-steps from rest, Strouhal number and
drag; `value` is the scattered least-squares rate.

`--workload porous_box`: one porous sample of Sec. 3.2 at full size (seed 3,
~960k nodes, porosity 0.7, K = 16, tau = 1, interpolated bounce-back, s = 1/2,
g = 1e-5 along x); ~450 MB of stencil rows per step, larger than L2, so
steps are timed back to back.  Under torchrun every rank steps its own box
(seed 3 + rank).  After the timed steps (N = 1 only, unless --no-steady) the
box runs from rest to steady state at four (s, g): one Darcy and three
inertial runs.

Arms:
  default            the CUDA path through the C ABI (device-resident state)
  --impl reference   the FP64 CPU oracle on a bounded node sample of the
                     same workload (the reference arm; no GPU)
  --variant V        a fixed step kernel variant instead of the autotuner
Multi-GPU (torchrun): every rank owns whole samples and nothing is exchanged
while stepping; `--scaling weak` (default) gives every rank its own 64
samples (seeds offset by the rank), `--scaling strong` splits the one set of
64 among the ranks, balanced by node count.
Output: one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mnode-updates/s (FP32, err vs FP64 stated); time-to-steady warm vs cold"
UNIT = "Mnode-updates/s"
ORDER_NAMES = ["hilbert", "morton", "rows", "input"]

# vortex-street sweep
U0, D = 0.05, 40.0
CASES = [(re, s) for re in (100, 200) for s in (0.5, 0.25, 0.125)]
# single porous box
BOX_SEED, BOX_S, BOX_G = 3, 0.5, 1e-5

# time-to-steady legs (criterion of the learned warm-start configuration)
TOL, WINDOW, CHECK = 1e-7, 1000, 100
PAPER_THRESHOLD, PAPER_DN, PAPER_CHECK = 1e-2, 20000, 1000
# nodes per timed oracle step: the oracle runs node sets of 16384 or more on
# all host threads (smaller ones on one)
ORACLE_SAMPLE = 32768


def tau_of(re, s):
    return 3.0 * U0 * (D / s) / re + 0.5


def algorithmic_bytes(info, K, model="bgk", rows=6):
    """Bytes one fused step must move at minimum, per node kind.
    BGK: least-squares node 4*(9+9) populations + 4*6K matrix + 4K indices +
    1 meta (RBF-FD stencils: rows = 8 weight rows instead of the 6 matrix
    rows); Lagrange node 4*(9+9) + 4*12 indices + 4 (s/h) + 1; equilibrium
    node 16 + 36 + 1.  tau = 1: the state is (rho, u_x, u_y), 3 floats read
    and 3 written, so 4*(3+3) replaces 4*(9+9) and an equilibrium node costs
    12 + 12 + 1 (the 16-byte padding of the stored state is not the method's
    work and is not counted)."""
    state = 4 * 6 if model == "tau1" else 4 * 18
    wls = state + 4 * rows * K + 4 * K + 1
    lag = state + 4 * 12 + 4 + 1
    eq = 12 + 12 + 1 if model == "tau1" else 16 + 36 + 1
    return info["n_wls"] * wls + info["n_lagrange"] * lag + info["n_eq"] * eq


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels_bgk.cu", "kernels_bgk_generic.cu", "kernels_bgk_alt.cu", "kernels_tau1.cu",
              "kernels_rbf.cu", "kernels_ring1.cu",
              "kernels_tma.cu", "step_node.cuh", "ring.cuh", "launch_util.cuh", "device_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2312_14789_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


TRAFFIC = {"porous_batch": os.path.join(ROOT, "profiles", "tau1_step_porous_batch.json"),
           "karman_sweep": os.path.join(ROOT, "profiles", "bgk_step_karman_sweep.json"),
           "porous_box": os.path.join(ROOT, "profiles", "tau1_step_porous_box.json")}


def measured_traffic(workload, variant, order=0, node_updates=None):
    """DRAM bytes per launch of the step kernel from the committed ncu
    record of this workload (profiles/*.json, written from an ncu capture),
    or None when it was taken on another kernel source, variant or node
    order.  A record taken on a smaller case of the same kernel is scaled to
    this launch by the node updates it processes."""
    try:
        rec = json.load(open(TRAFFIC[workload]))
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash() or rec.get("node_order", "hilbert") != ORDER_NAMES[order]:
        return None
    by_variant = rec.get("dram_bytes_per_launch_by_variant") or {str(rec.get("kernel_variant")): rec.get(
        "dram_bytes_per_launch")}
    if str(variant) not in by_variant:
        return None
    t = float(by_variant[str(variant)])
    if node_updates and rec.get("node_updates_per_launch"):
        t *= node_updates / float(rec["node_updates_per_launch"])
    return t


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class Clocks:
    """nvidia-smi sampled every 50 ms; samples at >= 50% utilisation count
    as under load."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        return self.parse(out)

    @staticmethod
    def parse(out):
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 7]
        sm_all, sm_load, mx, reasons = [], [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm, mx, util = float(r[0]), float(r[1]), float(r[3])
            except ValueError:
                continue
            sm_all.append(sm)
            if util >= 50:
                sm_load.append(sm)
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        use = sm_load or sm_all
        return {"sm_mhz": statistics.median(use) if use else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm_all), "samples_under_load": len(sm_load)}


# ------------------------------------------------------------------ workloads
def porous_specs(args, rank, world):
    """This rank's sample specs and the assignment (strong scaling) or seed
    offset (weak scaling)."""
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import shard
    if args.scaling == "strong" and world > 1:
        specs = I.porous_batch_specs(args.samples)
        assignment = shard.assign_balanced([s["n_target"] for s in specs], world)
        return [specs[i] for i in assignment[rank]], assignment
    first = 1000 + shard.rank_seed_offset(rank, args.samples)
    return I.porous_batch_specs(args.samples, first_seed=first), None


def make_inputs(args, rank, world):
    """Node sets of this rank (spawned worker processes; called before CUDA
    is touched)."""
    from paper_2312_14789_gb300 import inputs as I
    if args.workload in ("karman_sweep", "lattice_compare"):
        return {"karman": I.karman(seed=2)}
    if args.workload == "porous_box":
        return {"box": I.porous(seed=BOX_SEED + rank)}
    specs, assignment = porous_specs(args, rank, world)
    procs = min(16, int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), len(specs))
    out = {"specs": specs, "assignment": assignment, "batch": I.generate(specs, procs=procs)}
    if rank == 0 and world == 1 and args.steady:
        test = [{"seed": 20000 + i, "n_target": 200_000, "porosity": 0.7} for i in range(args.steady_samples)]
        train = [{"seed": 10000 + i, "n_target": args.train_nodes, "porosity": 0.7}
                 for i in range(args.train_samples)]
        ws = I.generate(test + train)
        out["steady_test"], out["steady_train"] = ws[:len(test)], ws[len(test):]
    return out


def build_batch(args, inputs):
    """Stencils, params and per-sample byte counts of the timed batch."""
    from paper_2312_14789_gb300 import mlbm
    if args.workload == "karman_sweep":
        w = inputs["karman"]
        st_by_s = {s: mlbm.build_stencils_for(w, K=16, s=s, bb_mode=mlbm.BB_SIMPLE)
                   for s in sorted({s for _, s in CASES})}
        sts = [st_by_s[s] for _, s in CASES]
        params = [mlbm.Params(mlbm.MODEL_BGK, tau_of(re, s), 0.0, 0.0, 0.0) for re, s in CASES]
        return sts, params, "bgk", list(st_by_s.values())
    if args.workload == "porous_box":
        st = mlbm.build_stencils_for(inputs["box"], K=16, s=BOX_S, bb_mode=mlbm.BB_INTERPOLATED)
        return [st], [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, BOX_G, 0.0)], "tau1", [st]
    sts = [mlbm.build_stencils_for(w, K=16, s=sp["s"], bb_mode=mlbm.BB_INTERPOLATED)
           for w, sp in zip(inputs["batch"], inputs["specs"])]
    params = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, sp["g"], 0.0) for sp in inputs["specs"]]
    return sts, params, "tau1", sts


def workload_config(args, inputs, infos, n, world):
    if args.workload == "lattice_compare":
        return {"workload": "karman_lattice_vs_meshless", "Re": LC_RE, "U0": U0, "D_node_spacings": D, "s": LC_S,
                "nodes": inputs["karman"].n, "seed": 2, "node_updates_per_step": n,
                "timed_here": "the meshless step on the scattered set (the oracle's BGK step)"}
    if args.workload == "karman_sweep":
        w = inputs["karman"]
        return {"workload": "karman_vortex_street_sweep",
                "runs": [{"Re": re, "s": s, "tau": round(tau_of(re, s), 4)} for re, s in CASES],
                "nodes_per_run": w.n, "K": 16, "model": "BGK", "D_spacings": 40, "U0": U0, "seed": 2,
                "bounce_back": "simple", "node_updates_per_step": n,
                "l2": "working set ~780 MB > L2 (129 MB): steps timed back to back, no flush"}
    if args.workload == "porous_box":
        w = inputs["box"]
        return {"workload": "porous_box", "seed": BOX_SEED, "nodes": w.n, "porosity": round(w.meta["porosity"], 4),
                "s": BOX_S, "g": BOX_G, "K": 16, "model": "MLBM1 (tau = 1)", "bounce_back": "interpolated",
                "node_updates_per_step": n,
                "l2": "working set ~480 MB > L2 (129 MB): steps timed back to back, no flush"}
    ws = inputs["batch"]
    return {"workload": "porous_batch_64" if args.samples == 64 else f"porous_batch_{args.samples}",
            "samples_per_rank": len(ws), "seeds": [sp["seed"] for sp in inputs["specs"]][:1] +
            [sp["seed"] for sp in inputs["specs"]][-1:],
            "nodes_range": [min(w.n for w in ws), max(w.n for w in ws)],
            "porosity_range": [round(min(w.meta["porosity"] for w in ws), 4),
                               round(max(w.meta["porosity"] for w in ws), 4)],
            "s_cycle": [1.0, 0.5, 0.25], "g_cycle": [1e-6, 5e-6, 2e-5], "K": 16, "model": "MLBM1 (tau = 1)",
            "bounce_back": "interpolated", "node_updates_per_step": n,
            "l2": "working set ~6 GB > L2 (129 MB): steps timed back to back, no flush"}


# ---------------------------------------------------------------- reference
def oracle_sample_rate(args, inputs, n_sample, seed, min_seconds=0.0, max_reps=1, reps=None):
    """Time the oracle's step on a random sample of n_sample nodes of one
    sample of the workload (a sampled rate: the gathers of scattered targets
    miss cache more often than an in-order sweep would).  Runs exactly `reps`
    steps when given, else until min_seconds have passed (at most max_reps).
    Returns (Mnode-updates/s, threads, description, seconds per step)."""
    import oracle as O
    rng = np.random.default_rng(seed)
    if args.workload in ("karman_sweep", "lattice_compare"):
        w, s, model = inputs["karman"], 0.5, "bgk"
        what = f"the {w.n}-node vortex-street node set (Re = 100, s = 1/2)"
    elif args.workload == "porous_box":
        w, s, model = inputs["box"], BOX_S, "tau1"
        what = f"the porous box (seed {BOX_SEED}, {w.n} nodes, s = {BOX_S})"
    else:
        i = int(np.argsort([w.n for w in inputs["batch"]])[len(inputs["batch"]) // 2])
        w, s, model = inputs["batch"][i], inputs["specs"][i]["s"], "tau1"
        what = f"porous sample seed {inputs['specs'][i]['seed']} ({w.n} nodes, s = {s})"
    t = np.sort(rng.choice(w.n, size=min(n_sample, w.n), replace=False))
    op = O.Operator(w, K=16, s=s, bb_mode=0 if model == "bgk" else 1, targets=t).check()
    if model == "bgk":
        state = O.equilibrium(np.ones(w.n), 0.0, 0.0)
        step = lambda: O.bgk_step(op, state, tau_of(100, 0.5))
    else:
        state = np.zeros((w.n, 3))
        state[:, 0] = 1.0
        step = lambda: O.mlbm1_step(op, state, (1e-6, 0.0))
    per = []
    while (len(per) < reps) if reps is not None else (len(per) < max_reps and (sum(per) < min_seconds or not per)):
        t0 = time.perf_counter()
        step()
        per.append(time.perf_counter() - t0)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return (len(t) * len(per) / sum(per) / 1e6, threads,
            f"sampled rate: {len(t)} random nodes of {what} x {len(per)} steps", per)


def run_reference(args, rank, world):
    if rank != 0:
        return
    inputs = make_inputs(argparse.Namespace(**{**vars(args), "steady": False}), 0, 1)
    if args.workload == "karman_sweep":
        n = inputs["karman"].n * len(CASES)
    elif args.workload == "lattice_compare":
        n = inputs["karman"].n
    elif args.workload == "porous_box":
        n = inputs["box"].n
    else:
        n = sum(w.n for w in inputs["batch"])
    # a sample large enough for the oracle to use every host core
    oracle_sample_rate(args, inputs, ORACLE_SAMPLE, 0, reps=args.warmup)     # untimed warm-up steps
    value, threads, desc, per = oracle_sample_rate(args, inputs, ORACLE_SAMPLE, 0, reps=args.steps)
    total = sum(per)
    cfg = workload_config(args, inputs, None, n, 1)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- ours
def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the job's time is its slowest
    rank's); the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist, device):
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(nodes_per_rank, steps, world, ms):
    """Mnode-updates/s of the whole job when every rank advances the same
    number of node updates (weak scaling), timed by the slowest rank."""
    return nodes_per_rank * steps * world / (ms / 1e3) / 1e6


def job_rate(total_node_updates, ms):
    """Mnode-updates/s of the node updates of all ranks over the slowest
    rank's time."""
    return total_node_updates / (ms / 1e3) / 1e6


# the porous box to steady state: (s, g) of a Darcy and three inertial runs
BOX_STEADY = [(1.0, 1e-6), (0.5, 8e-5), (0.25, 2e-5), (0.125, 5e-6)]


def box_steady_legs(w, log):
    """The single porous box from rest to steady state (the criterion of the
    time-to-steady legs) at each (s, g) of BOX_STEADY: steps, seconds
    (context creation, run and observables), permeability in units of s^2
    and of the node spacing, tortuosity and the grain Reynolds numbers
    Re_d = U d / nu with d the mean disk diameter in units of s and U the
    superficial velocity (re_d) or the mean pore velocity (re_d_intrinsic)."""
    import torch
    from paper_2312_14789_gb300 import mlbm
    nu = (1.0 - 0.5) / 3.0
    d_mean = 2.0 * float(np.mean(w.disks[:, 2]))
    out = {"criterion": f"|u(t) - u(t-{WINDOW})| / ({WINDOW} |u(t)|) < {TOL:g}, checked every {CHECK} steps",
           "nodes": w.n, "node_areas": "uniform", "runs": []}
    for s, g in BOX_STEADY:
        st = mlbm.build_stencils_for(w, K=16, s=s, bb_mode=mlbm.BB_INTERPOLATED)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0))
        steps = mlbm.run_to_steady(ctx, TOL, WINDOW, 400_000, check=CHECK)
        pm = mlbm.permeability(ctx)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        out["runs"].append({"s": s, "g": g, "steps": int(steps), "seconds": sec, "mnups": w.n * steps / sec / 1e6,
                            "k": pm["k"], "k_node_spacing_units": pm["k"] * s * s,
                            "tortuosity": pm["tortuosity"], "re_d": pm["u_superficial"] * (d_mean / s) / nu,
                            "re_d_intrinsic": pm["u_intrinsic"] * (d_mean / s) / nu})
        log(f"box s = {s}: {steps} steps, {sec:.2f} s")
        del ctx, st
    return out


def steady_legs(inputs, log):
    """Time to steady state on held-out porous samples: cold single-instance,
    cold batched, learned warm start (batched and single), and the paper's
    criterion on the cold batch.  Everything runs through the C ABI; the
    network is trained here by the library's kernels."""
    import torch
    from paper_2312_14789_gb300 import mlbm
    from paper_2312_14789_gb300 import warmstart as W
    sync = torch.cuda.synchronize
    g = 1e-6
    test, train = inputs["steady_test"], inputs["steady_train"]
    out = {"criterion": f"|u(t) - u(t-{WINDOW})| / ({WINDOW} |u(t)|) < {TOL:g}, checked every {CHECK} steps",
           "samples": len(test), "nodes": [w.n for w in test], "s": 1.0, "g": g, "tau": 1.0,
           "seeds": [int(w.meta["seed"]) for w in test]}
    t0 = time.perf_counter()
    sts = W.build(test)
    out["stencil_build_s"] = time.perf_counter() - t0
    ps = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0) for _ in test]
    n_test = sum(w.n for w in test)

    # cold, single instance (the plain solver a user runs per sample)
    cold1 = []
    for st, p in zip(sts, ps):
        sync()
        t0 = time.perf_counter()
        ctx = mlbm.init(st, p)
        steps = mlbm.run_to_steady(ctx, TOL, WINDOW, 400_000, check=CHECK)
        k = mlbm.permeability(ctx)["k"]
        sync()
        cold1.append({"steps": steps, "s": time.perf_counter() - t0, "k": k})
        del ctx
    k_cold = np.array([r["k"] for r in cold1])
    out["cold_single"] = {"steps": [r["steps"] for r in cold1], "seconds_total": sum(r["s"] for r in cold1),
                          "mnups": sum(r["steps"] * w.n for r, w in zip(cold1, test)) /
                          sum(r["s"] for r in cold1) / 1e6}
    log(f"cold single: {out['cold_single']['seconds_total']:.2f} s")

    # cold, batched (all held-out samples in one context)
    ru_c, st_c, sec_c, k_c = W.solve(sts, ps, tol=TOL, window=WINDOW, check=CHECK)
    out["cold_batched"] = {"steps": [int(v) for v in st_c], "seconds": sec_c,
                           "mnups": n_test * int(max(st_c)) / sec_c / 1e6,
                           "k_rel_diff_vs_single_max": float(np.max(np.abs(k_c / k_cold - 1)))}
    log(f"cold batched: {sec_c:.2f} s")

    # learned warm start: training data from cold batched solves of the
    # training samples, then the network (velocity + density outputs)
    t0 = time.perf_counter()
    sts_tr = W.build(train)
    t_build_tr = time.perf_counter() - t0
    ps_tr = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0) for _ in train]
    ru_tr, steps_tr, sec_tr, _ = W.solve(sts_tr, ps_tr, tol=W.TRAIN_TOL, window=WINDOW, check=CHECK)
    del sts_tr
    X = W.features(train)
    T = torch.from_numpy(W.targets(train, ru_tr, ps_tr, 3)).cuda()
    net = mlbm.Mlp(7, 3)
    sync()
    t0 = time.perf_counter()
    losses = W.train(net, X, T, 8000, batch=65536)
    sync()
    t_train = time.perf_counter() - t0
    out["training"] = {"samples": len(train), "rows": int(X.shape[0]),
                       "nodes_mean": float(np.mean([w.n for w in train])), "seeds_first": int(train[0].meta["seed"]),
                       "cold_solve_s": sec_tr, "target_tol": W.TRAIN_TOL, "stencil_build_s": t_build_tr,
                       "adam_steps": 8000,
                       "train_s": t_train, "minibatch_loss_last": losses[-1]}
    del X, T
    sync()
    t0 = time.perf_counter()
    Xt = W.features(test)
    sync()
    t_feat = time.perf_counter() - t0
    t0 = time.perf_counter()
    ru_w, st_w, sec_w, k_w = W.solve(sts, ps, init=W.warm_init(net, Xt, test, ps), tol=TOL, window=WINDOW,
                                     check=CHECK)
    out["warm_batched"] = {"steps": [int(v) for v in st_w], "seconds": sec_w, "features_s": t_feat,
                           "steps_ratio_over_cold_mean": float(np.mean(np.asarray(st_w, float) /
                                                                      np.asarray(st_c, float))),
                           "seconds_ratio_over_cold": (sec_w + t_feat) / sec_c,
                           "k_rel_diff_vs_cold_max": float(np.max(np.abs(k_w / k_c - 1)))}
    log(f"warm batched: {sec_w:.2f} s")
    # learned warm start, single instance (features + inference + solve)
    warm1 = []
    for w, st, p in zip(test, sts, ps):
        sync()
        t0 = time.perf_counter()
        ctx = mlbm.init(st, p)
        Xi = W.features([w])
        L = W.length_scale(w)
        mlbm.warm_start(ctx, net, Xi.data_ptr(), W.velocity_scale(g, 1.0, L), W.density_scale(g, L))
        steps = mlbm.run_to_steady(ctx, TOL, WINDOW, 400_000, check=CHECK)
        k = mlbm.permeability(ctx)["k"]
        sync()
        warm1.append({"steps": steps, "s": time.perf_counter() - t0, "k": k})
        del ctx, Xi
    out["warm_single"] = {"steps": [r["steps"] for r in warm1], "seconds_total": sum(r["s"] for r in warm1),
                          "seconds_ratio_over_cold": sum(r["s"] for r in warm1) / out["cold_single"]["seconds_total"],
                          "k_rel_diff_vs_cold_max": float(np.max(np.abs(np.array([r["k"] for r in warm1]) /
                                                                        k_cold - 1)))}
    # the paper's criterion on the cold batch (Sec. 3.2)
    ctx = mlbm.batch_init(sts, ps)
    mlbm.autotune(ctx, 5)
    mlbm.set_fields(ctx, np.concatenate([np.column_stack([np.ones(w.n), np.zeros(w.n), np.zeros(w.n)])
                                         for w in test]))
    sync()
    t0 = time.perf_counter()
    st_p = mlbm.batch_run_to_steady_mean(ctx, PAPER_THRESHOLD, PAPER_DN, PAPER_CHECK, None, max_steps=1_000_000)
    sec_p = time.perf_counter() - t0
    k_p = mlbm.batch_permeability(ctx)["k"]
    out["paper_criterion_cold_batched"] = {
        "criterion": f"|<u>(t) - <u>(t-{PAPER_DN})| / (<u>(t-{PAPER_DN}) dt {PAPER_DN}) < {PAPER_THRESHOLD:g}, "
                     f"dt = nu (s/L)^2 (side 1, nu = 1), checked every {PAPER_CHECK} steps",
        "steps": [int(v) for v in st_p], "seconds": sec_p,
        "k_rel_diff_vs_field_norm_criterion_max": float(np.max(np.abs(k_p / k_c - 1)))}
    del ctx
    return out


def share_host_cores(world):
    """Ranks on one node split the host cores between them (stencil builds
    and the oracle use OpenMP; node generation uses worker processes);
    must run before torch or the library is loaded."""
    local = int(os.environ.get("LOCAL_WORLD_SIZE", world))
    per = max(1, (os.cpu_count() or 1) // max(local, 1))
    if local > 1 and "OMP_NUM_THREADS" not in os.environ:
        os.environ["OMP_NUM_THREADS"] = str(per)
    return per


def run_ours(args, rank, world, local_rank):
    t_setup0 = time.perf_counter()
    share_host_cores(world)
    inputs = make_inputs(args, rank, world)      # worker processes, before CUDA is touched
    t_gen = time.perf_counter() - t_setup0
    import torch
    from paper_2312_14789_gb300 import mlbm

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    log = (lambda m: print(m, file=sys.stderr, flush=True)) if rank == 0 else (lambda m: None)
    t0 = time.perf_counter()
    sts, params, model, distinct = build_batch(args, inputs)
    t_build = time.perf_counter() - t0
    infos = [mlbm.stencils_info(st) for st in sts]
    log(f"inputs {t_gen:.1f} s, stencils {t_build:.1f} s")
    t0 = time.perf_counter()
    if args.variant >= 0:
        order, variant, tune_ms = ORDER_NAMES.index(args.node_order), args.variant, None
        for st in distinct:
            mlbm.stencils_set_order(st, order)
        ctx = mlbm.batch_init(sts, params)
        mlbm.set_kernel_variant(ctx, variant)
    elif args.tune_order:
        order, variant, tune_ms = mlbm.autotune_order(sts, params, 5)
        ctx = mlbm.batch_init(sts, params)
        mlbm.set_kernel_variant(ctx, variant)
    else:
        order = ORDER_NAMES.index(args.node_order)
        for st in distinct:
            mlbm.stencils_set_order(st, order)
        ctx = mlbm.batch_init(sts, params)
        variant, tune_ms = mlbm.autotune(ctx, 5)
    tune_all = {str(v): round(ms, 4) for v, ms in mlbm.autotune_times(ctx).items()}
    stream = torch.cuda.Stream()
    mlbm.set_stream(ctx, stream.cuda_stream)
    # one-off setup before the timed region: both step graphs captured and
    # instantiated for the chosen variant and this stream
    mlbm.prepare_graphs(ctx)
    t_tune = time.perf_counter() - t0
    n = ctx.n
    with torch.cuda.stream(stream):
        mlbm.step(ctx, args.warmup)
    torch.cuda.synchronize()
    clocks = Clocks(local_rank) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    time.sleep(0.2 if clocks else 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        mlbm.step(ctx, args.steps)
        e1.record(stream)
    torch.cuda.synchronize()
    my_ms = float(e0.elapsed_time(e1))
    total_ms = max_over_ranks(my_ms, dist, "cuda")
    total_updates = sum_over_ranks(n * args.steps, dist, "cuda")
    if dist:
        dist.barrier()
    value = job_rate(total_updates, total_ms)

    # end to end through the public API with host buffers: upload every
    # sample's state from pinned memory, advance, read the fields and the
    # per-sample observables back
    e2e_steps = max(args.steps, 1)
    ru_host = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    ru_host[:] = mlbm.get_fields(ctx)
    out_host = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    mlbm.set_fields(ctx, ru_host)
    mlbm.step(ctx, e2e_steps)
    r = mlbm.lib().mlbm_get_fields(ctx.handle, out_host.ctypes.data)
    if model == "tau1":
        obs = mlbm.batch_permeability(ctx)["k"]
    else:
        obs = mlbm.batch_drag_lift(ctx, D, U0)["cd"]
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    assert r == 0
    e2e_value = total_updates / args.steps * e2e_steps / e2e_s / 1e6
    per_sample = [float(v) for v in obs]
    del ctx

    if dist is not None:
        gathered = [None] * world
        dist.all_gather_object(gathered, per_sample)
        if args.scaling == "strong" and inputs.get("assignment"):
            from paper_2312_14789_gb300 import shard
            per_sample = shard.merge_by_sample(gathered, inputs["assignment"], args.samples)
        else:
            per_sample = [v for part in gathered for v in part]
        dist.barrier()
    steady = None
    if rank == 0 and world == 1 and args.steady and args.workload == "porous_batch":
        steady = steady_legs(inputs, log)
    elif rank == 0 and world == 1 and args.steady and args.workload == "porous_box":
        steady = box_steady_legs(inputs["box"], log)
    clk = clocks.stop() if clocks else None
    if rank != 0:
        return
    pk, pk_kind = peaks()
    bytes_launch = sum(algorithmic_bytes(i, 16, model) for i in infos)
    avg_ms = my_ms / args.steps
    achieved = bytes_launch / (avg_ms / 1e3) / 1e9
    traffic = measured_traffic(args.workload, variant, order, n)
    cpu_val, cpu_threads, cpu_desc, _ = oracle_sample_rate(args, inputs, ORACLE_SAMPLE, 1, min_seconds=10.0,
                                                           max_reps=20000)
    cfg = dict(workload_config(args, inputs, infos, n, world), parallelism=(
        f"{world} ranks x own samples (weak)" if args.scaling == "weak" else f"{args.samples} samples split over "
        f"{world} ranks (strong)"), kernel_variant=variant, node_order=ORDER_NAMES[order],
        autotune_ms_per_step=tune_ms, autotune_ms_by_variant=tune_all or None, cuda_graph_chunk=16,
        n_wls=int(sum(i["n_wls"] for i in infos)), n_links=int(sum(i["n_links"] for i in infos)))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": args.scaling, "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "note": f"rank 0's step kernel: {bytes_launch} algorithmic bytes per launch "
                             f"({'473' if model == 'tau1' else '521'} B per least-squares node update); "
                             f"peak {pk_kind} burst copy"},
        "cpu_baseline": {"value": cpu_val, "unit": UNIT, "cores": cpu_threads, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 3 * 8 / e2e_steps,
                "d2h_bytes_per_step": (n * 3 * 8 + 8 * len(per_sample)) / e2e_steps,
                "note": f"set_fields from pinned host memory + {e2e_steps} steps + get_fields + per-sample "
                        f"{'permeability' if model == 'tau1' else 'drag'}, wall clock"},
        "gpu_launches": args.steps,
        "setup_s": {"inputs": t_gen, "stencils": t_build, "tune_and_graphs": t_tune},
        "clocks": clk,
        "per_sample_after_e2e": [round(v, 6) for v in per_sample][:8],
    }
    if steady is not None:
        out["time_to_steady"] = steady
    print(json.dumps(out))


# ------------------------------------------- lattice LBM vs meshless (Sec. 3.1)
LC_RE, LC_S, LC_EVERY = 100, 0.5, 50


def strouhal_of(cl, every, d_lb, u0):
    """St = f D / U0 from the mean spacing of the upward zero crossings of
    C_L - mean(C_L), interpolated linearly between samples; None with fewer
    than three crossings."""
    c = np.asarray(cl, np.float64) - np.mean(cl)
    i = np.nonzero((c[:-1] < 0) & (c[1:] >= 0))[0]
    if len(i) < 3:
        return None
    tz = (i + (-c[i]) / (c[i + 1] - c[i])) * every
    return float(d_lb / (np.mean(np.diff(tz)) * u0))


def lattice_compare_methods():
    """(name, node set, interpolant, K, weight rows) of the meshless runs."""
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm
    return [("meshless_scattered", I.karman(seed=2), mlbm.INTERP_WLS, 16, 6),
            ("meshless_hybrid", I.karman(seed=2, lattice_beyond_d=1.0), mlbm.INTERP_WLS, 16, 6),
            ("meshless_hybrid_coarse", I.karman(seed=2, lattice_beyond_d=1.0, coarse_beyond_d=2.0),
             mlbm.INTERP_WLS, 16, 6),
            ("meshless_scattered_rbf_points", I.karman(seed=2), mlbm.INTERP_RBF_POINTS, 64, 8)]


def run_lattice_compare(args, rank, local_rank):
    """The paper's comparison of lattice LBM and meshless LBM (Sec. 3.1) on
    one GPU.  The vortex street at Re = 100: the regular lattice with D = 80
    spacings (equilibrium sides, half-way bounce-back, the meshless step's
    FP32 collision) against the meshless step on node sets with D = 40 node
    spacings and s = 1/2, which take the same time step.  The node sets:
    scattered least squares; hybrid (Lagrange bulk beyond 1 D); coarsened
    hybrid (spacing 2 beyond 2 D); and the paper's RBF-FD interpolant with a
    stencil per Lagrangian point (the 25 nearest nodes).  Per method: time per
    step (CUDA events, `--steps` steps back to back after `--warmup`, variant
    from the autotuner), node updates per second, and, with --vortex-steps >
    0, the Strouhal number and mean drag over the second half of that many
    steps from rest (momentum exchange; for the meshless sets also the
    stress integrated along the cylinder's wall nodes).  `value` is the
    scattered least-squares rate.  Rank 0 only."""
    if rank != 0:
        return
    import torch
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm
    torch.cuda.set_device(local_rank)
    log = lambda m: print(m, file=sys.stderr, flush=True)
    u0, d = U0, D
    d_lb = d / LC_S
    tau = 3.0 * u0 * d_lb / LC_RE + 0.5
    p = mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0)
    n_rec = args.vortex_steps // LC_EVERY
    half = n_rec // 2
    comp = {}
    clocks = Clocks(local_rank)

    # lattice LBM
    cell, eqv = I.karman_lattice(d_lb, u0)
    lat = mlbm.Lattice(cell, p, periodic=(False, False), eq_values=eqv)
    lat.time_steps(args.warmup)
    us_lat = lat.time_steps(args.steps) * 1e3 / args.steps
    n_lat = int((cell != 1).sum())
    comp["lattice"] = {"cells": int(cell.size), "fluid_and_boundary_cells": n_lat, "us_per_step": us_lat,
                       "mnups": n_lat / us_lat, "algorithmic_bytes_per_step": int(cell.size) * 73}
    if n_rec:
        lat = mlbm.Lattice(cell, p, periodic=(False, False), eq_values=eqv)
        cd, cl = np.empty(n_rec), np.empty(n_rec)
        for i in range(n_rec):
            lat.step(LC_EVERY)
            fx, fy = lat.force()
            cd[i], cl[i] = 2 * fx / (u0 ** 2 * d_lb), 2 * fy / (u0 ** 2 * d_lb)
        comp["lattice"].update(strouhal=strouhal_of(cl[half:], LC_EVERY, d_lb, u0),
                               cd_mean=float(np.mean(cd[half:])), cl_amplitude=float(np.ptp(cl[half:]) / 2))
    del lat
    log(f"lattice: {us_lat:.2f} us/step")
    return lattice_compare_meshless(args, comp, p, tau, d_lb, n_rec, half, clocks, log)


def lattice_compare_meshless(args, comp, p, tau, d_lb, n_rec, half, clocks, log):
    """The meshless half of run_lattice_compare, then its JSON line."""
    import torch
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm
    u0, d = U0, D
    keep = {}
    for name, w, interp, K, rows in lattice_compare_methods():
        st = mlbm.build_stencils_for(w, K=K, s=LC_S, bb_mode=mlbm.BB_SIMPLE, interp=interp, n_l=25)
        info = mlbm.stencils_info(st)
        ctx = mlbm.init(st, p)
        variant, _ = mlbm.autotune(ctx, 5)
        stream = torch.cuda.Stream()
        mlbm.set_stream(ctx, stream.cuda_stream)
        mlbm.prepare_graphs(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            mlbm.step(ctx, args.warmup)
            e0.record(stream)
            mlbm.step(ctx, args.steps)
            e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / args.steps
        r = {"nodes": int(w.n), "n_lagrange": int(info["n_lagrange"]), "K": K, "variant": int(variant),
             "us_per_step": us, "mnups": w.n / us, "time_per_step_over_lattice": us / comp["lattice"]["us_per_step"],
             "algorithmic_bytes_per_step": int(algorithmic_bytes(info, K, "bgk", rows))}
        if n_rec:
            ctx = mlbm.init(st, p)
            mlbm.set_kernel_variant(ctx, variant)
            # the stress-integrated force needs the least-squares fit
            geo = I.wall_geometry(w) if interp == mlbm.INTERP_WLS else None
            cd, cl, cds = np.empty(n_rec), np.empty(n_rec), np.empty(n_rec)
            for i in range(n_rec):
                mlbm.step(ctx, LC_EVERY)
                _, _, cd[i], cl[i] = mlbm.drag_lift(ctx, d, u0)
                if geo is not None:
                    cds[i] = 2 * mlbm.wall_stress_force(ctx, *geo)[0] / (u0 ** 2 * d_lb)
            r.update(strouhal=strouhal_of(cl[half:], LC_EVERY, d_lb, u0), cd_mean=float(np.mean(cd[half:])),
                     cl_amplitude=float(np.ptp(cl[half:]) / 2),
                     cd_mean_stress=float(np.mean(cds[half:])) if geo is not None else None)
        comp[name] = r
        log(f"{name}: {us:.2f} us/step (variant {variant})")
        if name == "meshless_scattered":
            keep = {"w": w, "st": st, "info": info, "variant": variant, "us": us}
        del ctx, st
    clk = clocks.stop()
    # end to end on the scattered set: populations up from pinned memory,
    # the timed steps, populations and the drag back
    w, info = keep["w"], keep["info"]
    ctx = mlbm.init(keep["st"], p)
    mlbm.set_kernel_variant(ctx, keep["variant"])
    f_in = torch.empty((w.n, 9), dtype=torch.float64, pin_memory=True).numpy()
    f_in[:] = mlbm.get_populations(ctx)
    f_out = torch.empty((w.n, 9), dtype=torch.float64, pin_memory=True).numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mlbm.set_populations(ctx, f_in)
    mlbm.step(ctx, args.steps)
    assert mlbm.lib().mlbm_get_populations(ctx.handle, f_out.ctypes.data) == 0
    mlbm.drag_lift(ctx, d, u0)
    e2e_s = time.perf_counter() - t0
    del ctx
    pk, pk_kind = peaks()
    keep_bytes = comp["meshless_scattered"]["algorithmic_bytes_per_step"]
    achieved = keep_bytes / (keep["us"] * 1e-6) / 1e9
    cpu_val, cpu_threads, cpu_desc, _ = oracle_sample_rate(argparse.Namespace(workload="karman_sweep"),
                                                           {"karman": w}, ORACLE_SAMPLE, 1, min_seconds=10.0,
                                                           max_reps=20000)
    print(json.dumps({
        "metric": METRIC, "value": w.n / keep["us"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": keep["us"] / 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "karman_lattice_vs_meshless", "Re": LC_RE, "U0": u0, "D_node_spacings": d, "s": LC_S,
                   "D_lattice_spacings": d_lb, "tau": tau, "vortex_steps": args.vortex_steps,
                   "sample_every": LC_EVERY, "node_areas": "fluid-Voronoi", "bounce_back": "simple (meshless), "
                   "half-way (lattice)", "seed": 2,
                   "l2": "working sets of 33-134 MB, largely L2-resident: steps timed back to back, no flush; "
                         "these are latency numbers, not HBM fractions"},
        "comparison": comp,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": None,
                     "note": f"the scattered least-squares step: {keep_bytes} algorithmic bytes per launch "
                             f"(521 B per least-squares node update); the node set is L2-resident, so part of "
                             f"these bytes come from L2; peak {pk_kind} burst copy"},
        "cpu_baseline": {"value": cpu_val, "unit": UNIT, "cores": cpu_threads, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": w.n * args.steps / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": w.n * 72 / args.steps,
                "d2h_bytes_per_step": (w.n * 72 + 32) / args.steps,
                "note": f"set_populations from pinned host memory + {args.steps} steps + get_populations + drag, "
                        "wall clock, scattered set"},
        "gpu_launches": args.steps,
        "clocks": clk,
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="porous_batch", choices=["porous_batch", "karman_sweep", "porous_box", "lattice_compare"])
    ap.add_argument("--samples", type=int, default=64, help="porous samples per batch (64: the configuration)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"])
    ap.add_argument("--variant", type=int, default=-1,
                    help="fixed step kernel variant instead of the autotuner (-1: autotune)")
    ap.add_argument("--node-order", default="hilbert", choices=ORDER_NAMES)
    ap.add_argument("--tune-order", action="store_true", help="autotune the node order with the variant")
    ap.add_argument("--no-steady", dest="steady", action="store_false", help="skip the time-to-steady legs")
    ap.add_argument("--steady-samples", type=int, default=8)
    ap.add_argument("--train-samples", type=int, default=32)
    ap.add_argument("--train-nodes", type=int, default=100_000)
    ap.add_argument("--vortex-steps", type=int, default=200_000,
                    help="lattice_compare: steps from rest for the Strouhal number and drag (0: timing only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "lattice_compare":
        run_lattice_compare(args, rank, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
