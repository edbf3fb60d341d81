"""Benchmark of the fused MLBM step on the vortex-street configuration.

Workload: the Karman vortex street configuration as a whole -- a channel
22D x 4.1D around a cylinder of diameter D = 40 node spacings, ~260k
scattered Poisson-disk nodes refined near the cylinder (seed 2), K = 16
least-squares stencils, BGK in FP32, simple bounce-back on the cylinder,
equilibrium inflow/outflow/side nodes -- run for its six (Re, s) cases
Re in {100, 200} x streaming distance s in {1/2, 1/4, 1/8} node spacings
(D = 80, 160, 320 lattice units, U0 = 0.05, tau = 3 U0 D / Re + 1/2), all six
advanced together in one batched context (one fused launch per time step,
replayed from captured CUDA graphs).  One bench "step" = one time step of all
six runs = 6 x 259,971 node updates.  The working set (~780 MB) is larger
than L2, so consecutive steps are timed back to back without a flush.

Arms:
  default            the CUDA path through the C ABI (device-resident state)
  --impl reference   the FP64 CPU oracle on a bounded node sample (the
                     reference arm; no GPU)
  --variant V        a fixed step kernel variant (and --node-order) instead
                     of the autotuner, for profiler runs
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
U0, D = 0.05, 40.0
CASES = [(re, s) for re in (100, 200) for s in (0.5, 0.25, 0.125)]


def tau_of(re, s):
    return 3.0 * U0 * (D / s) / re + 0.5


WORKLOAD = {"workload": "karman_vortex_street_sweep", "runs": [{"Re": re, "s": s, "tau": round(tau_of(re, s), 4)}
                                                               for re, s in CASES],
            "nodes_per_run": None, "node_updates_per_step": None, "K": 16, "model": "BGK", "D_spacings": 40,
            "U0": U0, "seed": 2, "bounce_back": "simple",
            "l2": "working set ~780 MB > L2; steps timed back to back"}
TAU, S_STREAM = tau_of(100, 0.5), 0.5
PROFILE = os.path.join(ROOT, "profiles", "bgk_step_karman_sweep.md")


def algorithmic_bytes(info, K):
    """Bytes one fused step must move at minimum, per node kind: least-squares
    node 4*(9+9) populations + 4*6K matrix + 4K indices + 1 meta; Lagrange
    node 4*(9+9) + 4*12 indices + 4 (s/h) + 1; equilibrium node 16 + 36 + 1."""
    wls = 4 * 18 + 4 * 6 * K + 4 * K + 1
    lag = 4 * 18 + 4 * 12 + 4 + 1
    eq = 16 + 36 + 1
    return info["n_wls"] * wls + info["n_lagrange"] * lag + info["n_eq"] * eq


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "device_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2312_14789_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


ORDER_NAMES = ["hilbert", "morton", "rows", "input"]


def measured_traffic(variant, order=0):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when it was taken on a different kernel source, variant or node
    order."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != kernel_source_hash() or vals.get("kernel_variant") != str(variant) \
            or vals.get("node_order", "hilbert") != ORDER_NAMES[order]:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 6]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except ValueError:
                continue
            for nm, v in zip(names, r[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload():
    from paper_2312_14789_gb300 import inputs as I
    return I.karman(seed=2)


def oracle_sample_rate(w, n_sample, seed, min_seconds, max_reps):
    """Time the oracle's BGK step on n_sample nodes of the workload; returns
    (Mnode-updates/s, threads, description)."""
    import oracle as O
    rng = np.random.default_rng(seed)
    t = np.sort(rng.choice(w.n, size=n_sample, replace=False))
    op = O.Operator(w, K=16, s=S_STREAM, bb_mode=0, targets=t).check()
    f = O.equilibrium(np.ones(w.n), 0.0, 0.0)
    reps, elapsed = 0, 0.0
    while reps < max_reps and (elapsed < min_seconds or reps == 0):
        t0 = time.perf_counter()
        O.bgk_step(op, f, TAU)
        elapsed += time.perf_counter() - t0
        reps += 1
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n_sample * reps / elapsed / 1e6, threads, f"{n_sample} random nodes of the {w.n}-node workload x {reps} steps"


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = make_workload()
    per_step = []
    import oracle as O
    rng = np.random.default_rng(0)
    n_sample = 4096
    t = np.sort(rng.choice(w.n, size=n_sample, replace=False))
    op = O.Operator(w, K=16, s=S_STREAM, bb_mode=0, targets=t).check()
    f = O.equilibrium(np.ones(w.n), 0.0, 0.0)
    # one of the six runs (Re = 100, s = 1/2); the others cost the same per node
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.bgk_step(op, f, TAU)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            per_step.append(dt)
    total = sum(per_step)
    value = n_sample * args.steps / total / 1e6
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cfg = dict(WORKLOAD, nodes_per_run=w.n, node_updates_per_step=w.n * len(CASES))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n_sample} random nodes of the {w.n}-node vortex-street node set (Re=100, s=1/2) per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the job's time is its slowest
    rank's); the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(nodes_per_rank, steps, world, ms):
    """Mnode-updates/s of the whole job: every rank advances its own replica
    of the workload (weak scaling), timed by the slowest rank."""
    return nodes_per_rank * steps * world / (ms / 1e3) / 1e6


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2312_14789_gb300 import mlbm

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = make_workload()
    st_by_s = {s: mlbm.build_stencils_for(w, K=16, s=s, bb_mode=mlbm.BB_SIMPLE) for s in sorted({s for _, s in CASES})}
    sts = [st_by_s[s] for _, s in CASES]
    params = [mlbm.Params(mlbm.MODEL_BGK, tau_of(re, s), 0.0, 0.0, 0.0) for re, s in CASES]
    infos = [mlbm.stencils_info(st) for st in sts]
    if args.variant >= 0:
        # fixed choice (for profiler runs, where the tuner's timings are distorted)
        order, variant, tune_ms = ORDER_NAMES.index(args.node_order), args.variant, None
        for st in st_by_s.values():
            mlbm.stencils_set_order(st, order)
    else:
        # node order and kernel variant picked together by the library's autotuner
        order, variant, tune_ms = mlbm.autotune_order(sts, params, 10)
    ctx = mlbm.batch_init(sts, params)
    mlbm.set_kernel_variant(ctx, variant)
    stream = torch.cuda.Stream()
    mlbm.set_stream(ctx, stream.cuda_stream)
    n = ctx.n
    with torch.cuda.stream(stream):
        mlbm.step(ctx, args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    with torch.cuda.stream(stream):
        e0.record(stream)
        mlbm.step(ctx, args.steps)
        e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(float(e0.elapsed_time(e1)), dist, "cuda")
    if dist:
        dist.barrier()
    value = whole_job_rate(n, args.steps, world, total_ms)

    # end to end through the public API with host buffers: upload the state
    # of all six runs from pinned memory, advance, read the fields and the
    # per-run cylinder forces back
    e2e_steps = max(args.steps, 1)
    f_host = torch.empty((n, 9), dtype=torch.float64, pin_memory=True).numpy()
    f_host[:] = mlbm.get_populations(ctx)
    ru_host = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mlbm.set_populations(ctx, f_host)
    mlbm.step(ctx, e2e_steps)
    r = mlbm.lib().mlbm_get_fields(ctx.handle, ru_host.ctypes.data)
    forces = mlbm.batch_drag_lift(ctx, D, U0)
    e2e_s = time.perf_counter() - t0
    assert r == 0
    e2e_value = n * e2e_steps * world / e2e_s / 1e6

    if rank != 0:
        return
    pk, pk_kind = peaks()
    bytes_launch = sum(algorithmic_bytes(i, 16) for i in infos)
    avg_ms = total_ms / args.steps
    achieved = bytes_launch / (avg_ms / 1e3) / 1e9
    traffic = measured_traffic(variant, order)
    cpu_val, cpu_threads, cpu_desc = oracle_sample_rate(w, 8192, 1, 10.0, 20000)
    cfg = dict(WORKLOAD, nodes_per_run=w.n, node_updates_per_step=n, parallelism=f"replicas x{world}",
               n_wls=int(sum(i["n_wls"] for i in infos)), n_eq=int(sum(i["n_eq"] for i in infos)),
               n_links=int(sum(i["n_links"] for i in infos)), kernel_variant=variant, node_order=ORDER_NAMES[order],
               autotune_ms_per_step=tune_ms, cuda_graph_chunk=16)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "note": f"algorithmic bytes {bytes_launch} per launch; peak {pk_kind} (burst copy)"},
        "cpu_baseline": {"value": cpu_val, "unit": UNIT, "cores": cpu_threads, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 9 * 8 / e2e_steps,
                "d2h_bytes_per_step": (n * 3 * 8 + 4 * 8 * len(CASES)) / e2e_steps,
                "note": f"set_populations from pinned host memory + {e2e_steps} steps + get_fields + batch_drag_lift"},
        "gpu_launches": args.steps,
        "clocks": clk,
        "cd_after_e2e": [round(float(v), 4) for v in forces["cd"]],
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", type=int, default=-1,
                    help="fixed step kernel variant instead of the autotuner (-1: autotune)")
    ap.add_argument("--node-order", default="hilbert", choices=ORDER_NAMES,
                    help="node order used with --variant")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
