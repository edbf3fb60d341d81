"""Measurement studies beyond the single-workload benchmark.

    python -m paper_2312_14789_gb300.studies batch [--samples 64] [--steps 20]
    python -m paper_2312_14789_gb300.studies warm [--train 512] [--test 64] [--nodes 200000]
    python -m paper_2312_14789_gb300.studies hybrid [--steps 200000] [--lattice-d 1.0]
    python -m paper_2312_14789_gb300.studies porous [--nodes 1000000]
    python -m paper_2312_14789_gb300.studies lbm [--steps 200000]
    python -m paper_2312_14789_gb300.studies rbf [--steps 200000]
    python -m paper_2312_14789_gb300.studies kernels [--nodes 1000000]

batch: 64 porous samples (seeds 1000..1063) with node counts U(50k, 400k),
porosity U(0.5, 0.85) and a mix of Darcy (s = 1) and inertial (s = 1/2, 1/4)
streaming distances, tau = 1 (MLBM1), K = 16, interpolated bounce-back.
Reports the aggregate node-updates/s of the batched context (all samples in
the same launches, CUDA-graph replay) against the sum of sequential
single-instance runs of the same samples, each timed with CUDA events.

warm: learned warm start.  Porous samples (porosity 0.7, radii U(8, 16),
seeds 10000.. for training and 20000.. held out), MLBM1 (tau = 1), s = 1,
K = 16, interpolated bounce-back, body force g = 1e-6 along x (Darcy).
Training samples are solved from rest to steady state (|u(t) - u(t-1000)| /
(1000 |u(t)|) < 1e-7) in batches, stencil builds of the next batch
overlapping the solves; the network is trained on their features and
normalised steady velocities; the held-out samples are then solved from rest,
from the network's prediction and from a uniform Kozeny-Carman estimate.
Reports steps and seconds to steady state, permeability differences against
the cold start and the prediction error.

Each study prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _sample_spec(i):
    rng = np.random.default_rng(1000 + i)
    n = int(rng.uniform(50_000, 400_000))
    phi = float(rng.uniform(0.5, 0.85))
    s = [1.0, 0.5, 0.25][i % 3]
    g = [1e-6, 5e-6, 2e-5][i % 3]
    return {"seed": 1000 + i, "n_target": n, "porosity": phi, "s": s, "g": g}


def _make(spec):
    from paper_2312_14789_gb300 import inputs as I
    # porosity below ~0.55 is out of reach for non-overlapping disks with a
    # 2-spacing gap; the sampler then keeps the porosity it reached
    w = I.porous(seed=spec["seed"], n_target=spec["n_target"], porosity=spec["porosity"],
                 gap=1.0 if spec["porosity"] < 0.6 else 2.0)
    return w


def batch_study(args):
    import torch
    from paper_2312_14789_gb300 import mlbm

    specs = [_sample_spec(i) for i in range(args.samples)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        ws = pool.map(_make, specs)
    t_gen = time.time() - t0
    t0 = time.time()
    sts = [mlbm.build_stencils_for(w, K=16, s=sp["s"], bb_mode=mlbm.BB_INTERPOLATED) for w, sp in zip(ws, specs)]
    t_build = time.time() - t0
    ps = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, sp["g"], 0.0) for sp in specs]
    n_tot = sum(w.n for w in ws)

    def timed(ctx, steps):
        st = torch.cuda.Stream()
        mlbm.set_stream(ctx, st.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            mlbm.step(ctx, 16)
            e0.record(st)
            mlbm.step(ctx, steps)
            e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    # node order: time every order (stencils re-ordered, variants tuned), then
    # let the library's order autotuner pick
    order_ms = {}
    for o, name in enumerate(["hilbert", "morton", "rows", "input"]):
        for st in sts:
            mlbm.stencils_set_order(st, o)
        b = mlbm.batch_init(sts, ps)
        _, order_ms[name] = mlbm.autotune(b, 5)
        del b
    order, variant, _ = mlbm.autotune_order(sts, ps, 5)
    batch = mlbm.batch_init(sts, ps)
    mlbm.set_kernel_variant(batch, variant)
    t_batch = timed(batch, args.steps)
    k_batch = mlbm.batch_permeability(batch)["k"]
    del batch
    t_seq = 0.0
    variants = []
    k_single = []
    for st, p in zip(sts, ps):
        ctx = mlbm.init(st, p)
        v, _ = mlbm.autotune(ctx, 5)
        variants.append(v)
        t_seq += timed(ctx, args.steps)
        k_single.append(mlbm.permeability(ctx)["k"])
        del ctx
    k_single = np.array(k_single)
    out = {
        "study": "batch", "samples": args.samples, "nodes_total": n_tot, "steps": args.steps,
        "batched_mnups": n_tot * args.steps / t_batch / 1e6,
        "sequential_mnups": n_tot * args.steps / t_seq / 1e6,
        "speedup": t_seq / t_batch, "batch_variant": variant, "batch_node_order": order,
        "autotune_ms_per_step_by_order": order_ms,
        "single_variants": sorted(set(variants)),
        "permeability_max_rel_diff_batch_vs_single": float(np.max(np.abs(k_batch - k_single) / np.abs(k_single))),
        "porosity_range": [float(min(w.meta["porosity"] for w in ws)), float(max(w.meta["porosity"] for w in ws))],
        "node_range": [min(w.n for w in ws), max(w.n for w in ws)],
        "generate_s": t_gen, "stencil_build_s": t_build,
        "algorithmic_bytes_per_step": sum(32 + 24 * 16 + 4 * 16 + 1 for _ in range(1)) * n_tot,
    }
    out["hbm_gbs_batched"] = out["algorithmic_bytes_per_step"] / (t_batch / args.steps) / 1e9
    print(json.dumps(out))


def warm_study(args):
    import concurrent.futures as cf

    import torch
    from paper_2312_14789_gb300 import mlbm
    from paper_2312_14789_gb300 import warmstart as W

    log = (lambda m: print(m, file=sys.stderr, flush=True))
    t_all = time.time()
    train_seeds = list(range(10000, 10000 + args.train))
    test_seeds = list(range(20000, 20000 + args.test))
    t0 = time.time()
    ws_train = W.make_samples(train_seeds, args.nodes)
    ws_test = W.make_samples(test_seeds, args.nodes)
    t_gen = time.time() - t0
    log(f"generated {len(ws_train)} + {len(ws_test)} samples in {t_gen:.1f} s")
    par = lambda ws: [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, args.g, 0.0) for _ in ws]

    # ---- training data: batched cold solves, next group's stencils built meanwhile
    groups = [ws_train[i:i + args.group] for i in range(0, len(ws_train), args.group)]
    X_parts, T_parts, train_steps = [], [], []
    t_solve = t_build = 0.0
    with cf.ThreadPoolExecutor(1) as ex:
        def timed_build(ws):
            t = time.time()
            return W.build(ws), time.time() - t
        fut = ex.submit(timed_build, groups[0])
        for gi, ws in enumerate(groups):
            sts, tb = fut.result()
            t_build += tb
            if gi + 1 < len(groups):
                fut = ex.submit(timed_build, groups[gi + 1])
            ps = par(ws)
            ru, steps, sec, _ = W.solve(sts, ps)
            t_solve += sec
            train_steps += list(steps)
            X_parts.append(W.features(ws))
            T_parts.append(torch.from_numpy(W.targets(ws, ru, ps, 3)).cuda())
            del sts
            log(f"group {gi}: {sum(w.n for w in ws)} nodes, steps {int(np.mean(steps))} mean, {sec:.1f} s")
    X = torch.cat(X_parts)
    T = torch.cat(T_parts)
    del X_parts, T_parts
    n_rows = X.shape[0]

    # ---- training: a velocity-only network (2 outputs) and a velocity +
    # density network (3 outputs) on the same rows
    T2 = T[:, :2].contiguous()
    t_var = {"velocity": float(((T2 - T2.mean(0)) ** 2).sum(1).mean()),
             "density": float(((T[:, 2] - T[:, 2].mean()) ** 2).mean())}
    nets, train_info = {}, {}
    for no, TT in ((2, T2), (3, T)):
        net = mlbm.Mlp(args.seed, no)
        l0 = net.gradients(X.data_ptr(), TT.data_ptr(), n_rows)
        torch.cuda.synchronize()
        t0 = time.time()
        losses = W.train(net, X, TT, args.steps, batch=args.batch, log=log)
        torch.cuda.synchronize()
        train_info[no] = {"seconds": time.time() - t0, "loss_initial": l0, "minibatch_losses": losses,
                          "loss_final": net.gradients(X.data_ptr(), TT.data_ptr(), n_rows)}
        nets[no] = net
        if args.save:
            np.save(f"{args.save}_out{no}.npy", net.get_params())
    del X, T, T2

    # ---- held-out samples: cold, learned warm (2 and 3 outputs), Kozeny
    sts = W.build(ws_test)
    ps = par(ws_test)
    Xt = W.features(ws_test)
    ru_c, st_c, sec_c, k_c = W.solve(sts, ps)
    ru_2, st_2, sec_2, k_2 = W.solve(sts, ps, init=W.warm_init(nets[2], Xt, ws_test, ps))
    ru_3, st_3, sec_3, k_3 = W.solve(sts, ps, init=W.warm_init(nets[3], Xt, ws_test, ps))
    ru_k, st_k, sec_k, k_k = W.solve(sts, ps, init=W.kozeny_init(ws_test, ps))
    # prediction error of the initial state against the converged cold state
    Yd = torch.empty((Xt.shape[0], 3), dtype=torch.float32, device="cuda")
    nets[3].forward(Xt.data_ptr(), Xt.shape[0], Yd.data_ptr())
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.float64)
    err_u, err_r, o = [], [], 0
    for w, p in zip(ws_test, ps):
        L = W.length_scale(w)
        u = ru_c[o:o + w.n, 1:]
        err_u.append(float(np.linalg.norm(W.velocity_scale(p.gx, p.tau, L) * Y[o:o + w.n, :2] - u) / np.linalg.norm(u)))
        dr = ru_c[o:o + w.n, 0] - 1.0
        pr = W.density_scale(p.gx, L) * Y[o:o + w.n, 2]
        pr = pr - np.sum(pr * w.area) / np.sum(w.area)
        err_r.append(float(np.linalg.norm(pr - dr) / np.linalg.norm(dr)))
        o += w.n
    # single-instance time to steady state (what one user run sees), first
    # samples; the warm start's time includes features and inference
    single = []
    for i in range(min(args.single, len(ws_test))):
        row = {}
        for mode in ("cold", "warm"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = mlbm.init(sts[i], ps[i])
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if mode == "warm":
                Xi = W.features([ws_test[i]])
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                L = W.length_scale(ws_test[i])
                mlbm.warm_start(ctx, nets[3], Xi.data_ptr(), W.velocity_scale(args.g, 1.0, L), W.density_scale(args.g, L))
                torch.cuda.synchronize()
                row["features_s"] = t2 - t1
                row["inference_and_set_s"] = time.perf_counter() - t2
            t3 = time.perf_counter()
            taken = mlbm.run_to_steady(ctx, W.TOL, W.WINDOW, 400_000, check=W.CHECK)
            torch.cuda.synchronize()
            row[mode + "_solve_s"] = time.perf_counter() - t3
            row[mode + "_s"] = time.perf_counter() - t1
            row[mode + "_steps"] = int(taken)
            row[mode + "_k"] = mlbm.permeability(ctx)["k"]
            del ctx
        single.append(row)
    rel = lambda a, b: np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))
    mean_ratio = lambda a, b: float(np.mean(np.asarray(a, float) / np.asarray(b, float)))
    out = {
        "study": "warm", "train_samples": len(ws_train), "test_samples": len(ws_test),
        "nodes_mean": float(np.mean([w.n for w in ws_train + ws_test])), "train_rows": int(n_rows),
        "g": args.g, "tol": W.TOL, "window": W.WINDOW, "check_every": W.CHECK,
        "train_steps_to_steady_mean": float(np.mean(train_steps)),
        "mlp_steps": args.steps, "mlp_batch": args.batch, "target_variance": t_var,
        "training": {f"outputs_{k}": v for k, v in train_info.items()},
        "test_steps_mean": {"cold": float(np.mean(st_c)), "warm_velocity": float(np.mean(st_2)),
                            "warm_velocity_density": float(np.mean(st_3)), "kozeny": float(np.mean(st_k))},
        "test_steps_ratio_over_cold": {"warm_velocity": mean_ratio(st_2, st_c),
                                       "warm_velocity_density": mean_ratio(st_3, st_c),
                                       "kozeny": mean_ratio(st_k, st_c)},
        "test_steps": {"cold": [int(v) for v in st_c], "warm_velocity": [int(v) for v in st_2],
                       "warm_velocity_density": [int(v) for v in st_3]},
        "test_batch_seconds": {"cold": sec_c, "warm_velocity": sec_2, "warm_velocity_density": sec_3,
                               "kozeny": sec_k},
        "k_rel_diff_vs_cold_max": {"warm_velocity": float(rel(k_2, k_c).max()),
                                   "warm_velocity_density": float(rel(k_3, k_c).max()),
                                   "kozeny": float(rel(k_k, k_c).max())},
        "prediction_rel_l2_mean": {"velocity": float(np.mean(err_u)), "density": float(np.mean(err_r))},
        "single_instance": single,
        "seconds": {"generate": t_gen, "stencil_build": t_build, "train_solves": t_solve,
                    "total": time.time() - t_all},
    }
    print(json.dumps(out))


def _strouhal(cl, every, d_lb, u0):
    """St = f D / U0 from the mean spacing of upward zero crossings of
    C_L - mean(C_L) (linear interpolation between samples)."""
    c = np.asarray(cl, np.float64) - np.mean(cl)
    i = np.nonzero((c[:-1] < 0) & (c[1:] >= 0))[0]
    if len(i) < 3:
        return float("nan")
    tz = (i + (-c[i]) / (c[i + 1] - c[i])) * every
    return float(d_lb / (np.mean(np.diff(tz)) * u0))


def hybrid_study(args):
    """Scattered vs hybrid (lattice bulk beyond --lattice-d diameters of the
    cylinder surface, scattered refinement inside) vortex street at Re = 100,
    s = 1/2: step throughput (autotuned, CUDA events, graphs), HBM fraction of
    the algorithmic bytes, and the Strouhal number and mean drag after
    --steps steps from rest."""
    import torch
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm
    sys.path.insert(0, ROOT)
    import bench

    re_, s_, u0, d = 100, 0.5, 0.05, 40.0
    tau = 3.0 * u0 * (d / s_) / re_ + 0.5
    peak = bench.peaks()[0]["hbm_gbs"]
    out = {"study": "hybrid", "Re": re_, "s": s_, "tau": tau, "steps": args.steps}
    for name, w in (("scattered", I.karman(seed=2)), ("hybrid", I.karman(seed=2, lattice_beyond_d=args.lattice_d))):
        st = mlbm.build_stencils_for(w, K=16, s=s_, bb_mode=mlbm.BB_SIMPLE)
        info = mlbm.stencils_info(st)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0))
        variant, _ = mlbm.autotune(ctx, 10, flush_l2=True)
        stream = torch.cuda.Stream()
        mlbm.set_stream(ctx, stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            mlbm.step(ctx, 32)
            e0.record(stream)
            mlbm.step(ctx, 2048)
            e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / 2048
        alg = bench.algorithmic_bytes(info, 16)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0))
        mlbm.set_kernel_variant(ctx, variant)
        every = 50
        cd, cl = np.empty(args.steps // every), np.empty(args.steps // every)
        for i in range(len(cd)):
            mlbm.step(ctx, every)
            _, _, cd[i], cl[i] = mlbm.drag_lift(ctx, d, u0)
        h = len(cd) // 2
        out[name] = {"nodes": int(w.n), "n_wls": info["n_wls"], "n_lagrange": info["n_lagrange"],
                     "n_eq": info["n_eq"], "variant": variant, "us_per_step": us,
                     "mnups": w.n / us, "algorithmic_bytes_per_step": alg,
                     "hbm_frac_of_measured_peak": alg / (us * 1e-6) / 1e9 / peak,
                     "strouhal": _strouhal(cl[h:], every, d / s_, u0), "cd_mean": float(np.mean(cd[h:])),
                     "cl_amplitude": float(np.ptp(cl[h:]) / 2)}
    out["time_per_step_ratio_hybrid_over_scattered"] = out["hybrid"]["us_per_step"] / out["scattered"]["us_per_step"]
    print(json.dumps(out))


def porous_study(args):
    """The ~1M-node porous box (porosity 0.7, radii U(8, 16), seed 3), tau = 1
    (MLBM1), K = 16, interpolated bounce-back, from rest to steady state:
    Darcy (s = 1, g = 1e-6) and faster flows at smaller streaming distances
    (s = 1/2, 1/4, 1/8 with g chosen for a pore velocity of ~0.03, Re_d ~ 10-40).  Reports the
    permeability, the pore Reynolds number Re_d = U_intrinsic d / nu (d the
    mean disk diameter in lattice units d/s), steps and seconds to steady
    state, the step throughput (autotuned, CUDA events) and its fraction of
    the HBM roofline (481 algorithmic bytes per node-update)."""
    import torch
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm
    sys.path.insert(0, ROOT)
    import bench

    w = I.porous(seed=3, n_target=args.nodes, porosity=0.7, areas=args.areas)
    d_mean = float(2 * w.disks[:, 2].mean())
    peak = bench.peaks()[0]["hbm_gbs"]
    out = {"study": "porous", "nodes": int(w.n), "porosity": w.meta["porosity"], "disks": int(len(w.disks)),
           "node_areas": args.areas,
           "runs": []}
    for s_, g in ((1.0, 1e-6), (0.5, 8e-5), (0.25, 2e-5), (0.125, 5e-6)):
        st = mlbm.build_stencils_for(w, K=16, s=s_, bb_mode=mlbm.BB_INTERPOLATED)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0))
        variant, _ = mlbm.autotune(ctx, 10, flush_l2=True)
        stream = torch.cuda.Stream()
        mlbm.set_stream(ctx, stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            mlbm.step(ctx, 32)
            e0.record(stream)
            mlbm.step(ctx, 512)
            e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / 512
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0))
        mlbm.set_kernel_variant(ctx, variant)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps = mlbm.run_to_steady(ctx, 1e-7, 1000, 2_000_000, check=100)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        pm = mlbm.permeability(ctx)
        nu = 0.5 / 3.0
        out["runs"].append({"s": s_, "g": g, "variant": variant, "us_per_step": us, "mnups": w.n / us,
                            "hbm_frac_of_measured_peak": w.n * 481 / (us * 1e-6) / 1e9 / peak,
                            "steps_to_steady": int(steps), "seconds_to_steady": sec,
                            "mnups_to_steady": w.n * steps / sec / 1e6,
                            "k": pm["k"], "u_intrinsic": pm["u_intrinsic"], "tortuosity": pm["tortuosity"],
                            "Re_d": pm["u_intrinsic"] * (d_mean / s_) / nu})
        print(json.dumps(out["runs"][-1]), file=sys.stderr, flush=True)
    print(json.dumps(out))


def lattice_karman(d_lb, u0=0.05, length_d=22.0, height_d=4.1, center_d=(2.0, 2.0)):
    """Cells of the vortex-street channel on a regular lattice: D = d_lb
    spacings, equilibrium cells on the four sides (parabolic inflow and
    outflow with maximum u0, rest on the top and bottom), solid cells whose
    centre lies inside the cylinder."""
    nx, ny = int(round(length_d * d_lb)), int(round(height_d * d_lb))
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cx, cy, r = center_d[0] * d_lb, center_d[1] * d_lb, 0.5 * d_lb
    cell = np.zeros((ny, nx), np.uint8)
    cell[(x - cx) ** 2 + (y - cy) ** 2 < r * r] = 1
    side = (x == 0) | (x == nx - 1) | (y == 0) | (y == ny - 1)
    cell[side] = 2
    eqv = np.zeros((ny, nx, 3))
    eqv[..., 0] = 1.0
    h = ny - 1.0
    lr = (x == 0) | (x == nx - 1)
    eqv[..., 1] = np.where(lr & ~((y == 0) | (y == ny - 1)), 4.0 * u0 * y * (h - y) / (h * h), 0.0)
    return cell, eqv


def lbm_study(args):
    """The paper's comparison, lattice LBM vs meshless LBM (Sec. 3.1), on
    GB300: the vortex street at Re = 100 on the regular lattice with D = 80
    spacings (the lattice resolution of the meshless run with D = 40 node
    spacings and s = 1/2, so both take the same time step) against the
    meshless step on the scattered, the hybrid and the coarsened hybrid
    (spacing 2 beyond 2 D) node sets.  Per method:
    nodes, time per step (CUDA events, back to back), algorithmic bytes per
    step, Strouhal number and mean drag over the second half of --steps (for
    the meshless sets from the momentum exchange and from the stress
    integrated along the cylinder's wall nodes)."""
    import torch
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm

    re_, u0, d = 100, 0.05, 40.0
    s_ = 0.5
    d_lb = d / s_
    tau = 3.0 * u0 * d_lb / re_ + 0.5
    every = 50
    out = {"study": "lbm", "Re": re_, "D_lattice_units": d_lb, "tau": tau, "steps": args.steps,
           "node_areas": args.areas}

    def timed(step_fn, stream, n=2048):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            step_fn(32)
            e0.record(stream)
            step_fn(n)
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / n

    # lattice LBM
    cell, eqv = lattice_karman(d_lb, u0)
    lat = mlbm.Lattice(cell, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0), periodic=(False, False), eq_values=eqv)
    lat.time_steps(32)
    us_lat = lat.time_steps(2048) * 1e3 / 2048
    lat = mlbm.Lattice(cell, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0), periodic=(False, False), eq_values=eqv)
    cd, cl = np.empty(args.steps // every), np.empty(args.steps // every)
    for i in range(len(cd)):
        lat.step(every)
        fx, fy = lat.force()
        cd[i], cl[i] = 2 * fx / (u0 ** 2 * d_lb), 2 * fy / (u0 ** 2 * d_lb)
    h = len(cd) // 2
    n_lat = int((cell != 1).sum())
    out["lattice"] = {"cells": int(cell.size), "fluid_and_boundary_cells": n_lat, "us_per_step": us_lat,
                      "mnups": n_lat / us_lat, "algorithmic_bytes_per_step": int(cell.size) * 73,
                      "strouhal": _strouhal(cl[h:], every, d_lb, u0), "cd_mean": float(np.mean(cd[h:])),
                      "cl_amplitude": float(np.ptp(cl[h:]) / 2)}
    print(json.dumps(out["lattice"]), file=sys.stderr, flush=True)
    # meshless on the scattered and the hybrid node sets
    for name, w in (("meshless_scattered", I.karman(seed=2, areas=args.areas)),
                    ("meshless_hybrid", I.karman(seed=2, lattice_beyond_d=1.0, areas=args.areas)),
                    ("meshless_hybrid_coarse", I.karman(seed=2, lattice_beyond_d=1.0, coarse_beyond_d=2.0,
                                                        areas=args.areas))):
        st = mlbm.build_stencils_for(w, K=16, s=s_, bb_mode=mlbm.BB_SIMPLE)
        info = mlbm.stencils_info(st)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0))
        variant, _ = mlbm.autotune(ctx, 10)
        stream = torch.cuda.Stream()
        mlbm.set_stream(ctx, stream.cuda_stream)
        us = timed(lambda k: mlbm.step(ctx, k), stream)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0))
        mlbm.set_kernel_variant(ctx, variant)
        geo = I.wall_geometry(w)
        cd_st, cl_st = np.empty(len(cd)), np.empty(len(cd))
        for i in range(len(cd)):
            mlbm.step(ctx, every)
            _, _, cd[i], cl[i] = mlbm.drag_lift(ctx, d, u0)
            fx, fy = mlbm.wall_stress_force(ctx, *geo)
            cd_st[i], cl_st[i] = 2 * fx / (u0 ** 2 * d_lb), 2 * fy / (u0 ** 2 * d_lb)
        import bench
        out[name] = {"nodes": int(w.n), "n_lagrange": info["n_lagrange"], "variant": variant, "us_per_step": us,
                     "mnups": w.n / us, "algorithmic_bytes_per_step": int(bench.algorithmic_bytes(info, 16)),
                     "strouhal": _strouhal(cl[h:], every, d_lb, u0), "cd_mean": float(np.mean(cd[h:])),
                     "cl_amplitude": float(np.ptp(cl[h:]) / 2),
                     "cd_mean_stress": float(np.mean(cd_st[h:])), "cl_amplitude_stress": float(np.ptp(cl_st[h:]) / 2),
                     "strouhal_stress": _strouhal(cl_st[h:], every, d_lb, u0)}
        print(json.dumps(out[name]), file=sys.stderr, flush=True)
    for name in ("meshless_scattered", "meshless_hybrid", "meshless_hybrid_coarse"):
        out[name]["time_per_step_over_lattice"] = out[name]["us_per_step"] / out["lattice"]["us_per_step"]
    print(json.dumps(out))


def rbf_study(args):
    """The paper's RBF-FD interpolant against the least-squares fit on the
    vortex street (Re = 100, s = 1/2, scattered node set, fluid-Voronoi
    areas): step time with the L2 flushed before every step (autotuned), its
    fraction of the HBM roofline (algorithmic bytes: 4 (9 + 9) + 32 K + 4 K + 1
    per RBF-FD node, 4 (9 + 9) + 24 K + 4 K + 1 per least-squares node), and
    the Strouhal number and mean drag after --steps steps from rest."""
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm
    sys.path.insert(0, ROOT)
    import bench

    re_, s_, u0, d = 100, 0.5, 0.05, 40.0
    tau = 3.0 * u0 * (d / s_) / re_ + 0.5
    peak = bench.peaks()[0]["hbm_gbs"]
    w = I.karman(seed=2)
    every = 50
    out = {"study": "rbf", "Re": re_, "s": s_, "tau": tau, "steps": args.steps, "nodes": int(w.n)}
    for name, interp, K in (("wls_K16", mlbm.INTERP_WLS, 16), ("rbf_K16", mlbm.INTERP_RBF, 16),
                            ("rbf_K24", mlbm.INTERP_RBF, 24)):
        st = mlbm.build_stencils_for(w, K=K, s=s_, bb_mode=mlbm.BB_SIMPLE, interp=interp)
        info = mlbm.stencils_info(st)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0))
        variant, ms = mlbm.autotune(ctx, 10, flush_l2=True)
        per_node = 4 * 18 + (32 if interp == mlbm.INTERP_RBF else 24) * K + 4 * K + 1
        alg = info["n_wls"] * per_node + info["n_lagrange"] * (4 * 18 + 4 * 12 + 4 + 1) + info["n_eq"] * (16 + 36 + 1)
        ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, 0.0, 0.0))
        mlbm.set_kernel_variant(ctx, variant)
        cd, cl = np.empty(args.steps // every), np.empty(args.steps // every)
        for i in range(len(cd)):
            mlbm.step(ctx, every)
            _, _, cd[i], cl[i] = mlbm.drag_lift(ctx, d, u0)
        h = len(cd) // 2
        out[name] = {"K": K, "variant": variant, "us_per_step_flushed": ms * 1e3, "mnups": w.n / (ms * 1e3),
                     "algorithmic_bytes_per_step": int(alg),
                     "hbm_frac_of_measured_peak": alg / (ms * 1e-3) / 1e9 / peak,
                     "strouhal": _strouhal(cl[h:], every, d / s_, u0), "cd_mean": float(np.mean(cd[h:])),
                     "cl_amplitude": float(np.ptp(cl[h:]) / 2)}
        print(json.dumps(out[name]), file=sys.stderr, flush=True)
    print(json.dumps(out))


def _alg_bytes(info, K, model):
    """Bytes one step must move at minimum, by node kind.  BGK: least-squares
    node 4 (9 + 9) + 24 K + 4 K + 1, Lagrange node 4 (9 + 9) + 48 + 4 + 1,
    equilibrium node 16 + 36 + 1.  tau = 1 (state (rho - 1, u, v) padded to
    16 B): least-squares node 16 + 16 + 24 K + 4 K + 1, Lagrange node
    16 + 16 + 48 + 4 + 1, equilibrium node 16 + 16 + 1."""
    pops = 32 if model == 1 else 72
    wls = pops + 28 * K + 1
    lag = pops + 48 + 4 + 1
    eq = 16 + (16 if model == 1 else 36) + 1
    return info["n_wls"] * wls + info["n_lagrange"] * lag + info["n_eq"] * eq


def kernels_study(args):
    """Step throughput on single workloads, each autotuned over the kernel
    variants with the L2 flushed before every timed step: one vortex-street
    run (BGK, K = 16, s = 1/2, simple bounce-back), the ~1M-node porous box
    under tau = 1 and under BGK (K = 16, s = 1/2, interpolated bounce-back,
    and BGK with simple bounce-back to show what the interpolated links cost).
    Reports the best variant, microseconds per step, node-updates/s and the
    fraction of the measured HBM copy bandwidth reached by the algorithmic
    bytes, both with the L2 flushed before each step and for steps run back
    to back (where a working set near the L2 size partly stays in L2)."""
    import torch
    from paper_2312_14789_gb300 import inputs as I
    from paper_2312_14789_gb300 import mlbm
    sys.path.insert(0, ROOT)
    import bench

    peak = bench.peaks()[0]["hbm_gbs"]
    wk = I.karman(seed=2)
    wp = I.porous(seed=3, n_target=args.nodes, porosity=0.7)
    cases = (("karman_one_bgk", wk, mlbm.BB_SIMPLE, mlbm.MODEL_BGK, 0.62, 0.0),
             ("porous_tau1", wp, mlbm.BB_INTERPOLATED, mlbm.MODEL_TAU1, 1.0, 1e-6),
             ("porous_bgk", wp, mlbm.BB_INTERPOLATED, mlbm.MODEL_BGK, 0.8, 1e-6),
             ("porous_bgk_simple_bb", wp, mlbm.BB_SIMPLE, mlbm.MODEL_BGK, 0.8, 1e-6))
    out = {"study": "kernels", "peak_hbm_gbs": peak, "runs": []}
    for name, w, bb, model, tau, g in cases:
        st = mlbm.build_stencils_for(w, K=16, s=0.5, bb_mode=bb)
        info = mlbm.stencils_info(st)
        ctx = mlbm.init(st, mlbm.Params(model, tau, 0.0, g, 0.0))
        variant, ms = mlbm.autotune(ctx, args.steps, flush_l2=True)
        alg = _alg_bytes(info, 16, model)
        stream = torch.cuda.Stream()
        mlbm.set_stream(ctx, stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            mlbm.step(ctx, 32)
            e0.record(stream)
            mlbm.step(ctx, 256)
            e1.record(stream)
        torch.cuda.synchronize()
        us_b2b = e0.elapsed_time(e1) * 1e3 / 256
        out["runs"].append({"workload": name, "nodes": int(w.n), "n_link_nodes": int(info["n_link_nodes"]),
                            "n_links": int(info["n_links"]), "variant": variant,
                            "us_per_step_flushed": ms * 1e3, "mnups_flushed": w.n / (ms * 1e3),
                            "hbm_frac_flushed": alg / (ms * 1e-3) / 1e9 / peak,
                            "us_per_step_back_to_back": us_b2b, "mnups_back_to_back": w.n / us_b2b,
                            "hbm_frac_back_to_back": alg / (us_b2b * 1e-6) / 1e9 / peak,
                            "algorithmic_bytes_per_step": int(alg)})
        print(json.dumps(out["runs"][-1]), file=sys.stderr, flush=True)
        del ctx
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("batch")
    b.add_argument("--samples", type=int, default=64)
    b.add_argument("--steps", type=int, default=20)
    w = sub.add_parser("warm")
    w.add_argument("--train", type=int, default=512)
    w.add_argument("--test", type=int, default=64)
    w.add_argument("--nodes", type=int, default=200_000)
    w.add_argument("--group", type=int, default=64)
    w.add_argument("--g", type=float, default=1e-6)
    w.add_argument("--steps", type=int, default=8000)
    w.add_argument("--batch", type=int, default=65536)
    w.add_argument("--seed", type=int, default=1)
    w.add_argument("--single", type=int, default=4)
    w.add_argument("--save", default="")
    po = sub.add_parser("porous")
    po.add_argument("--nodes", type=int, default=1_000_000)
    po.add_argument("--areas", default="voronoi", choices=["uniform", "voronoi"])
    rb = sub.add_parser("rbf")
    rb.add_argument("--steps", type=int, default=200_000)
    lb = sub.add_parser("lbm")
    lb.add_argument("--steps", type=int, default=200_000)
    lb.add_argument("--areas", default="voronoi", choices=["spacing", "voronoi"])
    kn = sub.add_parser("kernels")
    kn.add_argument("--nodes", type=int, default=1_000_000)
    kn.add_argument("--steps", type=int, default=20)
    hb = sub.add_parser("hybrid")
    hb.add_argument("--steps", type=int, default=200_000)
    hb.add_argument("--lattice-d", type=float, default=1.0)
    args = ap.parse_args()
    if args.cmd == "kernels":
        kernels_study(args)
    elif args.cmd == "hybrid":
        hybrid_study(args)
    elif args.cmd == "lbm":
        lbm_study(args)
    elif args.cmd == "rbf":
        rbf_study(args)
    elif args.cmd == "porous":
        porous_study(args)
    elif args.cmd == "batch":
        batch_study(args)
    elif args.cmd == "warm":
        warm_study(args)


if __name__ == "__main__":
    main()
