"""Learned warm start for body-force driven porous flow (MLBM1, tau = 1).

Workflow, all compute in the library's kernels (torch only holds device
arrays):
  1. solve training samples from rest to steady state (batched contexts);
  2. features (mlbm_features_device) and normalised targets
     t = (u nu / (g L^2), (rho - 1) / (3 g L)) of every node, L = mean disk
     radius of the sample, nu = (tau - 1/2) / 3 (Sec. 2.1: viscosity of the
     BGK relaxation), 3 (rho - 1) the pressure deviation over c_s^2;
  3. train the 16-64-64-64-n_out network with Adam on minibatches
     (mlbm_mlp_train_device); n_out = 2 predicts the velocity only, n_out = 3
     also the density;
  4. start a new sample from the prediction (mlbm_warm_start) and run to
     steady state.
In the Darcy regime the steady velocity is proportional to g / nu and the
pressure deviation to g L, so the normalised targets depend on geometry
alone.  The velocity-only start leaves the pressure field to build up from
uniform density through slowly damped acoustic modes, which dominate the
approach to steady state; predicting the density as well removes most of
that.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np

from . import mlbm

TOL, WINDOW = 1e-7, 1000   # steady when |u(t) - u(t - W)| / (W |u(t)|) < TOL
CHECK = 100                # the criterion is evaluated every CHECK steps
# training samples are solved ten times below the criterion the warm start is
# judged by, so that the targets stand for the steady state rather than the
# first state that passes the criterion
TRAIN_TOL = 1e-8


def length_scale(w) -> float:
    """Mean disk radius of the sample (spacing units)."""
    return float(w.disks[:, 2].mean()) if len(w.disks) else 8.0 * w.h_ref


def velocity_scale(g: float, tau: float, L: float) -> float:
    nu = (tau - 0.5) / 3.0
    return g * L * L / nu


def density_scale(g: float, L: float) -> float:
    return 3.0 * g * L


def _make(spec):
    from . import inputs as I
    return I.porous(seed=spec["seed"], n_target=spec["n_target"], porosity=spec["porosity"])


def make_samples(seeds, n_target, porosity=0.7, procs=None):
    """Porous samples (periodic in x, solid walls top and bottom), generated
    in a spawn-started process pool."""
    specs = [{"seed": int(s), "n_target": int(n_target), "porosity": float(porosity)} for s in seeds]
    procs = procs or min(16, os.cpu_count() or 4, len(specs))
    if procs <= 1:
        return [_make(s) for s in specs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_make, specs)


def build(ws, K=16, s=1.0):
    return [mlbm.build_stencils_for(w, K=K, s=s, bb_mode=mlbm.BB_INTERPOLATED) for w in ws]


def features(ws, device="cuda"):
    """Concatenated features [sum n][16] (torch, on the device)."""
    import torch
    n = sum(w.n for w in ws)
    X = torch.empty((n, 16), dtype=torch.float32, device=device)
    o = 0
    for w in ws:
        if w.n:
            mlbm.features_for(w, length_scale(w), X[o:o + w.n].data_ptr())
        o += w.n
    return X


def solve(sts, params, tol=TOL, window=WINDOW, max_steps=400_000, init=None, check=CHECK):
    """Batched run to steady state.  init(ctx) may set the initial state.
    Returns (fields [sum n][3] rho, ux, uy; steps per sample; seconds;
    permeability per sample)."""
    import torch
    ctx = mlbm.batch_init(sts, params)
    mlbm.autotune(ctx, 5)          # keeps the state
    if init is not None:
        init(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = mlbm.batch_run_to_steady(ctx, tol, window, max_steps, check=check)
    sec = time.perf_counter() - t0
    k = mlbm.batch_permeability(ctx)["k"]
    ru = mlbm.get_fields(ctx)
    return ru, steps, sec, k


def targets(ws, ru, params, n_out=3):
    """Normalised steady velocities (and density deviations) [sum n][n_out]
    (float32, host)."""
    T = np.empty((len(ru), n_out), np.float32)
    o = 0
    for w, p in zip(ws, params):
        L = length_scale(w)
        T[o:o + w.n, :2] = ru[o:o + w.n, 1:] / velocity_scale(abs(p.gx), p.tau, L)
        if n_out == 3:
            T[o:o + w.n, 2] = (ru[o:o + w.n, 0] - 1.0) / density_scale(abs(p.gx), L)
        o += w.n
    return T


def train(net, X, T, steps, batch=65536, lr=(2e-3, 1e-3, 3e-4, 1e-4), seed=12345, log=None):
    """Adam over `steps` minibatch steps, the learning rate stepping through
    `lr` in equal parts.  Returns the loss of the last minibatch of each part."""
    n = X.shape[0]
    batch = min(batch, n)
    part = max(1, steps // len(lr))
    losses = []
    for i, rate in enumerate(lr):
        k = part if i < len(lr) - 1 else steps - part * (len(lr) - 1)
        if k <= 0:
            continue
        losses.append(net.train(X.data_ptr(), T.data_ptr(), n, batch, k, rate, seed + i))
        if log:
            log(f"train part {i}: lr {rate:g} steps {k} loss {losses[-1]:.4g}")
    return losses


def warm_init(net, X, ws, params):
    """init callback of solve(): the network's prediction per sample."""
    su = [velocity_scale(abs(p.gx), p.tau, length_scale(w)) for w, p in zip(ws, params)]
    sr = [density_scale(abs(p.gx), length_scale(w)) for w, p in zip(ws, params)] if net.n_out == 3 else None

    def f(ctx):
        cold = mlbm.warm_start(ctx, net, X.data_ptr(), su, sr)
        if cold:
            raise RuntimeError(f"{cold} samples fell back to a cold start")
    return f


def kozeny_init(ws, params):
    """init callback of solve(): uniform intrinsic velocity U_s / phi from a
    Kozeny-Carman permeability k = phi^3 d^2 / (180 (1 - phi)^2), d the mean
    disk diameter (a naive control, not a learned prediction)."""
    def f(ctx):
        rus = []
        for w, p in zip(ws, params):
            phi = w.meta["porosity"]
            d = 2.0 * length_scale(w)
            k = phi ** 3 * d * d / (180.0 * (1.0 - phi) ** 2)
            nu = (p.tau - 0.5) / 3.0
            ru = np.zeros((w.n, 3))
            ru[:, 0] = 1.0
            ru[:, 1] = k * p.gx / nu / phi
            rus.append(ru)
        mlbm.set_fields(ctx, np.concatenate(rus, 0))
    return f
