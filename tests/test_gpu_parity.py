"""GPU parity of the fused CUDA step (through the C ABI) against the FP64 oracle.

Tolerances.  The GPU computes in FP32 with populations stored minus their
weights; one step moves each stored value by at most a few ulp of the largest
stencil term (|w_i| <= ~2, K <= 16 terms, values ~1e-2 after the shift), so
the per-step absolute error on a population is ~1e-8.  Over n steps it grows
at most linearly (the step is a contraction plus round-off), hence the
population tolerance 2e-8 * (n + 10) used below.  For velocity fields the
contract is the relative L2 error <= 1e-5 against the FP64 oracle for
laminar cases.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2312_14789_gb300 import inputs as I
from paper_2312_14789_gb300 import mlbm

pytestmark = pytest.mark.gpu


def pop_tol(n_steps):
    return 2e-8 * (n_steps + 10)


def random_populations(n, seed, amp=2e-3):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.01 * rng.standard_normal(n)
    ux = 0.02 * rng.standard_normal(n)
    uy = 0.02 * rng.standard_normal(n)
    return O.equilibrium(rho, ux, uy) + amp * I.uniform_noise((n, 9), seed + 1)


def to_f32_state(f):
    """The exact FP32 state the GPU stores (f - omega rounded to FP32)."""
    _, W, _ = O.lattice_constants()
    return (f - W).astype(np.float32).astype(np.float64) + W


def gpu_ctx(w, K, s, bb_mode, params, sigma=0.7071067811865476, use_lagrange=True, variant=None):
    st = mlbm.build_stencils_for(w, K=K, s=s, sigma_factor=sigma, bb_mode=bb_mode, use_lagrange=use_lagrange)
    ctx = mlbm.init(st, params)
    if variant is not None:
        mlbm.set_kernel_variant(ctx, variant)
    return ctx


VARIANTS = list(range(30))


# ----------------------------------------------------------------- plain MLBM
def test_poiseuille_channel_2000_steps_matches_oracle():
    """Plain MLBM Poiseuille case: 40x50 jittered grid, K=12, tau=0.8, s=1,
    g=1e-6, 2000 steps; relative L2 velocity error <= 1e-5."""
    w = I.poiseuille_channel(40, 50, 0.2, seed=1)
    g = (1e-6, 0.0)
    ctx = gpu_ctx(w, 12, 1.0, 1, mlbm.Params(mlbm.MODEL_BGK, 0.8, 0.0, *g))
    mlbm.step(ctx, 2000)
    rho, u = mlbm.macroscopics(ctx)
    op = O.Operator(w, K=12, s=1.0, bb_mode=1).check()
    f = O.run_bgk(op, O.equilibrium(np.ones(w.n), 0, 0), 0.8, g, 2000)
    rho_o, ux_o, uy_o = O.macroscopics(f, g)
    err = np.linalg.norm(np.stack([u[:, 0] - ux_o, u[:, 1] - uy_o])) / np.linalg.norm(np.stack([ux_o, uy_o]))
    assert err <= 1e-5, err
    assert np.abs(rho - rho_o).max() < 1e-6


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", ["lattice", "channel_halfway", "jittered", "karman_small", "karman_hybrid_small",
                                  "karman_coarse_small", "porous_small"])
def test_bgk_steps_match_oracle_elementwise(case, variant):
    if case == "lattice":
        w, K, s, bb, tau, g = I.lattice(33, 17), 12, 1.0, 1, 0.7, (1e-5, -2e-6)
    elif case == "channel_halfway":
        w, K, s, bb, tau, g = I.lattice_channel(21, 13, 0.5), 16, 1.0, 0, 0.9, (1e-5, 0.0)
    elif case == "jittered":
        w, K, s, bb, tau, g = I.jittered_periodic(37, 29, 0.25, seed=4), 16, 0.8, 1, 0.75, (1e-5, 3e-6)
    elif case == "karman_small":
        w, K, s, bb, tau, g = I.karman(seed=2, scale=0.25), 16, 0.5, 0, 0.62, (0.0, 0.0)
    elif case == "karman_hybrid_small":
        w, K, s, bb, tau, g = I.karman(seed=2, scale=0.25, lattice_beyond_d=1.0), 16, 0.5, 0, 0.62, (0.0, 0.0)
    elif case == "karman_coarse_small":
        w = I.karman(seed=2, scale=0.25, lattice_beyond_d=1.0, coarse_beyond_d=2.0)
        K, s, bb, tau, g = 16, 0.5, 0, 0.62, (0.0, 0.0)
    else:
        w, K, s, bb, tau, g = I.porous(seed=5, n_target=15000), 16, 0.5, 1, 0.8, (1e-5, 0.0)
    f0 = to_f32_state(random_populations(w.n, 11))
    ctx = gpu_ctx(w, K, s, bb, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, *g), variant=variant)
    mlbm.set_populations(ctx, f0)
    assert np.array_equal(mlbm.get_populations(ctx), f0)
    op = O.Operator(w, K=K, s=s, bb_mode=bb).check()
    f = f0
    done = 0
    for n_steps in (1, 9):
        mlbm.step(ctx, n_steps)
        for _ in range(n_steps):
            f = O.bgk_step(op, f, tau, g)
        done += n_steps
        fg = mlbm.get_populations(ctx)
        err = np.abs(fg - f).max()
        assert err < pop_tol(done), (case, done, err)


@pytest.mark.parametrize("variant", [0, 10, 11, 12, 20, 21])
@pytest.mark.parametrize("case", ["jittered", "karman_small", "karman_hybrid_small", "porous_small"])
def test_rbf_steps_match_oracle_elementwise(case, variant):
    """RBF-FD stencils (the paper's interpolant, Sec. 2.2): the GPU step against
    the oracle's step with its own RBF-FD weights, 10 steps from a random state."""
    if case == "jittered":
        w, K, s, bb, tau, g = I.jittered_periodic(37, 29, 0.25, seed=4), 16, 0.8, 1, 0.75, (1e-5, 3e-6)
    elif case == "karman_small":
        w, K, s, bb, tau, g = I.karman(seed=2, scale=0.25), 16, 0.5, 0, 0.62, (0.0, 0.0)
    elif case == "karman_hybrid_small":
        w, K, s, bb, tau, g = I.karman(seed=2, scale=0.25, lattice_beyond_d=1.0), 24, 0.5, 0, 0.62, (0.0, 0.0)
    else:
        w, K, s, bb, tau, g = I.porous(seed=5, n_target=15000), 16, 0.5, 1, 0.8, (1e-5, 0.0)
    st = mlbm.build_stencils_for(w, K=K, s=s, bb_mode=bb, interp=mlbm.INTERP_RBF)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, *g))
    mlbm.set_kernel_variant(ctx, variant)
    f0 = to_f32_state(random_populations(w.n, 11))
    mlbm.set_populations(ctx, f0)
    op = O.Operator(w, K=K, s=s, bb_mode=bb, interp="rbf").check()
    f = f0
    done = 0
    for n_steps in (1, 9):
        mlbm.step(ctx, n_steps)
        for _ in range(n_steps):
            f = O.bgk_step(op, f, tau, g)
        done += n_steps
        err = np.abs(mlbm.get_populations(ctx) - f).max()
        assert err < pop_tol(done), (case, done, err)
    fx, fy, _, _ = mlbm.drag_lift(ctx, 1.0, 1.0)
    ox, oy = O.force_bgk(op, mlbm.get_populations(ctx))
    assert abs(fx - ox) <= 1e-4 * max(abs(ox), 1e-12) + 1e-9 and abs(fy - oy) <= 1e-4 * max(abs(ox), 1e-12) + 1e-9


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("case", ["jittered", "karman_small", "porous_small", "porous_tau1"])
def test_rbf_points_steps_match_oracle_elementwise(case, variant):
    """RBF-FD with a stencil per Lagrangian point (Sec. 2.2, N_L = 25 nearest
    nodes of every departure point; union stencils 64 wide): the GPU step
    against the oracle's step with its own stencils and weights, 10 steps
    from a random state, BGK and tau = 1."""
    model = mlbm.MODEL_BGK
    if case == "jittered":
        w, s, bb, tau, g = I.jittered_periodic(37, 29, 0.25, seed=4), 0.8, 1, 0.75, (1e-5, 3e-6)
    elif case == "karman_small":
        w, s, bb, tau, g = I.karman(seed=2, scale=0.25), 0.5, 0, 0.62, (0.0, 0.0)
    elif case == "porous_small":
        w, s, bb, tau, g = I.porous(seed=5, n_target=8000), 1.0, 1, 0.8, (1e-5, 0.0)
    else:
        w, s, bb, tau, g = I.porous(seed=6, n_target=8000), 1.0, 1, 1.0, (1e-5, 0.0)
        model = mlbm.MODEL_TAU1
    st = mlbm.build_stencils_for(w, K=64, s=s, bb_mode=bb, interp=mlbm.INTERP_RBF_POINTS, n_l=25)
    ctx = mlbm.init(st, mlbm.Params(model, tau, 0.0, *g))
    mlbm.set_kernel_variant(ctx, variant)
    op = O.Operator(w, K=16, s=s, bb_mode=bb, interp="rbf_points", n_l=25, k_max=64).check()
    if model == mlbm.MODEL_BGK:
        f0 = to_f32_state(random_populations(w.n, 11))
        mlbm.set_populations(ctx, f0)
        f, done = f0, 0
        for n_steps in (1, 9):
            mlbm.step(ctx, n_steps)
            for _ in range(n_steps):
                f = O.bgk_step(op, f, tau, g)
            done += n_steps
            err = np.abs(mlbm.get_populations(ctx) - f).max()
            assert err < pop_tol(done), (case, done, err)
    else:
        rng = np.random.default_rng(12)
        ru = np.column_stack([1 + 0.01 * rng.standard_normal(w.n), 0.01 * rng.standard_normal(w.n),
                              0.01 * rng.standard_normal(w.n)])
        ru = ru.astype(np.float32).astype(np.float64)
        mlbm.set_fields(ctx, ru)
        r, done = mlbm.get_fields(ctx), 0
        for n_steps in (1, 9):
            mlbm.step(ctx, n_steps)
            for _ in range(n_steps):
                r = O.mlbm1_step(op, r, g)
            done += n_steps
            err = np.abs(mlbm.get_fields(ctx) - r).max()
            assert err < 5 * pop_tol(done), (case, done, err)


def test_rbf_poiseuille_2000_steps_matches_oracle():
    w = I.poiseuille_channel(40, 50, 0.2, seed=1)
    g = (1e-6, 0.0)
    st = mlbm.build_stencils_for(w, K=12, s=1.0, bb_mode=1, interp=mlbm.INTERP_RBF)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, 0.8, 0.0, *g))
    mlbm.step(ctx, 2000)
    _, u = mlbm.macroscopics(ctx)
    op = O.Operator(w, K=12, s=1.0, bb_mode=1, interp="rbf").check()
    f = O.run_bgk(op, O.equilibrium(np.ones(w.n), 0, 0), 0.8, g, 2000)
    _, ux, uy = O.macroscopics(f, g)
    err = np.linalg.norm(np.stack([u[:, 0] - ux, u[:, 1] - uy])) / np.linalg.norm(np.stack([ux, uy]))
    assert err <= 1e-5, err


@pytest.mark.parametrize("variant", [0, 11, 12])
def test_rbf_tau1_steps_match_oracle(variant):
    """tau = 1 (MLBM1) with RBF-FD stencils on a porous box with interpolated
    bounce-back: 10 steps from a random (rho, u) against the oracle."""
    w = I.porous(seed=5, n_target=15000)
    g = (1e-5, 0.0)
    st = mlbm.build_stencils_for(w, K=16, s=0.5, bb_mode=1, interp=mlbm.INTERP_RBF)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, *g))
    mlbm.set_kernel_variant(ctx, variant)
    rng = np.random.default_rng(4)
    ru = np.stack([1 + (0.01 * rng.standard_normal(w.n)).astype(np.float32).astype(np.float64),
                   (0.01 * rng.standard_normal(w.n)).astype(np.float32).astype(np.float64),
                   (0.01 * rng.standard_normal(w.n)).astype(np.float32).astype(np.float64)], 1)
    mlbm.set_fields(ctx, ru)
    op = O.Operator(w, K=16, s=0.5, bb_mode=1, interp="rbf").check()
    a = ru
    for _ in range(10):
        a = O.mlbm1_step(op, a, g)
    mlbm.step(ctx, 10)
    b = mlbm.get_fields(ctx)
    assert np.abs(b - a).max() < 5 * pop_tol(10)


def test_regular_lattice_streaming_is_exact_in_fp32():
    """s = h on a regular lattice: the Lagrange weights are exactly one-hot, so
    with tau = 1 and no force the GPU step is the index shift of Eq. (1) followed
    by the FP32 equilibrium; with g = 0 and a uniform state nothing changes."""
    w = I.lattice(24, 16)
    ctx = gpu_ctx(w, 12, 1.0, 1, mlbm.Params(mlbm.MODEL_BGK, 1.0, 0.0, 0.0, 0.0))
    rng = np.random.default_rng(3)
    # one moving population pattern, everything else at rest equilibrium
    _, W, _ = O.lattice_constants()
    f0 = np.tile(W, (w.n, 1))
    f0[:, 1] += 1e-3 * rng.integers(0, 4, w.n)  # exact small binary fractions
    mlbm.set_populations(ctx, f0)
    op = O.Operator(w, K=12, s=1.0, bb_mode=1).check()
    # streaming alone is exact: compare the moments the collision sees
    mlbm.step(ctx, 1)
    f1 = O.bgk_step(op, to_f32_state(f0), 1.0)
    assert np.abs(mlbm.get_populations(ctx) - f1).max() < 1e-7
    mass0 = f0.sum()
    mlbm.step(ctx, 200)
    assert abs(mlbm.get_populations(ctx).sum() - mass0) / mass0 < 1e-6


def test_trt_matches_oracle():
    w = I.poiseuille_channel(30, 20, 0.2, seed=7)
    tau_p = 0.7
    tau_m = 0.5 + (3 / 16) / (tau_p - 0.5)
    g = (1e-5, 0.0)
    ctx = gpu_ctx(w, 16, 1.0, 1, mlbm.Params(mlbm.MODEL_BGK, tau_p, tau_m, *g))
    mlbm.step(ctx, 500)
    op = O.Operator(w, K=16, s=1.0, bb_mode=1).check()
    f = O.run_bgk(op, O.equilibrium(np.ones(w.n), 0, 0), tau_p, g, 500, tau_minus=tau_m)
    _, ux, uy = O.macroscopics(f, g)
    _, u = mlbm.macroscopics(ctx)
    assert O.relative_l2(u[:, 0], ux) < 1e-5


# --------------------------------------------------------------- tau = 1
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", ["lattice", "porous_small", "porous_small_s4", "channel_simple"])
def test_tau1_steps_match_oracle(case, variant):
    if case == "lattice":
        w, K, s, bb = I.lattice(20, 20), 12, 1.0, 1
    elif case == "porous_small":
        w, K, s, bb = I.porous(seed=6, n_target=20000), 16, 1.0, 1
    elif case == "porous_small_s4":
        w, K, s, bb = I.porous(seed=6, n_target=20000), 16, 0.25, 1
    else:
        w, K, s, bb = I.lattice_channel(15, 12, 0.5), 16, 1.0, 0
    g = (1e-5, 2e-6)
    rng = np.random.default_rng(2)
    ru = np.stack([1 + 0.01 * rng.standard_normal(w.n), 0.01 * rng.standard_normal(w.n),
                   0.01 * rng.standard_normal(w.n)], 1)
    ru = np.stack([(ru[:, 0] - 1).astype(np.float32).astype(np.float64) + 1,
                   ru[:, 1].astype(np.float32).astype(np.float64),
                   ru[:, 2].astype(np.float32).astype(np.float64)], 1)
    ctx = gpu_ctx(w, K, s, bb, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, *g), variant=variant)
    mlbm.set_fields(ctx, ru)
    op = O.Operator(w, K=K, s=s, bb_mode=bb).check()
    a = ru
    done = 0
    for n_steps in (1, 9):
        mlbm.step(ctx, n_steps)
        for _ in range(n_steps):
            a = O.mlbm1_step(op, a, g)
        done += n_steps
        b = mlbm.get_fields(ctx)
        err = np.abs(b - a).max()
        assert err < 5 * pop_tol(done), (case, done, err)


def test_tau1_poiseuille_relative_l2():
    w = I.poiseuille_channel(40, 50, 0.2, seed=1)
    g = (1e-6, 0.0)
    ctx = gpu_ctx(w, 12, 1.0, 1, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, *g))
    mlbm.step(ctx, 2000)
    ru = mlbm.get_fields(ctx)
    op = O.Operator(w, K=12, s=1.0, bb_mode=1).check()
    r0 = np.zeros((w.n, 3))
    r0[:, 0] = 1
    ro = O.run_mlbm1(op, r0, g, 2000)
    assert O.relative_l2(ru[:, 1:], ro[:, 1:]) <= 1e-5


# ------------------------------------------------------------ observables
def test_force_and_permeability_match_oracle():
    w = I.porous(seed=8, n_target=12000)
    g = (1e-5, 0.0)
    ctx = gpu_ctx(w, 16, 1.0, 1, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, *g))
    mlbm.step(ctx, 300)
    op = O.Operator(w, K=16, s=1.0, bb_mode=1).check()
    r0 = np.zeros((w.n, 3))
    r0[:, 0] = 1
    ro = O.run_mlbm1(op, r0, g, 300)
    fx, fy, cd, cl = mlbm.drag_lift(ctx, 1.0, 1.0)
    ox, oy = O.force_mlbm1(op, ro, g)
    scale = abs(ox) + abs(oy)
    assert abs(fx - ox) / scale < 1e-4 and abs(fy - oy) / scale < 1e-4
    pm = mlbm.permeability(ctx)
    fluid = w.node_class != I.EQ
    us, ui = O.mean_velocity(ro[:, 1], w.area, fluid, total_area=(w.box[2] - w.box[0]) * (w.box[3] - w.box[1]))
    assert abs(pm["u_superficial"] / us - 1) < 1e-5
    assert abs(pm["u_intrinsic"] / ui - 1) < 1e-5
    assert abs(pm["k"] / O.permeability(us, 1.0, g[0]) - 1) < 1e-5
    assert abs(pm["tortuosity"] / O.tortuosity(ro[:, 1], ro[:, 2], w.area) - 1) < 1e-5


def test_karman_drag_matches_oracle():
    w = I.karman(seed=2, scale=0.25)
    U0 = w.meta["U0"]
    ctx = gpu_ctx(w, 16, 0.5, 0, mlbm.Params(mlbm.MODEL_BGK, 0.62, 0.0, 0.0, 0.0))
    mlbm.step(ctx, 300)
    op = O.Operator(w, K=16, s=0.5, bb_mode=0).check()
    f = O.run_bgk(op, O.equilibrium(np.ones(w.n), 0, 0), 0.62, (0, 0), 300)
    fx, fy, cd, cl = mlbm.drag_lift(ctx, w.meta["D"], U0)
    ox, oy = O.force_bgk(op, f)
    assert abs(fx - ox) / abs(ox) < 1e-4
    assert abs(fy - oy) < 1e-4 * abs(ox)
    assert abs(cd - 2 * ox / (U0 ** 2 * w.meta["D"] / 0.5)) / abs(cd) < 1e-4


# ------------------------------------------------------- full-size samples
def _sample_targets(w, n_rand, seed, link_nodes=None):
    rng = np.random.default_rng(seed)
    t = rng.choice(w.n, size=n_rand, replace=False)
    if link_nodes is not None and len(link_nodes):
        t = np.concatenate([t, rng.choice(link_nodes, size=min(100, len(link_nodes)), replace=False)])
    return np.unique(t)


def test_karman_full_size_one_step_sampled():
    """Cylinder channel at full size (~260k nodes, K=16, simple bounce-back):
    one fused step from a random state, 400 sampled nodes (plus link nodes)
    checked one by one against the oracle."""
    w = I.karman(seed=2)
    assert w.n > 200000
    st = mlbm.build_stencils_for(w, K=16, s=0.5, bb_mode=0)
    ex = mlbm.stencils_export(st)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_BGK, 0.62, 0.0, 0.0, 0.0))
    f0 = to_f32_state(random_populations(w.n, 21))
    mlbm.set_populations(ctx, f0)
    mlbm.step(ctx, 1)
    fg = mlbm.get_populations(ctx)
    t = _sample_targets(w, 400, 5, np.nonzero(ex["link_mask"])[0])
    op = O.Operator(w, K=16, s=0.5, bb_mode=0, targets=t).check()
    assert np.array_equal(op.idx, ex["idx"][t])
    fo = O.bgk_step(op, f0, 0.62)
    assert np.abs(fg[t] - fo).max() < pop_tol(1)


def test_porous_full_size_tau1_one_step_sampled():
    """Porous box at full size (~1M nodes, K=16, interpolated bounce-back,
    tau = 1): one step from a random state, sampled nodes against the oracle."""
    w = I.porous(seed=3, n_target=1_000_000)
    st = mlbm.build_stencils_for(w, K=16, s=0.5, bb_mode=1)
    ex = mlbm.stencils_export(st)
    g = (1e-5, 0.0)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, *g))
    rng = np.random.default_rng(4)
    ru = np.stack([1 + (0.01 * rng.standard_normal(w.n)).astype(np.float32).astype(np.float64),
                   (0.01 * rng.standard_normal(w.n)).astype(np.float32).astype(np.float64),
                   (0.01 * rng.standard_normal(w.n)).astype(np.float32).astype(np.float64)], 1)
    mlbm.set_fields(ctx, ru)
    mlbm.step(ctx, 1)
    b = mlbm.get_fields(ctx)
    t = _sample_targets(w, 400, 6, np.nonzero(ex["link_mask"])[0])
    op = O.Operator(w, K=16, s=0.5, bb_mode=1, targets=t).check()
    a = O.mlbm1_step(op, ru, g)
    assert np.abs(b[t] - a).max() < 5 * pop_tol(1)


@pytest.mark.parametrize("s,g", [(1.0, 1e-6), (0.25, 2e-5)])
def test_porous_tau1_steady_state_matches_oracle(s, g):
    """Body-force driven flow through a small porous box (~8k nodes, tau = 1,
    interpolated bounce-back) from rest to steady state on the GPU (Darcy,
    s = 1, and a faster flow at s = 1/4); the oracle runs the same number of
    steps.  Laminar contract: relative L2 velocity error <= 1e-5, and the
    permeability of the two fields within 1e-5."""
    w = I.porous(seed=41, n_target=8000, porosity=0.7)
    st = mlbm.build_stencils_for(w, K=16, s=s, bb_mode=1)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0))
    steps = mlbm.run_to_steady(ctx, 1e-7, 1000, 60_000, check=100)
    ru = mlbm.get_fields(ctx)
    k = mlbm.permeability(ctx)["k"]
    op = O.Operator(w, K=16, s=s, bb_mode=1).check()
    ru0 = np.zeros((w.n, 3))
    ru0[:, 0] = 1.0
    ro = O.run_mlbm1(op, ru0, (g, 0.0), steps)
    err = np.linalg.norm(ru[:, 1:] - ro[:, 1:]) / np.linalg.norm(ro[:, 1:])
    assert err <= 1e-5, (steps, err)
    box = (w.box[2] - w.box[0]) * (w.box[3] - w.box[1])
    us, _ = O.mean_velocity(ro[:, 1], w.area, None, total_area=box)
    ko = O.permeability(us, 1.0, g)
    assert abs(k / ko - 1) <= 1e-5, (k, ko)



def test_square_cylinder_array_steady_state_matches_oracle_and_closed_form():
    """Darcy flow through a square array of cylinders (radius 16 in a doubly
    periodic cell of side 80, tau = 1, s = 1, interpolated bounce-back,
    fluid-Voronoi areas) from rest to steady state on the GPU; the oracle
    runs the same number of steps.  Laminar contract on the velocity
    (relative L2 <= 1e-5), and the GPU permeability within 0.5% of the
    array's slow-flow closed form (0.28% below it at this resolution)."""
    from test_oracle_flows import _square_array_k
    L, a, g = 80.0, 16.0, 1e-6
    w = I.cylinder_array(L, a, seed=1)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=1)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0))
    steps = mlbm.run_to_steady(ctx, 1e-7, 1000, 100_000, check=100)
    ru = mlbm.get_fields(ctx)
    k = mlbm.permeability(ctx)["k"]
    assert abs(k / _square_array_k(L, a) - 1) <= 0.005, k
    op = O.Operator(w, K=16, s=1.0, bb_mode=1).check()
    ru0 = np.zeros((w.n, 3))
    ru0[:, 0] = 1.0
    ro = O.run_mlbm1(op, ru0, (g, 0.0), steps)
    err = np.linalg.norm(ru[:, 1:] - ro[:, 1:]) / np.linalg.norm(ro[:, 1:])
    assert err <= 1e-5, (steps, err)



@pytest.mark.parametrize("variant", [11, 12, 25, 26])
@pytest.mark.parametrize("model", ["bgk", "tau1"])
def test_graph_replay_matches_direct_launches(model, variant):
    """Steps replayed from captured graphs (chunks of 16 launches) leave the same
    state as the same steps launched one by one: plain and persistent grids,
    and the variants whose launches overlap through programmatic dependent
    launch (25, 26)."""
    if model == "bgk":
        w, K, s, bb = I.karman(seed=2, scale=0.25), 16, 0.5, 0
        p = mlbm.Params(mlbm.MODEL_BGK, 0.62, 0.0, 0.0, 0.0)
    else:
        w, K, s, bb = I.porous(seed=6, n_target=20000), 16, 0.5, 1
        p = mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0)
    out = []
    for graphs in (True, False):
        ctx = gpu_ctx(w, K, s, bb, p, variant=variant)
        mlbm.set_graphs(ctx, graphs)
        mlbm.step(ctx, 40)
        out.append(mlbm.get_fields(ctx))
    assert np.array_equal(out[0], out[1])



@pytest.mark.parametrize("model", ["tau1", "bgk"])
def test_wall_stress_force_matches_oracle_and_carries_the_body_force(model):
    """Body-force flow through a square array of cylinders (radius 8, cell 40,
    s = 1, interpolated bounce-back), 8000 steps from rest on the GPU and in
    the oracle.  The force from the stress integrated along the disk's wall
    nodes matches the oracle's on its own field to 1e-4 (relative to the
    drag), and carries the body force on the fluid within 5% (3% low at this
    resolution, in both models)."""
    L, a, g, steps = 40.0, 8.0, 1e-6, 8000
    tau = 1.0 if model == "tau1" else 0.8
    w = I.cylinder_array(L, a, seed=1)
    geo = I.wall_geometry(w)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=1)
    m = mlbm.MODEL_TAU1 if model == "tau1" else mlbm.MODEL_BGK
    ctx = mlbm.init(st, mlbm.Params(m, tau, 0.0, g, 0.0))
    mlbm.step(ctx, steps)
    fx, fy = mlbm.wall_stress_force(ctx, *geo)
    op = O.Operator(w, K=16, s=1.0, bb_mode=1).check()
    if model == "tau1":
        ru = np.zeros((w.n, 3))
        ru[:, 0] = 1.0
        ru = O.run_mlbm1(op, ru, (g, 0.0), steps)
    else:
        f = O.run_bgk(op, O.equilibrium(np.ones(w.n), 0, 0), tau, (g, 0.0), steps)
        ru = np.stack(O.macroscopics(f, (g, 0.0)), 1)
    ofx, ofy = O.wall_stress_force(op, ru, tau, *geo)
    assert abs(fx - ofx) <= 1e-4 * abs(ofx) and abs(fy - ofy) <= 1e-4 * abs(ofx), (fx, ofx, fy, ofy)
    body = g * np.sum(ru[:, 0] * w.area)
    assert abs(fx / body - 1) <= 0.05, fx / body
    with pytest.raises(mlbm.MlbmError):
        mlbm.wall_stress_force(ctx, [w.n], [[1.0, 0.0]], [1.0])


# ------------------------------------------------------------ host features
def test_save_load_continues_bitwise():
    w = I.poiseuille_channel(20, 16, 0.2, seed=3)
    p = mlbm.Params(mlbm.MODEL_BGK, 0.8, 0.0, 1e-5, 0.0)
    a = gpu_ctx(w, 12, 1.0, 1, p)
    mlbm.step(a, 100)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        mlbm.save(a, path)
        mlbm.step(a, 100)
        b = gpu_ctx(w, 12, 1.0, 1, p)
        mlbm.load(b, path)
        assert mlbm.step_count(b) == 100
        mlbm.step(b, 100)
    assert np.array_equal(mlbm.get_populations(a), mlbm.get_populations(b))


def test_run_to_steady_poiseuille():
    w = I.lattice_channel(4, 12, 0.5)
    g, tau = 1e-5, 0.8
    ctx = gpu_ctx(w, 16, 1.0, 0, mlbm.Params(mlbm.MODEL_BGK, tau, 0.0, g, 0.0))
    steps = mlbm.run_to_steady(ctx, 1e-9, 500, 50000)
    assert 0 < steps < 50000
    _, u = mlbm.macroscopics(ctx)
    uu = u[:, 0].reshape(12, 4)[:, 0]
    d2 = uu[2:] - 2 * uu[1:-1] + uu[:-2]
    nu = (tau - 0.5) / 3
    assert np.allclose(d2, -g / nu, rtol=1e-3)


def test_device_reduction_entry_point():
    torch = pytest.importorskip("torch")
    n = 300001
    rng = np.random.default_rng(0)
    h = {k: rng.uniform(0.5, 1.5, n).astype(np.float32) for k in ("rho", "ux", "uy", "area")}
    mask = (rng.uniform(size=n) > 0.1).astype(np.uint8)
    d = {k: torch.from_numpy(v).cuda() for k, v in h.items()}
    dm = torch.from_numpy(mask).cuda()
    ns = mlbm.reduce_scratch_doubles(n)
    scratch = torch.empty(ns, dtype=torch.float64, device="cuda")
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    mlbm.reduce_fields_device(d["rho"].data_ptr(), d["ux"].data_ptr(), d["uy"].data_ptr(), d["area"].data_ptr(),
                              dm.data_ptr(), n, scratch.data_ptr(), ns, out.data_ptr(), 0)
    torch.cuda.synchronize()
    m = mask.astype(bool)
    a, r, u, v = (h[k][m].astype(np.float64) for k in ("area", "rho", "ux", "uy"))
    ref = [a.sum(), (r * a).sum(), (u * a).sum(), (v * a).sum(), (np.hypot(u, v) * a).sum(), ((u * u + v * v) * a).sum()]
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12)
    with pytest.raises(mlbm.MlbmError):
        mlbm.reduce_fields_device(d["rho"].data_ptr(), d["ux"].data_ptr(), d["uy"].data_ptr(), d["area"].data_ptr(),
                                  0, n, scratch.data_ptr(), ns - 1, out.data_ptr(), 0)


def test_autotune_keeps_state_and_picks_a_variant():
    w = I.porous(seed=9, n_target=30000)
    ctx = gpu_ctx(w, 16, 1.0, 1, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0))
    mlbm.step(ctx, 5)
    before = mlbm.get_fields(ctx)
    v, ms = mlbm.autotune(ctx, 5)
    assert v in VARIANTS and ms > 0
    assert mlbm.step_count(ctx) == 5
    assert np.array_equal(mlbm.get_fields(ctx), before)


def test_karman_sweep_batch_full_size_one_step_sampled():
    """The benchmark's launch configuration: the six (Re, s) vortex-street runs
    in one batched context at full size, autotuned variant; one step from a
    random state, 150 sampled nodes of every run (plus link nodes) checked
    one by one against the oracle."""
    import bench
    w = I.karman(seed=2)
    st_by_s = {s: mlbm.build_stencils_for(w, K=16, s=s, bb_mode=0) for s in sorted({s for _, s in bench.CASES})}
    sts = [st_by_s[s] for _, s in bench.CASES]
    params = [mlbm.Params(mlbm.MODEL_BGK, bench.tau_of(re, s), 0.0, 0.0, 0.0) for re, s in bench.CASES]
    ctx = mlbm.batch_init(sts, params)
    mlbm.autotune(ctx, 3)
    f0 = to_f32_state(random_populations(w.n, 41))
    mlbm.set_populations(ctx, np.tile(f0, (len(bench.CASES), 1)))
    mlbm.step(ctx, 1)
    fg = mlbm.get_populations(ctx)
    for i, (re, s) in enumerate(bench.CASES):
        first, count = mlbm.batch_range(ctx, i)
        ex = mlbm.stencils_export(sts[i])
        t = _sample_targets(w, 150, 50 + i, np.nonzero(ex["link_mask"])[0])
        op = O.Operator(w, K=16, s=s, bb_mode=0, targets=t).check()
        fo = O.bgk_step(op, f0, bench.tau_of(re, s))
        assert np.abs(fg[first:first + count][t] - fo).max() < pop_tol(1), (re, s)


def test_porous_batch_full_size_sampled_and_graph_replay():
    """The benchmark's launch configuration: the 64 porous samples (seeds
    1000..1063, 13.3M nodes, tau = 1, interpolated bounce-back) in one
    batched context at full size with the autotuned variant.  One step from
    a random state: 30 sampled nodes of every sample (plus link nodes)
    checked one by one against the oracle.  Then 16 steps replayed from the
    captured graph equal 16 direct launches bit for bit at this size."""
    specs = I.porous_batch_specs(64)
    ws = I.generate(specs, procs=16)
    sts = [mlbm.build_stencils_for(w, K=16, s=sp["s"], bb_mode=1) for w, sp in zip(ws, specs)]
    ps = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, sp["g"], 0.0) for sp in specs]
    ctx = mlbm.batch_init(sts, ps)
    v, _ = mlbm.autotune(ctx, 3)
    n = sum(w.n for w in ws)
    rng = np.random.default_rng(8)
    ru = np.stack([1 + (0.01 * rng.standard_normal(n)).astype(np.float32).astype(np.float64),
                   (0.01 * rng.standard_normal(n)).astype(np.float32).astype(np.float64),
                   (0.01 * rng.standard_normal(n)).astype(np.float32).astype(np.float64)], 1)
    mlbm.set_fields(ctx, ru)
    mlbm.step(ctx, 1)
    b = mlbm.get_fields(ctx)
    for i, (w, sp) in enumerate(zip(ws, specs)):
        first, count = mlbm.batch_range(ctx, i)
        ex = mlbm.stencils_export(sts[i])
        t = _sample_targets(w, 30, 300 + i, np.nonzero(ex["link_mask"])[0])
        op = O.Operator(w, K=16, s=sp["s"], bb_mode=1, targets=t).check()
        a = O.mlbm1_step(op, ru[first:first + count], (sp["g"], 0.0))
        assert np.abs(b[first:first + count][t] - a).max() < 5 * pop_tol(1), (i, v)
    # graph replay (as the bench's timed steps) against direct launches
    direct = mlbm.batch_init(sts, ps)
    mlbm.set_kernel_variant(direct, v)
    mlbm.set_graphs(direct, False)
    for c in (ctx, direct):
        mlbm.set_fields(c, ru)
    mlbm.prepare_graphs(ctx)
    mlbm.step(ctx, 16)
    mlbm.step(direct, 16)
    assert np.array_equal(mlbm.get_fields(ctx), mlbm.get_fields(direct))
