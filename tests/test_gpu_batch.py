"""Batched multi-sample contexts and captured step graphs (GPU).

A batch runs independent samples in the same fused launches; every sample
must evolve exactly as it does alone in its own context (same per-node
arithmetic, only the node numbering is offset), and the per-sample
observables must match the single-context ones.
"""
import numpy as np
import pytest

from paper_2312_14789_gb300 import inputs as I
from paper_2312_14789_gb300 import mlbm

pytestmark = pytest.mark.gpu


def _samples():
    ws = [I.porous(seed=31, n_target=9000, porosity=0.75), I.porous(seed=32, n_target=14000, porosity=0.6),
          I.porous(seed=33, n_target=6000, porosity=0.85)]
    ss = [1.0, 0.5, 0.25]
    ps = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0), mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 2e-5, 1e-6),
          mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 5e-6, 0.0)]
    return ws, ss, ps


@pytest.mark.parametrize("variant", [1, 4, 11, 12])
def test_batch_samples_evolve_as_alone(variant):
    ws, ss, ps = _samples()
    sts = [mlbm.build_stencils_for(w, K=16, s=s, bb_mode=1) for w, s in zip(ws, ss)]
    batch = mlbm.batch_init(sts, ps)
    mlbm.set_kernel_variant(batch, variant)
    assert mlbm.batch_size(batch) == 3
    mlbm.step(batch, 40)
    fb = mlbm.get_fields(batch)
    pb = mlbm.batch_permeability(batch)
    for i, (st, p) in enumerate(zip(sts, ps)):
        ctx = mlbm.init(st, p)
        mlbm.set_kernel_variant(ctx, variant)
        mlbm.step(ctx, 40)
        first, count = mlbm.batch_range(batch, i)
        assert count == st.n
        assert np.array_equal(fb[first:first + count], mlbm.get_fields(ctx))
        pm = mlbm.permeability(ctx)
        assert pb["k"][i] == pm["k"] and pb["tortuosity"][i] == pm["tortuosity"]


@pytest.mark.parametrize("interp", ["rbf", "rbf_points"])
def test_rbf_batch_samples_evolve_as_alone(interp):
    """RBF-FD stencils in a batch (the weight rows are read from each
    sample's own stencils when the batch is built): every sample evolves
    exactly as alone."""
    ws, ss, ps = _samples()
    if interp == "rbf":
        sts = [mlbm.build_stencils_for(w, K=16, s=s, bb_mode=1, interp=mlbm.INTERP_RBF) for w, s in zip(ws, ss)]
    else:
        sts = [mlbm.build_stencils_for(w, K=64, s=s, bb_mode=1, interp=mlbm.INTERP_RBF_POINTS, n_l=25)
               for w, s in zip(ws, ss)]
    batch = mlbm.batch_init(sts, ps)
    mlbm.step(batch, 25)
    fb = mlbm.get_fields(batch)
    for i, (st, p) in enumerate(zip(sts, ps)):
        ctx = mlbm.init(st, p)
        mlbm.step(ctx, 25)
        first, count = mlbm.batch_range(batch, i)
        assert np.array_equal(fb[first:first + count], mlbm.get_fields(ctx)), i


def test_batch_bgk_with_per_sample_tau():
    w1 = I.poiseuille_channel(20, 16, 0.2, seed=3)
    w2 = I.poiseuille_channel(24, 20, 0.2, seed=4)
    s1 = mlbm.build_stencils_for(w1, K=12, s=1.0, bb_mode=1)
    s2 = mlbm.build_stencils_for(w2, K=12, s=1.0, bb_mode=1)
    p1 = mlbm.Params(mlbm.MODEL_BGK, 0.8, 0.0, 1e-5, 0.0)
    p2 = mlbm.Params(mlbm.MODEL_BGK, 0.65, 0.9, 2e-5, 0.0)
    b = mlbm.batch_init([s1, s2], [p1, p2])
    mlbm.step(b, 50)
    rho_b, u_b = mlbm.macroscopics(b)
    for i, (st, p) in enumerate(((s1, p1), (s2, p2))):
        c = mlbm.init(st, p)
        mlbm.step(c, 50)
        first, count = mlbm.batch_range(b, i)
        rho, u = mlbm.macroscopics(c)
        assert np.array_equal(u_b[first:first + count], u) and np.array_equal(rho_b[first:first + count], rho)


def test_batch_run_to_steady_reports_each_sample():
    ws = [I.lattice_channel(4, 8, 0.5), I.lattice_channel(4, 14, 0.5)]
    sts = [mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=0) for w in ws]
    ps = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0)] * 2
    b = mlbm.batch_init(sts, ps)
    taken = mlbm.batch_run_to_steady(b, 1e-8, 200, 40000)
    assert np.all(taken > 0)
    assert taken[0] < taken[1]  # the narrower channel relaxes first


@pytest.mark.parametrize("criterion", ["field_norm", "mean_velocity"])
@pytest.mark.parametrize("variant", [25, 5])
def test_batch_run_to_steady_holds_converged_samples(criterion, variant):
    """A tau = 1 batch holds each converged sample at its steady state: every
    sample ends bit for bit where a single-sample run of it ends, at the same
    step, and the batch's node kinds are restored afterwards (its next steps
    equal those of a fresh batch loaded with the same fields)."""
    ws, ss, ps = _samples()
    sts = [mlbm.build_stencils_for(w, K=16, s=s, bb_mode=1) for w, s in zip(ws, ss)]
    batch = mlbm.batch_init(sts, ps)
    mlbm.set_kernel_variant(batch, variant)
    if criterion == "field_norm":
        run_b = lambda c: mlbm.batch_run_to_steady(c, 1e-6, 200, 40000, check=100)
        run_1 = lambda c: mlbm.run_to_steady(c, 1e-6, 200, 40000, check=100)
    else:
        run_b = lambda c: mlbm.batch_run_to_steady_mean(c, 5e-2, 1000, 100, [1e-4] * 3, max_steps=40000)
        run_1 = lambda c: mlbm.run_to_steady_mean(c, 5e-2, 1000, 100, 1e-4, max_steps=40000)
    taken = run_b(batch)
    assert len(set(int(t) for t in taken)) > 1   # the samples converge at different steps
    fb = mlbm.get_fields(batch)
    for i, (st, p) in enumerate(zip(sts, ps)):
        ctx = mlbm.init(st, p)
        mlbm.set_kernel_variant(ctx, variant)
        t1 = run_1(ctx)
        first, count = mlbm.batch_range(batch, i)
        assert int(taken[i]) == int(t1)
        assert np.array_equal(fb[first:first + count], mlbm.get_fields(ctx)), i
    fresh = mlbm.batch_init(sts, ps)
    mlbm.set_kernel_variant(fresh, variant)
    mlbm.set_fields(fresh, fb)
    mlbm.step(batch, 37)
    mlbm.step(fresh, 37)
    assert np.array_equal(mlbm.get_fields(batch), mlbm.get_fields(fresh))


def test_graph_replay_matches_direct_launches():
    w = I.porous(seed=34, n_target=8000)
    st = mlbm.build_stencils_for(w, K=16, s=0.5, bb_mode=1)
    p = mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0)
    a = mlbm.init(st, p)
    b = mlbm.init(st, p)
    mlbm.set_graphs(b, False)
    for n in (16, 33, 48, 7):
        mlbm.step(a, n)
        mlbm.step(b, n)
    assert mlbm.step_count(a) == mlbm.step_count(b) == 104
    assert np.array_equal(mlbm.get_fields(a), mlbm.get_fields(b))


def test_node_order_autotuner():
    """The order autotuner tries every node order, leaves the stencils in the
    fastest, and the physics does not depend on the order (FP32 summation
    order only)."""
    from paper_2312_14789_gb300 import inputs as I
    ws = [I.porous(seed=s, n_target=8000, porosity=0.7) for s in (31, 32)]
    sts = [mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED) for w in ws]
    ps = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0)] * 2
    ref = mlbm.batch_init(sts, ps)
    mlbm.step(ref, 50)
    ru_ref = mlbm.get_fields(ref)
    order, variant, ms = mlbm.autotune_order(sts, ps, 3)
    assert order in (0, 1, 2, 3) and ms > 0
    assert all(mlbm.stencils_order(s) == order for s in sts)
    for o in (1, 2, 3):
        for s in sts:
            mlbm.stencils_set_order(s, o)
        c = mlbm.batch_init(sts, ps)
        mlbm.step(c, 50)
        ru = mlbm.get_fields(c)
        assert np.abs(ru[:, 1:] - ru_ref[:, 1:]).max() <= 1e-5 * np.abs(ru_ref[:, 1:]).max() + 1e-12
        assert np.abs(ru[:, 0] - ru_ref[:, 0]).max() <= 1e-6
