"""Steady-state detection on the GPU against the oracle.

* The paper's criterion (Sec. 3.2): the relative change of the mean
  x-velocity over dn steps, per unit of physical time, below a threshold.
  The GPU run stops at the step its criterion fires; the oracle advances the
  same porous sample (MLBM1, tau = 1) from rest, records <u> every `check`
  steps and applies its own criterion to that record.  The two steps must
  agree exactly unless the oracle's Delta u at the deciding record lies
  within 1e-4 (relative) of the threshold, where FP32 and FP64 may decide
  one record apart.
* Failure detection on host-made failures: a state with a NaN, or with a
  non-positive density, is reported as MLBM_E_DIVERGED at the first
  evaluation, and the context stays usable.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_14789_gb300 import inputs as I
from paper_2312_14789_gb300 import mlbm

pytestmark = pytest.mark.gpu


def _box(w):
    return (w.box[2] - w.box[0]) * (w.box[3] - w.box[1])


def _oracle_record(w, s, g, check, steps):
    op = O.Operator(w, K=16, s=s, bb_mode=1).check()
    ru = np.zeros((w.n, 3))
    ru[:, 0] = 1.0
    rec = [0.0]
    for _ in range(steps // check):
        ru = O.run_mlbm1(op, ru, (g, 0.0), check)
        rec.append(O.mean_velocity(ru[:, 1], w.area, None, total_area=_box(w))[0])
    return np.array(rec)


def _near_threshold(rec, t, check, dn, dt, thr):
    j, lag = t // check, dn // check
    rate = abs(rec[j] - rec[j - lag]) / (abs(rec[j - lag]) * dt * dn)
    return abs(rate / thr - 1) < 1e-4


def _assert_same_step(t_gpu, rec, check, dn, dt, thr):
    t_or = O.steady_mean_step(rec, check, dn, dt, thr)
    assert t_or > 0, "the oracle record is too short"
    if t_gpu != t_or:
        assert abs(t_gpu - t_or) == check and _near_threshold(rec, min(t_gpu, t_or), check, dn, dt, thr), \
            (t_gpu, t_or)


def test_paper_criterion_matches_oracle_single():
    w = I.porous(seed=43, n_target=4000, porosity=0.7)
    s, g, dn, check, thr = 1.0, 1e-5, 2000, 100, 1e-2
    st = mlbm.build_stencils_for(w, K=16, s=s, bb_mode=mlbm.BB_INTERPOLATED)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0))
    t_gpu = mlbm.run_to_steady_mean(ctx, thr, dn, check, 0.0, max_steps=200_000)
    # from rest the first evaluation (t = dn) compares against <u>(0) = 0
    assert t_gpu >= dn + check
    dt = O.paper_time_step(1.0, s, math.sqrt(_box(w)))
    rec = _oracle_record(w, s, g, check, t_gpu + 3 * dn)
    _assert_same_step(t_gpu, rec, check, dn, dt, thr)
    # the same context continued by the field-norm criterion is unaffected
    assert mlbm.permeability(ctx)["k"] > 0


def test_paper_criterion_matches_oracle_batch_with_explicit_time_steps():
    ws = [I.porous(seed=44, n_target=3000, porosity=0.7), I.porous(seed=45, n_target=5000, porosity=0.75)]
    ss, gs = [1.0, 0.5], [1e-5, 4e-5]
    dn, check, thr = 1000, 100, 2e-2
    sts = [mlbm.build_stencils_for(w, K=16, s=s, bb_mode=mlbm.BB_INTERPOLATED) for w, s in zip(ws, ss)]
    ps = [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, g, 0.0) for g in gs]
    dts = [2e-4, 5e-5]
    ctx = mlbm.batch_init(sts, ps)
    taken = mlbm.batch_run_to_steady_mean(ctx, thr, dn, check, dts, max_steps=200_000)
    for w, s, g, dt, t in zip(ws, ss, gs, dts, taken):
        assert t >= dn
        rec = _oracle_record(w, s, g, check, int(max(taken)) + 3 * dn)
        _assert_same_step(int(t), rec, check, dn, dt, thr)


def test_paper_criterion_rejects_bad_arguments():
    w = I.porous(seed=43, n_target=2000, porosity=0.7)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0))
    for args in [(0.0, 1000, 100, 0.0), (1e-2, 1000, 300, 0.0), (1e-2, 1000, 100, -1.0)]:
        with pytest.raises(mlbm.MlbmError) as e:
            mlbm.run_to_steady_mean(ctx, *args, max_steps=1000)
        assert e.value.status == 1
    b = mlbm.batch_init([st, st], [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0)] * 2)
    with pytest.raises(mlbm.MlbmError):
        mlbm.run_to_steady_mean(b, 1e-2, 1000, 100, 0.0, max_steps=1000)
    with pytest.raises(mlbm.MlbmError):
        mlbm.batch_run_to_steady_mean(b, 1e-2, 1000, 100, [1.0, 0.0], max_steps=1000)


# ------------------------------------------------------- divergence detection
def _porous_ctx(n=3000, seed=46):
    w = I.porous(seed=seed, n_target=n, porosity=0.7)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED)
    return w, st


@pytest.mark.parametrize("bad", ["nan_velocity", "negative_density", "inf_density"])
def test_host_injected_divergence_is_reported(bad):
    w, st = _porous_ctx()
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0))
    ru = np.zeros((w.n, 3))
    ru[:, 0] = 1.0
    i = w.n // 3
    if bad == "nan_velocity":
        ru[i, 1] = np.nan
    elif bad == "negative_density":
        ru[i, 0] = -0.5
    else:
        ru[i, 0] = np.inf
    mlbm.set_fields(ctx, ru)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.run_to_steady(ctx, 1e-7, 1000, 10_000, check=100)
    assert e.value.status == 5, str(e.value)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.run_to_steady_mean(ctx, 1e-2, 1000, 100, 0.0, max_steps=10_000)
    assert e.value.status == 5
    # the context stays usable: a clean state runs to steady state
    ru[i] = (1.0, 0.0, 0.0)
    mlbm.set_fields(ctx, ru)
    assert mlbm.run_to_steady(ctx, 1e-7, 1000, 100_000, check=100) > 0


def test_divergence_names_the_sample_in_a_batch():
    w, st = _porous_ctx()
    ps = [mlbm.Params(mlbm.MODEL_BGK, 0.8, 0.0, 1e-5, 0.0)] * 3
    ctx = mlbm.batch_init([st, st, st], ps)
    f = O.equilibrium(np.ones(3 * w.n), 0.0, 0.0)
    f[2 * w.n + 5, 3] = np.nan
    mlbm.set_populations(ctx, f)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.batch_run_to_steady(ctx, 1e-7, 1000, 10_000, check=100)
    assert e.value.status == 5 and "sample 2" in str(e.value)
