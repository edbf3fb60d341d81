"""Bounded device waits: a wait that runs out is reported, and the context
recovers.

The bulk-copy ring step kernels (variants 4..7) wait on shared-memory
barriers for their tile copies, each wait bounded by the context's wait
limit.  The test asks one launch to withhold the copies of block 0's first
tile (mlbm_test_withhold_copy), so that block's consumers wait for a tile
that never arrives: with a 1 ms limit the launch must end on its own, the
next synchronising call must return MLBM_E_TIMEOUT, and after a clean state
is loaded the context must step exactly as a fresh one.  Nothing faults or
traps: the kernel records an error word, drains its own copies in flight and
returns.
"""
import numpy as np
import pytest

from paper_2312_14789_gb300 import inputs as I
from paper_2312_14789_gb300 import mlbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [4, 7, 27, 28])
@pytest.mark.parametrize("model", ["bgk", "tau1"])
def test_withheld_copy_times_out_and_context_recovers(model, variant):
    w = I.porous(seed=47, n_target=20000, porosity=0.7)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED)
    p = mlbm.Params(mlbm.MODEL_BGK, 0.8, 0.0, 1e-5, 0.0) if model == "bgk" else \
        mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0)
    ref = mlbm.init(st, p)
    ctx = mlbm.init(st, p)
    for c in (ref, ctx):
        mlbm.set_kernel_variant(c, variant)
        mlbm.set_wait_limit(c, 1e-3)
    rng = np.random.default_rng(3)
    ru = np.zeros((w.n, 3))
    ru[:, 0] = 1.0 + 1e-3 * rng.standard_normal(w.n)
    ru[:, 1] = 1e-3 * rng.standard_normal(w.n)
    for c in (ref, ctx):
        mlbm.set_fields(c, ru)
    mlbm.step(ref, 3)
    want = mlbm.get_fields(ref)

    mlbm.test_withhold_copy(ctx)
    mlbm.step(ctx, 1)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.get_fields(ctx)
    assert e.value.status == 6, str(e.value)
    # the error word is cleared once reported; a clean state steps as usual
    mlbm.set_fields(ctx, ru)
    mlbm.step(ctx, 3)
    got = mlbm.get_fields(ctx)
    assert np.array_equal(got, want)


def test_withhold_needs_a_ring_variant_and_limits_are_checked():
    w = I.porous(seed=47, n_target=3000, porosity=0.7)
    st = mlbm.build_stencils_for(w, K=16, s=1.0, bb_mode=mlbm.BB_INTERPOLATED)
    ctx = mlbm.init(st, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-5, 0.0))
    mlbm.set_kernel_variant(ctx, 11)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.test_withhold_copy(ctx)
    assert e.value.status == 1
    for bad in (0.0, 5e-5, 61.0, float("nan")):
        with pytest.raises(mlbm.MlbmError):
            mlbm.set_wait_limit(ctx, bad)
    # a graph replay after the limit changed runs normally
    mlbm.set_kernel_variant(ctx, 5)
    mlbm.set_wait_limit(ctx, 0.5)
    mlbm.step(ctx, 32)
    ru = mlbm.get_fields(ctx)
    assert np.all(np.isfinite(ru))
