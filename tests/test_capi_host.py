"""Host-side checks of the C-ABI library (no GPU needed).

* libmlbm.so loads and exports every function include/mlbm.h declares.
* The host stencil builder (grid neighbour search, Householder QR, block
  detection, link geometry) agrees with the oracle on the same node sets:
  neighbour ids and order bit-exact, node kinds / links exact, q and the
  least-squares matrix to FP64 round-off.
* Argument and geometry errors come back as status codes.
"""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2312_14789_gb300 import inputs as I
from paper_2312_14789_gb300 import mlbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mlbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mlbm_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = mlbm.lib()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert "sm_103a" in mlbm.version()


def _compare(w, K, s, bb_mode, use_lagrange=True, sigma=0.7071067811865476):
    st = mlbm.build_stencils_for(w, K=K, s=s, sigma_factor=sigma, bb_mode=bb_mode, use_lagrange=use_lagrange)
    ex = mlbm.stencils_export(st)
    op = O.Operator(w, K=K, s=s, sigma_factor=sigma, bb_mode=bb_mode, use_lagrange=use_lagrange).check()
    assert np.array_equal(ex["idx"], op.idx)
    assert np.array_equal(ex["kind"], op.kind)
    mask = (op.link * (1 << np.arange(9))).sum(1)
    assert np.array_equal(ex["link_mask"], mask)
    assert np.allclose(ex["q"], op.q, rtol=0, atol=1e-12)
    lag = op.kind == 1
    assert np.array_equal(ex["lag_center"][lag], op.lag_center[lag])
    assert np.allclose(ex["lag_h"][lag], op.lag_h[lag], rtol=1e-15, atol=0)
    wls = op.kind == 0
    if wls.any():
        scale = np.abs(op.M[wls]).max(axis=(1, 2), keepdims=True)
        assert np.abs(ex["M"][wls] - op.M[wls]).max() / scale.max() < 1e-10
        assert (np.abs(ex["M"][wls] - op.M[wls]) / scale).max() < 1e-9
    info = mlbm.stencils_info(st)
    assert info["n_wls"] == int(wls.sum()) and info["n_lagrange"] == int(lag.sum())
    assert info["n_links"] == int(op.link.sum())
    return st, ex, op


def test_builder_matches_oracle_poiseuille_channel():
    _compare(I.poiseuille_channel(40, 50, 0.2, seed=1), K=12, s=1.0, bb_mode=1)


@pytest.mark.parametrize("s", [1.0, 0.5])
def test_builder_matches_oracle_lattices(s):
    _compare(I.lattice(16, 12), K=12, s=s, bb_mode=1)
    _, ex, _ = _compare(I.lattice_channel(8, 10, 0.5), K=16, s=s, bb_mode=0)
    _compare(I.lattice_channel(8, 10, 0.0), K=16, s=s, bb_mode=1)


def test_builder_matches_oracle_small_karman():
    w = I.karman(seed=2, scale=0.25)
    assert 10000 < w.n < 30000
    _compare(w, K=16, s=1.0, bb_mode=0)


def test_builder_matches_oracle_small_porous():
    w = I.porous(seed=5, n_target=15000)
    _compare(w, K=16, s=1.0, bb_mode=1)
    _compare(w, K=16, s=0.25, bb_mode=1)


def test_builder_errors():
    w = I.lattice(6, 6)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.build_stencils_for(w, K=10, s=1.0)
    assert e.value.status == 1
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.build_stencils_for(w, K=12, s=-1.0)
    assert e.value.status == 1
    # collinear nodes: degenerate least squares
    xy = np.stack([np.arange(20.0), np.full(20, 0.5)], 1)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.build_stencils(xy, np.zeros(20, np.uint8), (0, 0, 20, 1), (0, 0, 2, 2), K=8, use_lagrange=False)
    assert e.value.status == 2
    # node inside a disk
    xy = I.lattice(8, 8).xy
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.build_stencils(xy, np.zeros(64, np.uint8), (0, 0, 8, 8), (0, 0, 0, 0), disks=[[3.0, 3.0, 1.5]], K=12)
    assert e.value.status == 8


def test_builder_rejects_too_few_and_no_nodes():
    """Fewer nodes than the stencil size, and an empty node set, are
    MLBM_E_INVALID before any work; one partition per node is a valid split
    of a small set, more partitions than nodes is not."""
    xy = I.lattice(3, 3).xy
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.build_stencils(xy, np.zeros(9, np.uint8), (0, 0, 3, 3), (0, 0, 0, 0), K=12)
    assert e.value.status == 1
    with pytest.raises((mlbm.MlbmError, ValueError)) as e:
        mlbm.build_stencils(np.zeros((0, 2)), np.zeros(0, np.uint8), (0, 0, 3, 3), (0, 0, 0, 0), K=12)
    w = I.lattice(5, 5)
    st = mlbm.build_stencils_for(w, K=12, s=1.0)
    plan = mlbm.partition_plan(st, 25)
    assert np.all(plan["n_owned"] == 1) and np.all(plan["n_halo"] == 11)
    with pytest.raises(mlbm.MlbmError):
        mlbm.partition_plan(st, 26)


@pytest.mark.parametrize("order", [1, 2, 3, 0])
def test_reordering_keeps_the_stencils(order):
    """Re-ordering the device node order changes no stencil datum in the
    caller's order (bit-exact), and the orders differ as positions."""
    w = I.karman(seed=2, scale=0.25, lattice_beyond_d=1.0)
    st = mlbm.build_stencils_for(w, K=16, s=0.5, bb_mode=0)
    ref = mlbm.stencils_export(st)
    assert mlbm.stencils_order(st) == 0
    mlbm.stencils_set_order(st, order)
    assert mlbm.stencils_order(st) == order
    got = mlbm.stencils_export(st)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    # back to Hilbert and again
    mlbm.stencils_set_order(st, 0)
    got = mlbm.stencils_export(st)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    with pytest.raises(mlbm.MlbmError):
        mlbm.stencils_set_order(st, 7)


@pytest.mark.parametrize("case", ["porous", "karman"])
def test_builder_rbf_weights_match_oracle(case):
    """RBF-FD weights of the host builder (FP64 LU) against the oracle's
    (long-double Gauss-Jordan) for every interpolated direction, including
    the reflected points of interpolated bounce-back links."""
    if case == "porous":
        w, s, bb = I.porous(seed=5, n_target=4000), 0.5, 1
    else:
        w, s, bb = I.karman(seed=2, scale=0.25), 0.5, 0
    st = mlbm.build_stencils_for(w, K=16, s=s, bb_mode=bb, interp=mlbm.INTERP_RBF)
    W = mlbm.stencils_export_weights(st)
    ex = mlbm.stencils_export(st)
    op = O.Operator(w, K=16, s=s, bb_mode=bb, interp="rbf").check()
    assert np.array_equal(ex["kind"], op.kind)
    assert np.array_equal(ex["idx"], op.idx)
    sel = op.kind == 0
    for k in range(1, 9):
        interp_k = sel & ~((op.link[:, k] != 0) & (bb == 0))
        err = np.abs(W[interp_k, k] - op.W[interp_k, k]).max()
        assert err < 1e-8, (k, err)


@pytest.mark.parametrize("case", ["porous", "karman", "jittered"])
def test_builder_points_stencils_match_oracle(case):
    """RBF-FD stencils per Lagrangian point (Sec. 2.2, N_L = 25): the host
    builder's union stencils (grid search around each departure point) are
    the oracle's (brute force) node for node, and every direction's weights
    agree to FP64 round-off; a k_max below the union is rejected."""
    if case == "porous":
        w, s, bb = I.porous(seed=10, n_target=3000, porosity=0.7), 1.0, 1
    elif case == "karman":
        w, s, bb = I.karman(seed=2, scale=0.25), 0.5, 0
    else:
        w, s, bb = I.jittered_periodic(24, 20, 0.25, seed=7), 0.8, 1
    st = mlbm.build_stencils_for(w, K=64, s=s, bb_mode=bb, interp=mlbm.INTERP_RBF_POINTS, n_l=25)
    ex = mlbm.stencils_export(st)
    W = mlbm.stencils_export_weights(st)
    op = O.Operator(w, K=16, s=s, bb_mode=bb, interp="rbf_points", n_l=25, k_max=64).check()
    assert np.array_equal(ex["kind"], op.kind)
    sel = op.kind == 0
    assert np.array_equal(ex["idx"][sel], op.idx[sel])          # same union, same slot order
    for k in range(1, 9):
        rows = sel & ~((op.link[:, k] != 0) & (bb == 0))
        assert np.abs(W[rows, k] - op.W[rows, k]).max() < 1e-10, k
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.build_stencils_for(w, K=28, s=s, bb_mode=bb, interp=mlbm.INTERP_RBF_POINTS, n_l=25)
    assert e.value.status == 1


def test_context_calls_reject_null_arguments_without_a_device():
    """Argument checks come before any device work: a NULL context gives
    MLBM_E_INVALID (1) from the calls that take one."""
    L = mlbm.lib()
    d = np.zeros(2)
    assert L.mlbm_wall_stress_force(None, None, None, None, 0, d.ctypes.data, d.ctypes.data + 8) == 1
    assert L.mlbm_step(None, 1) == 1
    assert L.mlbm_drag_lift(None, 1.0, 1.0, None, None, None, None) == 1
    assert L.mlbm_permeability(None, None, None, None, None) == 1
