"""Pins of the oracle's RBF-FD weights (Sec. 2.2: cubic polyharmonic spline
with quadratic augmentation) against scipy's independent RBF interpolator,
exact quadratic reproduction, the interpolation property at stencil nodes,
and, through the whole step, textbook lattice streaming where the departure
points are stencil nodes."""
import numpy as np
import pytest

import oracle as O
from paper_2312_14789_gb300 import inputs as I


def _stencil(K, seed):
    rng = np.random.default_rng(seed)
    off = rng.uniform(-2.5, 2.5, (K, 2))
    off[0] = 0.0
    return off


@pytest.mark.parametrize("K,seed", [(12, 0), (16, 1), (24, 2), (32, 3)])
def test_matches_scipy_cubic_rbf_with_quadratic_tail(K, seed):
    RBFInterpolator = pytest.importorskip("scipy.interpolate").RBFInterpolator
    off = _stencil(K, seed)
    rng = np.random.default_rng(seed + 10)
    f = rng.normal(size=K)
    interp = RBFInterpolator(off, f, kernel="cubic", degree=2)
    for d in [(-0.5, 0.0), (0.35, -0.35), (0.0, 0.7), (1.3, 0.9)]:
        w = O.rbf_weights(off, d)
        ref = float(interp(np.array([d]))[0])
        assert abs(w @ f - ref) <= 1e-9 * max(1.0, abs(ref)), (d, w @ f, ref)


def test_reproduces_quadratics_and_interpolates():
    off = _stencil(16, 5)
    rng = np.random.default_rng(6)
    c = rng.normal(size=6)
    quad = lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
    f = quad(off[:, 0], off[:, 1])
    for d in [(-0.5, 0.0), (0.2, 0.9), (-1.1, -0.4)]:
        w = O.rbf_weights(off, d)
        assert abs(w @ f - quad(*d)) <= 1e-11
        assert abs(w.sum() - 1.0) <= 1e-12
    # at a stencil node the interpolant takes the node's value: one-hot weights
    w = O.rbf_weights(off, tuple(off[7]))
    e = np.zeros(16)
    e[7] = 1.0
    assert np.abs(w - e).max() <= 1e-10


def test_lattice_streaming_is_textbook_with_rbf():
    """On a periodic lattice with s = h and no Lagrange blocks, every departure
    point is a lattice node, so the interpolating RBF-FD weights stream exactly
    (the least-squares fit would smooth)."""
    w = I.lattice(17, 13)
    op = O.Operator(w, K=16, s=1.0, bb_mode=0, use_lagrange=False, interp="rbf").check()
    rng = np.random.default_rng(2)
    f = O.equilibrium(1 + 0.01 * rng.standard_normal(w.n), 0.01 * rng.standard_normal(w.n),
                      0.01 * rng.standard_normal(w.n))
    g = O.bgk_step(op, f, 1.0)
    # tau = 1: the result is the equilibrium of the streamed moments; stream by index shift
    E, _, _ = O.lattice_constants()
    nx, ny = 17, 13
    ix, iy = np.arange(w.n) % nx, np.arange(w.n) // nx
    streamed = np.empty_like(f)
    for k in range(9):
        src = ((iy - E[k, 1]) % ny) * nx + (ix - E[k, 0]) % nx
        streamed[:, k] = f[src, k]
    rho = streamed.sum(1)
    ux = (streamed @ E[:, 0]) / rho
    uy = (streamed @ E[:, 1]) / rho
    assert np.abs(g - O.equilibrium(rho, ux, uy)).max() <= 1e-12
    op_w = O.Operator(w, K=16, s=1.0, bb_mode=0, use_lagrange=False, interp="wls").check()
    assert np.abs(O.bgk_step(op_w, f, 1.0) - g).max() > 1e-8   # the fit does not interpolate


# ------------------------------------------- stencils per Lagrangian point
def _dep_rows(w, s, n_l, t):
    """Independent construction of node t's per-direction rows: scipy's
    periodic k-d tree for the n_l nearest nodes of each departure point
    x - s e_k (ties broken by node id afterwards), scipy's cubic RBF
    interpolator with quadratic tail for the weights (unit data vectors)."""
    spatial = pytest.importorskip("scipy.spatial")
    RBFInterpolator = pytest.importorskip("scipy.interpolate").RBFInterpolator
    E, _, _ = O.lattice_constants()
    x0, y0, x1, y1 = w.box
    L = np.array([x1 - x0, y1 - y0])
    per = np.array([w.sides[0] == I.PERIODIC, w.sides[2] == I.PERIODIC])
    rows = {}
    for k in range(1, 9):
        d = -s * E[k].astype(float)
        off = w.xy - w.xy[t]
        for a in range(2):
            if per[a]:
                off[:, a] = np.where(off[:, a] >= 0.5 * L[a], off[:, a] - L[a], off[:, a])
                off[:, a] = np.where(off[:, a] < -0.5 * L[a], off[:, a] + L[a], off[:, a])
        d2 = ((off - d) ** 2).sum(1)
        tree = spatial.cKDTree(off - d)
        _, cand = tree.query(np.zeros(2), k=n_l + 8)
        cand = np.asarray(cand)
        order = np.lexsort((cand, d2[cand]))      # by distance, then node id
        members = cand[order][:n_l]
        assert d2[cand[order][n_l]] >= d2[members[-1]]
        interp_w = np.empty(n_l)
        for m in range(n_l):
            e = np.zeros(n_l)
            e[m] = 1.0
            interp_w[m] = float(RBFInterpolator(off[members], e, kernel="cubic", degree=2)(d[None])[0])
        rows[k] = dict(zip(members.tolist(), interp_w))
    return rows


@pytest.mark.parametrize("case", ["jittered", "porous"])
def test_points_stencils_match_scipy_nearest_and_rbf(case):
    if case == "jittered":
        w, s = I.jittered_periodic(24, 20, 0.25, seed=7), 0.8
    else:
        w, s = I.porous(seed=9, n_target=2500, porosity=0.7), 1.0
    op = O.Operator(w, K=16, s=s, bb_mode=1, use_lagrange=False, interp="rbf_points", n_l=25, k_max=64).check()
    rng = np.random.default_rng(3)
    ts = [t for t in rng.choice(w.n, 40, replace=False) if op.kind[t] == 0 and not op.link[t].any()][:12]
    assert len(ts) >= 8
    for t in ts:
        rows = _dep_rows(w, s, 25, t)
        ids = op.idx[t]
        for k in range(1, 9):
            got = {int(j): float(v) for j, v in zip(ids, op.W[t, k]) if v != 0.0}
            assert set(got) <= set(rows[k]), (t, k)
            for j, v in rows[k].items():
                assert abs(got.get(j, 0.0) - v) <= 1e-9, (t, k, j, got.get(j, 0.0), v)


def test_points_stencils_union_layout_and_reproduction():
    """The union holds the node and every direction's stencil in increasing
    node id, padded with the node at zero weight; every row reproduces
    quadratics at its departure point and sums to one; a union larger than
    k_max is rejected."""
    w, s = I.porous(seed=10, n_target=2000, porosity=0.7), 1.0
    op = O.Operator(w, K=16, s=s, bb_mode=1, interp="rbf_points", n_l=25, k_max=64).check()
    E, _, _ = O.lattice_constants()
    rng = np.random.default_rng(4)
    c = rng.normal(size=6)
    quad = lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
    x0, y0, x1, y1 = w.box
    n_checked = 0
    for t in range(w.n):
        if op.kind[t] != 0:
            continue
        ids = op.idx[t]
        used = ids[np.abs(op.W[t, 1:]).sum(0) > 0]
        nu = len(np.unique(np.concatenate([[t], used])))
        assert np.all(np.diff(ids[:nu]) > 0) or nu == 1
        assert np.all(ids[nu:] == t) and np.all(op.W[t, :, nu:] == 0.0)
        off = w.xy[ids] - w.xy[t]
        off[:, 0] -= (x1 - x0) * np.round(off[:, 0] / (x1 - x0))     # periodic in x
        for k in range(1, 9):
            if op.link[t, k]:
                dk = (1 - 2 * op.q[t, k]) * s * E[k]
            else:
                dk = -s * E[k]
            row = op.W[t, k]
            assert abs(row.sum() - 1.0) <= 1e-10
            assert abs(row @ quad(off[:, 0], off[:, 1]) - quad(*dk)) <= 1e-8
        n_checked += 1
    assert n_checked > 1000
    with pytest.raises(ValueError):
        O.Operator(w, K=16, s=s, bb_mode=1, interp="rbf_points", n_l=25, k_max=28).check()
