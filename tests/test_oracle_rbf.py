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
