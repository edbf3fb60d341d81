"""The lattice LBM of the library (the paper's comparison method) against the
oracle: on a regular lattice with s = h the oracle's meshless step is
bitwise the textbook index-shift LBM (pinned in test_oracle_flows), so the
two must agree to FP32 round-off, in a periodic box with a body force and in
a half-way bounce-back channel; and the wall force of a steady channel must
balance the total body force."""
import numpy as np
import pytest

import oracle as O
from paper_2312_14789_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_14789_gb300 import mlbm
    return mlbm


def _random_state(n, seed, amp=2e-3):
    _, W, _ = O.lattice_constants()
    rng = np.random.default_rng(seed)
    f = np.tile(W, (n, 1)) * (1 + amp * rng.uniform(-1, 1, (n, 9)))
    # FP32-representable shifted populations, so both sides start equal
    return (f - W).astype(np.float32).astype(np.float64) + W


@pytest.mark.parametrize("tau,tau_minus", [(0.7, 0.0), (0.9, 0.6)])
def test_periodic_lattice_matches_oracle(M, tau, tau_minus):
    nx, ny = 33, 17
    g = (1e-5, -2e-6)
    w = I.lattice(nx, ny)
    L = M.Lattice(np.zeros((ny, nx), np.uint8), M.Params(M.MODEL_BGK, tau, tau_minus, *g), periodic=(True, True))
    f0 = _random_state(w.n, 3)
    L.set_populations(f0)
    op = O.Operator(w, K=12, s=1.0, bb_mode=0).check()
    f = f0
    for n_steps in (1, 9):
        L.step(n_steps)
        for _ in range(n_steps):
            f = O.bgk_step(op, f, tau, g, tau_minus if tau_minus > 0 else None)
        assert np.abs(L.get_populations() - f).max() < 2e-6


def test_halfway_channel_matches_oracle(M):
    nx, ny = 21, 13
    g = (1e-5, 0.0)
    w = I.lattice_channel(nx, ny, 0.5)
    cell = np.zeros((ny + 2, nx), np.uint8)
    cell[0] = 1
    cell[-1] = 1
    L = M.Lattice(cell, M.Params(M.MODEL_BGK, 0.9, 0.0, *g), periodic=(True, False))
    f0 = _random_state(w.n, 5)
    full = np.tile(O.lattice_constants()[1], (nx * (ny + 2), 1))
    full[nx:nx * (ny + 1)] = f0
    L.set_populations(full)
    op = O.Operator(w, K=16, s=1.0, bb_mode=0).check()
    f = f0
    L.step(10)
    for _ in range(10):
        f = O.bgk_step(op, f, 0.9, g)
    got = L.get_populations()[nx:nx * (ny + 1)]
    assert np.abs(got - f).max() < 2e-6


def test_steady_channel_force_balances_body_force(M):
    nx, ny, g = 8, 17, 1e-6
    cell = np.zeros((ny + 2, nx), np.uint8)
    cell[0] = 1
    cell[-1] = 1
    L = M.Lattice(cell, M.Params(M.MODEL_BGK, 0.8, 0.0, g, 0.0), periodic=(True, False))
    L.step(20000)
    fx, fy = L.force()
    f = L.get_populations()
    rho = f.sum(1)[nx:nx * (ny + 1)]
    total = g * rho.sum()
    assert abs(fx / total - 1) < 1e-4, (fx, total)
    assert abs(fy) < 1e-6 * total


def test_trt_magic_channel_is_exact_parabola(M):
    """TRT with Lambda = (tau+ - 1/2)(tau- - 1/2) = 3/16 puts the half-way
    wall exactly half-way: the steady profile is the parabola
    u(y) = g y (H - y) / (2 nu), y = j + 1/2, H = ny."""
    nx, ny, g, tp = 4, 17, 1e-6, 0.8
    tm = 0.5 + (3.0 / 16.0) / (tp - 0.5)
    cell = np.zeros((ny + 2, nx), np.uint8)
    cell[0] = 1
    cell[-1] = 1
    L = M.Lattice(cell, M.Params(M.MODEL_BGK, tp, tm, g, 0.0), periodic=(True, False))
    L.step(30000)
    f = L.get_populations()[nx:nx * (ny + 1)]
    rho, ux, uy = O.macroscopics(f, (g, 0.0))
    nu = (tp - 0.5) / 3.0
    y = np.repeat(np.arange(ny) + 0.5, nx)
    exact = g * y * (ny - y) / (2 * nu)
    assert np.abs(ux - exact).max() <= 1e-5 * exact.max(), np.abs(ux - exact).max() / exact.max()
