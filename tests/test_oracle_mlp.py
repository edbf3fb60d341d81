"""Pins of the MLP oracle: backpropagation against central finite differences
of the loss (FP64, no rounding), the Adam step against its closed form for a
single step, and the bfloat16 rounding helper against exact cases."""
import numpy as np
import pytest

from oracle import mlp as M


def test_bf16_rounding():
    assert M.bf16(1.0) == 1.0
    assert M.bf16(1.0 + 2 ** -9) == 1.0          # below half an ulp (ulp = 2^-7)
    assert M.bf16(1.0 + 2 ** -8) == 1.0          # tie -> even
    assert M.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie -> even (up)
    assert M.bf16(-3.0) == -3.0
    x = np.random.default_rng(0).normal(size=1000)
    assert np.all(np.abs(M.bf16(x) - x) <= np.abs(x) * 2 ** -8 + 1e-300)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradients_match_finite_differences(seed):
    rng = np.random.default_rng(seed)
    params = M.init_params(seed)
    for l in range(1, 8, 2):
        params[l] = 0.1 * rng.standard_normal(params[l].shape)   # non-zero biases
    X = rng.normal(size=(37, 16))
    T = rng.normal(size=(37, 2))
    g = M.gradients(params, X, T)
    h = 1e-6
    for pi, p in enumerate(params):
        flat = p.ravel()
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = M.loss(params, X, T)
            flat[i] = old - h
            lm = M.loss(params, X, T)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[pi].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (pi, i, fd, an)


def test_adam_first_step_closed_form():
    p = [np.array([1.0, -2.0])]
    gr = [np.array([0.5, -3.0])]
    m = [np.zeros(2)]
    v = [np.zeros(2)]
    newp, newm, newv = M.adam_step(p, gr, m, v, 1, lr=1e-2)
    # first bias-corrected step moves every parameter by lr * sign(g) (up to eps)
    assert np.allclose(newp[0], p[0] - 1e-2 * np.sign(gr[0]), rtol=0, atol=1e-9)
    assert np.allclose(newm[0], 0.1 * gr[0]) and np.allclose(newv[0], 0.001 * gr[0] ** 2)


def test_pack_roundtrip():
    params = M.init_params(3)
    v = M.pack(params)
    assert v.size == M.n_params() == 16 * 64 + 64 + 2 * (64 * 64 + 64) + 64 * 2 + 2
    for a, b in zip(params, M.unpack(v)):
        assert np.array_equal(a, b)
