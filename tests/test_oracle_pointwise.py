"""Pins of the oracle's point-wise formulas against closed forms.

Equilibrium (Eq. (7)-(8)), moments (Eq. (9)), the second-order force source,
and the TRT collision (Eq. (3)-(5)).  The expected values are moments of the
D2Q9 velocity set, written here from Eq. (2) and Eq. (8), not by calling the
oracle's own tables.
"""
import numpy as np
import pytest

import oracle as O

# Eq. (2) and Eq. (8), typed from the paper for the test only
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0


def test_lattice_constants_match_paper():
    e, w, opp = O.lattice_constants()
    assert np.array_equal(e, E.astype(np.int64))
    assert np.allclose(w, W, rtol=0, atol=1e-16)
    for k in range(9):
        assert np.array_equal(e[opp[k]], -e[k])


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.1 * rng.standard_normal()
    u = 0.1 * rng.standard_normal(2)
    f = np.array([O.feq(k, rho, *u) for k in range(9)])
    assert abs(f.sum() - rho) < 1e-15
    assert np.allclose(f @ E, rho * u, rtol=0, atol=1e-16)
    # second moment: rho cs^2 I + rho u u
    P = np.einsum("k,ka,kb->ab", f, E, E)
    assert np.allclose(P, rho * CS2 * np.eye(2) + rho * np.outer(u, u), rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_source_moments(seed):
    rng = np.random.default_rng(100 + seed)
    rho = 1 + 0.1 * rng.standard_normal()
    u = 0.1 * rng.standard_normal(2)
    g = 1e-3 * rng.standard_normal(2)
    S = np.array([O.source(k, rho, *u, *g) for k in range(9)])
    F = rho * g
    assert abs(S.sum()) < 1e-17
    assert np.allclose(S @ E, F, rtol=0, atol=1e-18)
    P = np.einsum("k,ka,kb->ab", S, E, E)
    assert np.allclose(P, np.outer(u, F) + np.outer(F, u), rtol=0, atol=1e-18)


@pytest.mark.parametrize("tau_p,tau_m", [(0.8, 0.8), (1.0, 1.0), (0.53, 0.53 + 0.2), (0.6, 0.5 + 0.1875 / 0.1)])
def test_collision_conserves_mass_and_adds_force(tau_p, tau_m):
    rng = np.random.default_rng(7)
    for _ in range(10):
        f = W * (1 + 0.05 * rng.standard_normal(9))
        g = 1e-4 * rng.standard_normal(2)
        out = O.collide(f, tau_p, tau_m, *g)
        rho = f.sum()
        assert abs(out.sum() - rho) < 1e-15
        # sum f* e = sum f e + F  (rho u = sum f e + F/2, collision adds F/2 more)
        assert np.allclose(out @ E, f @ E + rho * g, rtol=0, atol=2e-16)


def test_collision_relaxes_to_equilibrium_at_tau_one():
    rng = np.random.default_rng(8)
    f = W * (1 + 0.05 * rng.standard_normal(9))
    out = O.collide(f, 1.0, 1.0, 0.0, 0.0)
    rho = f.sum()
    u = (f @ E) / rho
    assert np.allclose(out, [O.feq(k, rho, *u) for k in range(9)], rtol=0, atol=1e-16)


def test_trt_relaxes_odd_part_with_tau_minus():
    """Eq. (3)-(4): with tau+ = 1 the even part jumps to equilibrium, the odd
    non-equilibrium part is scaled by (1 - 1/tau-)."""
    rng = np.random.default_rng(9)
    f = W * (1 + 0.05 * rng.standard_normal(9))
    tau_m = 0.7
    out = O.collide(f, 1.0, tau_m, 0.0, 0.0)
    rho = f.sum()
    u = (f @ E) / rho
    fe = np.array([O.feq(k, rho, *u) for k in range(9)])
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    neq = f - fe
    odd = 0.5 * (neq - neq[opp])
    assert np.allclose(out, fe + (1 - 1 / tau_m) * odd, rtol=0, atol=1e-16)


def test_macroscopics_of_post_collision_state():
    rng = np.random.default_rng(10)
    g = (2e-5, -1e-5)
    f = W * (1 + 0.05 * rng.standard_normal(9))
    rho0 = f.sum()
    u0 = (f @ E) / rho0 + 0.5 * np.array(g)
    out = O.collide(f, 0.8, 0.8, *g)
    rho, ux, uy = O.macroscopics(out[None, :], g)
    assert abs(rho[0] - rho0) < 1e-15
    assert np.allclose([ux[0], uy[0]], u0, rtol=0, atol=2e-16)
