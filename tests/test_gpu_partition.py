"""The partitioned step against the unpartitioned one, on one GPU.

A node set split into P position ranges, each advanced as its own context
with halo slots that receive the owners' new states after every step
(packed on the owner, copied into the receiver's own memory), must give the
unpartitioned context's states bit for bit: every node runs the same
arithmetic in the same order on the same neighbour values.  Cases cover the
tau = 1 and BGK models, interpolated and simple bounce-back, Lagrange,
equilibrium and least-squares nodes (the hybrid vortex street), equal and
uneven splits, and kernel variants from the plain, persistent,
dependent-launch and bulk-copy ring families.
"""
import numpy as np
import pytest

import oracle as O
from paper_2312_14789_gb300 import inputs as I
from paper_2312_14789_gb300 import mlbm

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "porous_tau1":
        w = I.porous(seed=50, n_target=30000, porosity=0.7)
        return w, 0.5, mlbm.BB_INTERPOLATED, mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 2e-5, 0.0)
    if name == "porous_bgk":
        w = I.porous(seed=51, n_target=20000, porosity=0.7)
        return w, 0.5, mlbm.BB_INTERPOLATED, mlbm.Params(mlbm.MODEL_BGK, 0.8, 0.0, 1e-5, 0.0)
    w = I.karman(seed=2, scale=0.25, lattice_beyond_d=1.0)
    return w, 0.5, mlbm.BB_SIMPLE, mlbm.Params(mlbm.MODEL_BGK, 0.62, 0.0, 0.0, 0.0)


def _initial(w, model, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 1e-2 * rng.standard_normal(w.n)
    ux, uy = 2e-2 * rng.standard_normal(w.n), 2e-2 * rng.standard_normal(w.n)
    if model == mlbm.MODEL_TAU1:
        return np.column_stack([rho, ux, uy])
    return O.equilibrium(rho, ux, uy) + 2e-3 * I.uniform_noise((w.n, 9), seed + 1)


@pytest.mark.parametrize("n_parts,variant,bounds", [(2, 26, None), (3, 11, None), (5, 4, None), (4, 25, "uneven"),
                                                    (2, 7, "uneven"), (1, 12, None), (3, 27, None)])
@pytest.mark.parametrize("name", ["porous_tau1", "porous_bgk", "karman_hybrid_bgk"])
def test_partitioned_step_is_bitwise_the_unpartitioned(name, n_parts, variant, bounds):
    w, s, bb, p = _case(name)
    st = mlbm.build_stencils_for(w, K=16, s=s, bb_mode=bb)
    if bounds == "uneven":
        cut = np.sort(np.random.default_rng(n_parts).choice(np.arange(1, w.n), n_parts - 1, replace=False))
        bounds = np.concatenate([[0], cut, [w.n]]).astype(np.int64)
    ref = mlbm.init(st, p)
    mlbm.set_kernel_variant(ref, variant)
    part = mlbm.Partitioned(st, p, n_parts, bounds)
    part.set_kernel_variant(variant)
    x0 = _initial(w, p.model, 3)
    if p.model == mlbm.MODEL_TAU1:
        mlbm.set_fields(ref, x0)
        part.set_fields(x0)
    else:
        mlbm.set_populations(ref, x0)
        part.set_populations(x0)
    plan = mlbm.partition_plan(st, n_parts, bounds)
    for q in range(n_parts):
        info = part.info(q)
        assert info["n_owned"] == plan["n_owned"][q] and info["n_halo"] == plan["n_halo"][q]
        assert info["halo_bytes_per_step"] == info["n_halo"] * (32 if p.model == mlbm.MODEL_BGK else 16)
    for n_steps in (1, 24):
        mlbm.step(ref, n_steps)
        part.step(n_steps)
        assert np.array_equal(part.get_fields(), mlbm.get_fields(ref)), (name, n_steps)
        if p.model == mlbm.MODEL_BGK:
            assert np.array_equal(part.get_populations(), mlbm.get_populations(ref))
    kp, kr = part.permeability(), mlbm.permeability(ref)
    for key in ("u_superficial", "u_intrinsic", "tortuosity"):
        assert abs(kp[key] - kr[key]) <= 1e-12 * max(abs(kr[key]), 1e-300), (key, kp[key], kr[key])
