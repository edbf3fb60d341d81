"""Thin ctypes binding of the C ABI in include/mlbm.h (argument marshalling only).

Every function here forwards to libmlbm.so with the same name; all compute
happens in the library (host stencil builder, CUDA kernels).  There is no
Python fallback: if the library cannot be built or loaded, importing fails
with the reason.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

MODEL_BGK, MODEL_TAU1 = 0, 1
INTERP_WLS, INTERP_RBF, INTERP_RBF_POINTS = 0, 1, 2
ORDER_HILBERT, ORDER_MORTON, ORDER_ROWS, ORDER_INPUT = 0, 1, 2, 3
BB_SIMPLE, BB_INTERPOLATED = 0, 1
NODE_FLUID, NODE_WALL, NODE_EQ = 0, 1, 2
SIDE_PERIODIC, SIDE_SOLID, SIDE_OPEN = 0, 1, 2

STATUS = {0: "OK", 1: "INVALID", 2: "SINGULAR_STENCIL", 3: "CUDA", 4: "OOM", 5: "DIVERGED", 6: "TIMEOUT",
          7: "NOT_CONVERGED", 8: "GEOMETRY", 9: "IO"}

_i64, _i32, _dbl, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class MlbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mlbm {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Nodes(ctypes.Structure):
    _fields_ = [("n", _i64), ("xy", _vp), ("node_class", _vp), ("eq_values", _vp), ("area", _vp)]


class _Geometry(ctypes.Structure):
    _fields_ = [("x0", _dbl), ("y0", _dbl), ("x1", _dbl), ("y1", _dbl), ("side", _i32 * 4),
                ("n_disks", _i32), ("disks", _vp)]


class _Params(ctypes.Structure):
    _fields_ = [("model", _i32), ("tau", _dbl), ("tau_minus", _dbl), ("gx", _dbl), ("gy", _dbl)]


class _Info(ctypes.Structure):
    _fields_ = [("n", _i64), ("K", _i32), ("s", _dbl), ("n_wls", _i64), ("n_lagrange", _i64), ("n_eq", _i64),
                ("n_link_nodes", _i64), ("n_links", _i64), ("build_seconds", _dbl)]


_LIB = None
_LOCK = threading.Lock()


def lib():
    """Build (if stale) and load libmlbm.so.  Raises when either fails."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(_build.build())
            st = ctypes.c_int
            sig = {
                "mlbm_build_stencils": (st, [_vp, _vp, _i32, _dbl, _dbl, _i32, _i32, _vp]),
                "mlbm_build_stencils_ex": (st, [_vp, _vp, _i32, _dbl, _dbl, _i32, _i32, _i32, _vp]),
                "mlbm_build_stencils_points": (st, [_vp, _vp, _i32, _i32, _dbl, _i32, _i32, _vp]),
                "mlbm_stencils_export_weights": (st, [_vp, _vp]),
                "mlbm_stencils_free": (None, [_vp]),
                "mlbm_stencils_info": (st, [_vp, _vp]),
                "mlbm_stencils_set_order": (st, [_vp, _i32]),
                "mlbm_stencils_order": (_i32, [_vp]),
                "mlbm_autotune_order": (st, [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp]),
                "mlbm_stencils_export": (st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
                "mlbm_init": (st, [_vp, _vp, _vp, _vp, _vp]),
                "mlbm_destroy": (None, [_vp]),
                "mlbm_set_stream": (st, [_vp, _vp]),
                "mlbm_set_populations": (st, [_vp, _vp]),
                "mlbm_set_fields": (st, [_vp, _vp]),
                "mlbm_get_populations": (st, [_vp, _vp]),
                "mlbm_get_fields": (st, [_vp, _vp]),
                "mlbm_step": (st, [_vp, _i64]),
                "mlbm_step_count": (_i64, [_vp]),
                "mlbm_macroscopics": (st, [_vp, _vp, _vp]),
                "mlbm_drag_lift": (st, [_vp, _dbl, _dbl, _vp, _vp, _vp, _vp]),
                "mlbm_wall_stress_force": (st, [_vp, _vp, _vp, _vp, _i64, _vp, _vp]),
                "mlbm_permeability": (st, [_vp, _vp, _vp, _vp, _vp]),
                "mlbm_run_to_steady": (st, [_vp, _dbl, _i64, _i64, _vp]),
                "mlbm_run_to_steady_ex": (st, [_vp, _dbl, _i64, _i64, _i64, _vp]),
                "mlbm_save": (st, [_vp, ctypes.c_char_p]),
                "mlbm_load": (st, [_vp, ctypes.c_char_p]),
                "mlbm_set_timing": (st, [_vp, _i32]),
                "mlbm_last_step_ms": (_dbl, [_vp]),
                "mlbm_set_kernel_variant": (st, [_vp, _i32]),
                "mlbm_kernel_variant": (_i32, [_vp]),
                "mlbm_autotune_times": (_i32, [_vp, _vp, _i32]),
                "mlbm_autotune": (st, [_vp, _i32, _vp]),
                "mlbm_autotune_ex": (st, [_vp, _i32, _i32, _vp]),
                "mlbm_batch_init": (st, [_vp, _vp, _vp, _i32]),
                "mlbm_batch_size": (_i32, [_vp]),
                "mlbm_batch_range": (st, [_vp, _i32, _vp, _vp]),
                "mlbm_batch_permeability": (st, [_vp, _vp, _vp, _vp, _vp]),
                "mlbm_batch_run_to_steady": (st, [_vp, _dbl, _i64, _i64, _vp]),
                "mlbm_batch_run_to_steady_ex": (st, [_vp, _dbl, _i64, _i64, _i64, _vp]),
                "mlbm_batch_drag_lift": (st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
                "mlbm_set_graphs": (st, [_vp, _i32]),
                "mlbm_prepare_graphs": (st, [_vp]),
                "mlbm_run_to_steady_mean": (st, [_vp, _dbl, _i64, _i64, _dbl, _i64, _vp]),
                "mlbm_batch_run_to_steady_mean": (st, [_vp, _dbl, _i64, _i64, _vp, _i64, _vp]),
                "mlbm_set_wait_limit": (st, [_vp, _dbl]),
                "mlbm_partition_plan": (st, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
                "mlbm_partition_nodes": (st, [_vp, _i32, _vp, _i32, _vp, _vp]),
                "mlbm_part_init": (st, [_vp, _vp, _vp, _i32, _vp]),
                "mlbm_part_destroy": (None, [_vp]),
                "mlbm_part_info": (st, [_vp, _i32, _vp, _vp, _vp, _vp]),
                "mlbm_part_set_kernel_variant": (st, [_vp, _i32]),
                "mlbm_part_step": (st, [_vp, _i64]),
                "mlbm_part_set_fields": (st, [_vp, _vp]),
                "mlbm_part_get_fields": (st, [_vp, _vp]),
                "mlbm_part_set_populations": (st, [_vp, _vp]),
                "mlbm_part_get_populations": (st, [_vp, _vp]),
                "mlbm_part_permeability": (st, [_vp, _vp, _vp, _vp, _vp]),
                "mlbm_test_withhold_copy": (st, [_vp]),
                "mlbm_reduce_scratch_doubles": (_i64, [_i64]),
                "mlbm_reduce_fields_device": (st, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64, _vp, _vp]),
                "mlbm_reduce_noalloc_max_nodes": (_i64, []),
                "mlbm_reduce_fields_device_noalloc": (st, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
                "mlbm_mlp_param_count": (_i64, [_i32]),
                "mlbm_mlp_create": (st, [_vp, _i32, ctypes.c_uint64]),
                "mlbm_mlp_destroy": (None, [_vp]),
                "mlbm_mlp_outputs": (_i32, [_vp]),
                "mlbm_mlp_set_params": (st, [_vp, _vp]),
                "mlbm_mlp_get_params": (st, [_vp, _vp]),
                "mlbm_mlp_forward_device": (st, [_vp, _vp, _i64, _vp, _vp]),
                "mlbm_mlp_gradients_device": (st, [_vp, _vp, _vp, _i64, _vp, _vp, _vp]),
                "mlbm_mlp_train_device": (st, [_vp, _vp, _vp, _i64, _i64, _i64, ctypes.c_float, ctypes.c_uint64,
                                               _vp, _vp]),
                "mlbm_features_device": (st, [_vp, _vp, _dbl, _vp]),
                "mlbm_warm_start": (st, [_vp, _vp, _vp, _vp, _vp, _vp]),
                "mlbm_lattice_init": (st, [_vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp]),
                "mlbm_lattice_destroy": (None, [_vp]),
                "mlbm_lattice_step": (st, [_vp, _i64]),
                "mlbm_lattice_sync": (st, [_vp]),
                "mlbm_lattice_time_steps": (st, [_vp, _i64, _vp]),
                "mlbm_lattice_set_populations": (st, [_vp, _vp]),
                "mlbm_lattice_get_populations": (st, [_vp, _vp]),
                "mlbm_lattice_force": (st, [_vp, _vp, _vp]),
                "mlbm_last_error": (ctypes.c_char_p, []),
                "mlbm_version": (ctypes.c_char_p, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def _check(status):
    if status != 0:
        raise MlbmError(status, lib().mlbm_last_error().decode())


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def version() -> str:
    return lib().mlbm_version().decode()


# ------------------------------------------------------------------ stencils
class Stencils:
    def __init__(self, handle, n, K, keep):
        self.handle, self.n, self.K = handle, n, K
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.mlbm_stencils_free(self.handle)
            self.handle = None


def build_stencils(xy, node_class, box, sides, disks=None, eq_values=None, area=None, K=16, s=1.0,
                   sigma_factor=0.7071067811865476, bb_mode=BB_INTERPOLATED, use_lagrange=True,
                   interp=INTERP_WLS, n_l=25) -> Stencils:
    xy = _f64(xy)
    n = xy.shape[0]
    cls = np.ascontiguousarray(node_class, dtype=np.uint8)
    eqv = _f64(eq_values)
    ar = _f64(area)
    dk = _f64(np.zeros((0, 3)) if disks is None else np.asarray(disks).reshape(-1, 3))
    nodes = _Nodes(n, _ptr(xy), _ptr(cls), _ptr(eqv), _ptr(ar))
    geo = _Geometry(float(box[0]), float(box[1]), float(box[2]), float(box[3]), (_i32 * 4)(*[int(v) for v in sides]),
                    len(dk), _ptr(dk) if len(dk) else None)
    h = _vp()
    if interp == INTERP_RBF_POINTS:
        # K is the union width k_max; the departure stencils hold n_l nodes
        _check(lib().mlbm_build_stencils_points(ctypes.byref(nodes), ctypes.byref(geo), int(n_l), int(K), float(s),
                                                int(bb_mode), int(bool(use_lagrange)), ctypes.byref(h)))
    else:
        _check(lib().mlbm_build_stencils_ex(ctypes.byref(nodes), ctypes.byref(geo), int(K), float(s),
                                            float(sigma_factor), int(bb_mode), int(bool(use_lagrange)), int(interp),
                                            ctypes.byref(h)))
    return Stencils(h, n, int(K), None)


def build_stencils_for(w, **kw) -> Stencils:
    """build_stencils for an inputs.Workload."""
    return build_stencils(w.xy, w.node_class, w.box, w.sides, w.disks, w.eq_values, w.area, **kw)


def stencils_info(st: Stencils) -> dict:
    info = _Info()
    _check(lib().mlbm_stencils_info(st.handle, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in _Info._fields_}


def stencils_export_weights(st: Stencils) -> np.ndarray:
    """RBF-FD stencils: per-direction weights [n][9][K] in the caller's order."""
    W = np.empty((st.n, 9, st.K))
    _check(lib().mlbm_stencils_export_weights(st.handle, _ptr(W)))
    return W


def stencils_set_order(st: Stencils, order: int):
    _check(lib().mlbm_stencils_set_order(st.handle, int(order)))


def stencils_order(st: Stencils) -> int:
    return int(lib().mlbm_stencils_order(st.handle))


def autotune_order(stencils: list, params: list, steps_per_variant: int = 10, flush_l2: bool = False) -> tuple:
    """Pick the node order and kernel variant together; leaves the stencils in
    the winning order.  Returns (order, variant, ms per step)."""
    arr = (_vp * len(stencils))(*[s.handle for s in stencils])
    par = (_Params * len(params))(*[_Params(int(p.model), float(p.tau), float(p.tau_minus), float(p.gx), float(p.gy))
                                    for p in params])
    o, v, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().mlbm_autotune_order(arr, par, len(stencils), int(steps_per_variant), int(bool(flush_l2)),
                                     ctypes.byref(o), ctypes.byref(v), ctypes.byref(ms)))
    return o.value, v.value, ms.value


def stencils_export(st: Stencils) -> dict:
    n, K = st.n, st.K
    out = {"idx": np.empty((n, K), np.int64), "M": np.empty((n, 6, K)), "kind": np.empty(n, np.int32),
           "link_mask": np.empty(n, np.int32), "q": np.empty((n, 9)), "lag_h": np.empty(n),
           "lag_center": np.empty(n, np.int32)}
    _check(lib().mlbm_stencils_export(st.handle, *[_ptr(out[k]) for k in
                                                   ("idx", "M", "kind", "link_mask", "q", "lag_h", "lag_center")]))
    return out


# ------------------------------------------------------------------- context
@dataclass
class Params:
    model: int = MODEL_BGK
    tau: float = 0.8
    tau_minus: float = 0.0
    gx: float = 0.0
    gy: float = 0.0


class Context:
    def __init__(self, handle, n, model, stencils):
        self.handle, self.n, self.model = handle, n, model
        self._stencils = stencils

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.mlbm_destroy(self.handle)
            self.handle = None


def init(st: Stencils, params: Params, rho0=None, u0=None) -> Context:
    p = _Params(int(params.model), float(params.tau), float(params.tau_minus), float(params.gx), float(params.gy))
    r = _f64(rho0)
    u = _f64(u0)
    h = _vp()
    _check(lib().mlbm_init(ctypes.byref(h), st.handle, ctypes.byref(p), _ptr(r), _ptr(u)))
    return Context(h, st.n, params.model, st)


def destroy(ctx: Context):
    if ctx.handle:
        lib().mlbm_destroy(ctx.handle)
        ctx.handle = None


def set_stream(ctx: Context, stream_handle: int | None):
    _check(lib().mlbm_set_stream(ctx.handle, _vp(stream_handle) if stream_handle else None))


def set_populations(ctx: Context, f):
    f = _f64(f)
    assert f.shape == (ctx.n, 9)
    _check(lib().mlbm_set_populations(ctx.handle, _ptr(f)))


def set_fields(ctx: Context, rho_u):
    a = _f64(rho_u)
    assert a.shape == (ctx.n, 3)
    _check(lib().mlbm_set_fields(ctx.handle, _ptr(a)))


def get_populations(ctx: Context) -> np.ndarray:
    f = np.empty((ctx.n, 9))
    _check(lib().mlbm_get_populations(ctx.handle, _ptr(f)))
    return f


def get_fields(ctx: Context) -> np.ndarray:
    a = np.empty((ctx.n, 3))
    _check(lib().mlbm_get_fields(ctx.handle, _ptr(a)))
    return a


def step(ctx: Context, n_steps: int = 1):
    _check(lib().mlbm_step(ctx.handle, int(n_steps)))


def step_count(ctx: Context) -> int:
    return int(lib().mlbm_step_count(ctx.handle))


def macroscopics(ctx: Context):
    rho = np.empty(ctx.n)
    u = np.empty((ctx.n, 2))
    _check(lib().mlbm_macroscopics(ctx.handle, _ptr(rho), _ptr(u)))
    return rho, u


def drag_lift(ctx: Context, ref_length: float = 1.0, u_ref: float = 1.0):
    v = [ctypes.c_double() for _ in range(4)]
    _check(lib().mlbm_drag_lift(ctx.handle, float(ref_length), float(u_ref), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def wall_stress_force(ctx: Context, nodes, normals, ds) -> tuple:
    """Force (fx, fy) of the fluid on the walls by integrating the fluid
    stress along the listed wall nodes (caller's ids), with unit normals out of
    the solid and wall lengths per node; see inputs.wall_geometry."""
    nodes = np.ascontiguousarray(nodes, np.int64)
    normals = _f64(np.asarray(normals, np.float64).reshape(-1, 2))
    ds = _f64(ds)
    if not (len(nodes) == len(normals) == len(ds)):
        raise ValueError("nodes, normals and ds must have the same length")
    fx, fy = ctypes.c_double(), ctypes.c_double()
    _check(lib().mlbm_wall_stress_force(ctx.handle, _ptr(nodes), _ptr(normals), _ptr(ds), len(nodes),
                                        ctypes.byref(fx), ctypes.byref(fy)))
    return fx.value, fy.value


def permeability(ctx: Context):
    v = [ctypes.c_double() for _ in range(4)]
    _check(lib().mlbm_permeability(ctx.handle, *[ctypes.byref(x) for x in v]))
    k, us, ui, tv = (x.value for x in v)
    return {"k": k, "u_superficial": us, "u_intrinsic": ui, "tortuosity": tv}


def run_to_steady(ctx: Context, tol: float, window: int, max_steps: int, raise_on_max: bool = True,
                  check: int | None = None) -> int:
    """Steps to steady state (criterion checked every `check` steps, default `window`)."""
    taken = ctypes.c_int64()
    st = lib().mlbm_run_to_steady_ex(ctx.handle, float(tol), int(window), int(check or window), int(max_steps),
                                     ctypes.byref(taken))
    if st == 7 and not raise_on_max:
        return -int(taken.value)
    _check(st)
    return int(taken.value)


def run_to_steady_mean(ctx: Context, threshold: float = 1e-2, dn: int = 20000, check: int = 1000,
                       dt: float = 0.0, max_steps: int = 10_000_000, raise_on_max: bool = True) -> int:
    """Steps to the paper's steady state (Sec. 3.2: relative change of the
    mean velocity over dn steps per unit time below threshold); dt = 0: the
    paper's units."""
    taken = ctypes.c_int64()
    st = lib().mlbm_run_to_steady_mean(ctx.handle, float(threshold), int(dn), int(check), float(dt), int(max_steps),
                                       ctypes.byref(taken))
    if st == 7 and not raise_on_max:
        return -int(taken.value)
    _check(st)
    return int(taken.value)


def set_wait_limit(ctx: Context, seconds: float):
    _check(lib().mlbm_set_wait_limit(ctx.handle, float(seconds)))


def test_withhold_copy(ctx: Context):
    _check(lib().mlbm_test_withhold_copy(ctx.handle))


def save(ctx: Context, path: str):
    _check(lib().mlbm_save(ctx.handle, path.encode()))


def load(ctx: Context, path: str):
    _check(lib().mlbm_load(ctx.handle, path.encode()))


def set_timing(ctx: Context, enable: bool):
    _check(lib().mlbm_set_timing(ctx.handle, int(bool(enable))))


def last_step_ms(ctx: Context) -> float:
    return float(lib().mlbm_last_step_ms(ctx.handle))


def set_kernel_variant(ctx: Context, variant: int):
    _check(lib().mlbm_set_kernel_variant(ctx.handle, int(variant)))


def kernel_variant(ctx: Context) -> int:
    return int(lib().mlbm_kernel_variant(ctx.handle))


def autotune(ctx: Context, steps_per_variant: int = 20, flush_l2: bool = False) -> tuple:
    """Pick the fastest kernel variant on this context; returns (variant, ms/step)."""
    ms = ctypes.c_double()
    _check(lib().mlbm_autotune_ex(ctx.handle, int(steps_per_variant), int(bool(flush_l2)), ctypes.byref(ms)))
    return kernel_variant(ctx), ms.value


def autotune_times(ctx: Context) -> dict:
    """ms per step of every variant timed by the last autotune {variant: ms}."""
    ms = np.full(64, -1.0)
    n = lib().mlbm_autotune_times(ctx.handle, _ptr(ms), 64)
    return {v: float(ms[v]) for v in range(max(n, 0)) if ms[v] >= 0}


def batch_init(stencils: list, params: list) -> Context:
    n = len(stencils)
    arr = (_vp * n)(*[st.handle for st in stencils])
    P = (_Params * n)(*[_Params(int(p.model), float(p.tau), float(p.tau_minus), float(p.gx), float(p.gy))
                        for p in params])
    h = _vp()
    _check(lib().mlbm_batch_init(ctypes.byref(h), arr, P, n))
    total = sum(st.n for st in stencils)
    return Context(h, total, params[0].model, list(stencils))


def batch_size(ctx: Context) -> int:
    return int(lib().mlbm_batch_size(ctx.handle))


def batch_range(ctx: Context, sample: int) -> tuple:
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().mlbm_batch_range(ctx.handle, int(sample), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def batch_permeability(ctx: Context) -> dict:
    m = batch_size(ctx)
    out = {k: np.empty(m) for k in ("k", "u_superficial", "u_intrinsic", "tortuosity")}
    _check(lib().mlbm_batch_permeability(ctx.handle, *[_ptr(out[k]) for k in
                                                       ("k", "u_superficial", "u_intrinsic", "tortuosity")]))
    return out


def batch_run_to_steady(ctx: Context, tol: float, window: int, max_steps: int, raise_on_max: bool = True,
                        check: int | None = None):
    taken = np.empty(batch_size(ctx), np.int64)
    st = lib().mlbm_batch_run_to_steady_ex(ctx.handle, float(tol), int(window), int(check or window),
                                           int(max_steps), _ptr(taken))
    if not (st == 7 and not raise_on_max):
        _check(st)
    return taken


def batch_run_to_steady_mean(ctx: Context, threshold: float = 1e-2, dn: int = 20000, check: int = 1000, dt=None,
                             max_steps: int = 10_000_000, raise_on_max: bool = True):
    taken = np.empty(batch_size(ctx), np.int64)
    d = None if dt is None else _f64(np.broadcast_to(np.asarray(dt, np.float64), (batch_size(ctx),)))
    st = lib().mlbm_batch_run_to_steady_mean(ctx.handle, float(threshold), int(dn), int(check), _ptr(d),
                                             int(max_steps), _ptr(taken))
    if not (st == 7 and not raise_on_max):
        _check(st)
    return taken


def batch_drag_lift(ctx: Context, ref_length, u_ref) -> dict:
    m = batch_size(ctx)
    L = _f64(np.broadcast_to(np.asarray(ref_length, np.float64), (m,)))
    U = _f64(np.broadcast_to(np.asarray(u_ref, np.float64), (m,)))
    out = {k: np.empty(m) for k in ("fx", "fy", "cd", "cl")}
    _check(lib().mlbm_batch_drag_lift(ctx.handle, _ptr(L), _ptr(U), *[_ptr(out[k]) for k in ("fx", "fy", "cd", "cl")]))
    return out


def set_graphs(ctx: Context, enable: bool):
    _check(lib().mlbm_set_graphs(ctx.handle, int(bool(enable))))


def prepare_graphs(ctx: Context):
    _check(lib().mlbm_prepare_graphs(ctx.handle))


def reduce_scratch_doubles(n: int) -> int:
    return int(lib().mlbm_reduce_scratch_doubles(int(n)))


def reduce_fields_device(rho_ptr, ux_ptr, uy_ptr, area_ptr, mask_ptr, n, scratch_ptr, scratch_len, out_ptr,
                         stream_handle=None):
    """Device pointers (ints), e.g. torch tensor .data_ptr() values."""
    _check(lib().mlbm_reduce_fields_device(_vp(rho_ptr), _vp(ux_ptr), _vp(uy_ptr), _vp(area_ptr),
                                           _vp(mask_ptr) if mask_ptr else None, int(n), _vp(scratch_ptr),
                                           int(scratch_len), _vp(out_ptr),
                                           _vp(stream_handle) if stream_handle else None))


def reduce_fields_device_noalloc(rho_ptr, ux_ptr, uy_ptr, area_ptr, mask_ptr, n, out_ptr, stream_handle=None):
    """As reduce_fields_device, with the library's own static scratch (no allocation)."""
    _check(lib().mlbm_reduce_fields_device_noalloc(_vp(rho_ptr), _vp(ux_ptr), _vp(uy_ptr), _vp(area_ptr),
                                                   _vp(mask_ptr) if mask_ptr else None, int(n), _vp(out_ptr),
                                                   _vp(stream_handle) if stream_handle else None))


# ---------------------------------------------------------- partitioned step
def _bounds(bounds, n_parts):
    if bounds is None:
        return None
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    if b.shape != (n_parts + 1,):
        raise ValueError("bounds needs n_parts + 1 entries")
    return b


def partition_plan(st: Stencils, n_parts: int, bounds=None) -> dict:
    """Host-only description of a split into n_parts position ranges."""
    b = _bounds(bounds, n_parts)
    out = {k: np.empty(n_parts, np.int64) for k in ("first", "n_owned", "n_halo")}
    out["halo_from"] = np.empty((n_parts, n_parts), np.int64)
    _check(lib().mlbm_partition_plan(st.handle, int(n_parts), _ptr(b), *[_ptr(out[k]) for k in
                                                                        ("first", "n_owned", "n_halo", "halo_from")]))
    return out


def partition_nodes(st: Stencils, n_parts: int, part: int, bounds=None) -> tuple:
    """(owned caller ids in local order, halo caller ids in slot order) of one partition."""
    plan = partition_plan(st, n_parts, bounds)
    owned = np.empty(int(plan["n_owned"][part]), np.int64)
    halo = np.empty(int(plan["n_halo"][part]), np.int64)
    _check(lib().mlbm_partition_nodes(st.handle, int(n_parts), _ptr(_bounds(bounds, n_parts)), int(part),
                                      _ptr(owned), _ptr(halo)))
    return owned, halo


class Partitioned:
    """Handle of a partitioned node set (mlbm_part_*)."""

    def __init__(self, st: Stencils, params: Params, n_parts: int, bounds=None):
        P = _Params(int(params.model), float(params.tau), float(params.tau_minus), float(params.gx), float(params.gy))
        h = _vp()
        b = _bounds(bounds, n_parts)
        _check(lib().mlbm_part_init(ctypes.byref(h), st.handle, ctypes.byref(P), int(n_parts), _ptr(b)))
        self.handle, self.n, self.n_parts, self.model, self._st = h, st.n, int(n_parts), params.model, st

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.mlbm_part_destroy(self.handle)
            self.handle = None

    def info(self, q: int) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib().mlbm_part_info(self.handle, int(q), *[ctypes.byref(x) for x in v]))
        return dict(zip(("first", "n_owned", "n_halo", "halo_bytes_per_step"), (x.value for x in v)))

    def set_kernel_variant(self, variant: int):
        _check(lib().mlbm_part_set_kernel_variant(self.handle, int(variant)))

    def step(self, n: int = 1):
        _check(lib().mlbm_part_step(self.handle, int(n)))

    def set_fields(self, ru):
        a = _f64(ru)
        _check(lib().mlbm_part_set_fields(self.handle, _ptr(a)))

    def get_fields(self) -> np.ndarray:
        a = np.empty((self.n, 3))
        _check(lib().mlbm_part_get_fields(self.handle, _ptr(a)))
        return a

    def set_populations(self, f):
        a = _f64(f)
        _check(lib().mlbm_part_set_populations(self.handle, _ptr(a)))

    def get_populations(self) -> np.ndarray:
        a = np.empty((self.n, 9))
        _check(lib().mlbm_part_get_populations(self.handle, _ptr(a)))
        return a

    def permeability(self) -> dict:
        v = [ctypes.c_double() for _ in range(4)]
        _check(lib().mlbm_part_permeability(self.handle, *[ctypes.byref(x) for x in v]))
        return dict(zip(("k", "u_superficial", "u_intrinsic", "tortuosity"), (x.value for x in v)))


# ------------------------------------------------------- learned warm start
# Device arrays are passed as integer device addresses (e.g. a torch CUDA
# tensor's .data_ptr()); streams as cudaStream_t handles (None: default).
def _sp(stream_handle):
    return _vp(stream_handle) if stream_handle else None


class Mlp:
    """Handle of the library's warm-start network (16-64-64-64-n_out)."""

    def __init__(self, seed: int = 1, n_out: int = 2):
        h = _vp()
        _check(lib().mlbm_mlp_create(ctypes.byref(h), int(n_out), ctypes.c_uint64(int(seed))))
        self.handle = h
        self.n_out = int(n_out)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.mlbm_mlp_destroy(self.handle)
            self.handle = None

    def param_count(self) -> int:
        return int(lib().mlbm_mlp_param_count(self.n_out))

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.param_count():
            raise ValueError(f"expected {self.param_count()} parameters, got {a.size}")
        _check(lib().mlbm_mlp_set_params(self.handle, _ptr(a)))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.param_count(), np.float32)
        _check(lib().mlbm_mlp_get_params(self.handle, _ptr(a)))
        return a

    def forward(self, X_ptr, n, Y_ptr, stream_handle=None):
        _check(lib().mlbm_mlp_forward_device(self.handle, _vp(X_ptr), int(n), _vp(Y_ptr), _sp(stream_handle)))

    def gradients(self, X_ptr, T_ptr, n, grads_ptr=None, stream_handle=None) -> float:
        loss = ctypes.c_double()
        _check(lib().mlbm_mlp_gradients_device(self.handle, _vp(X_ptr), _vp(T_ptr), int(n),
                                               _vp(grads_ptr) if grads_ptr else None, ctypes.byref(loss),
                                               _sp(stream_handle)))
        return loss.value

    def train(self, X_ptr, T_ptr, n, batch, steps, lr, seed, stream_handle=None) -> float:
        loss = ctypes.c_double()
        _check(lib().mlbm_mlp_train_device(self.handle, _vp(X_ptr), _vp(T_ptr), int(n), int(batch), int(steps),
                                           ctypes.c_float(lr), ctypes.c_uint64(int(seed)),
                                           ctypes.byref(loss) if steps > 0 else None, _sp(stream_handle)))
        return loss.value


def features_device(xy, box, sides, disks, L, X_ptr):
    """Geometry features [n][16] (FP32) of nodes xy into device memory X_ptr."""
    xy = _f64(xy)
    dk = _f64(np.zeros((0, 3)) if disks is None else np.asarray(disks).reshape(-1, 3))
    nodes = _Nodes(xy.shape[0], _ptr(xy), None, None, None)
    geo = _Geometry(float(box[0]), float(box[1]), float(box[2]), float(box[3]), (_i32 * 4)(*[int(v) for v in sides]),
                    len(dk), _ptr(dk) if len(dk) else None)
    _check(lib().mlbm_features_device(ctypes.byref(nodes), ctypes.byref(geo), float(L), _vp(X_ptr)))


def features_for(w, L, X_ptr):
    """features_device for an inputs.Workload."""
    features_device(w.xy, w.box, w.sides, w.disks, L, X_ptr)


def warm_start(ctx: Context, mlp: Mlp, X_ptr, scale_u, scale_rho=None) -> int:
    """Start ctx from the network's prediction (u = scale_u * Y[:, :2] and,
    with 3 outputs, rho = 1 + scale_rho * Y[:, 2] minus its sample mean);
    returns how many samples fell back to rest."""
    su = _f64(np.atleast_1d(np.asarray(scale_u, np.float64)))
    sr = None if scale_rho is None else _f64(np.atleast_1d(np.asarray(scale_rho, np.float64)))
    cold = ctypes.c_int()
    _check(lib().mlbm_warm_start(ctx.handle, mlp.handle, _vp(X_ptr), _ptr(su), _ptr(sr), ctypes.byref(cold)))
    return cold.value


# ------------------------------------------------------ lattice LBM (comparison)
class Lattice:
    """Regular-grid LBM of the library (the paper's comparison method)."""

    def __init__(self, cell, params: Params, periodic=(True, True), eq_values=None):
        cell = np.ascontiguousarray(cell, dtype=np.uint8)
        self.ny, self.nx = cell.shape
        eqv = None if eq_values is None else _f64(np.asarray(eq_values).reshape(-1, 3))
        p = _Params(int(params.model), float(params.tau), float(params.tau_minus), float(params.gx), float(params.gy))
        h = _vp()
        _check(lib().mlbm_lattice_init(ctypes.byref(h), self.nx, self.ny, int(bool(periodic[0])),
                                       int(bool(periodic[1])), _ptr(cell), _ptr(eqv), ctypes.byref(p)))
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.mlbm_lattice_destroy(self.handle)
            self.handle = None

    def step(self, n: int = 1):
        _check(lib().mlbm_lattice_step(self.handle, int(n)))

    def sync(self):
        _check(lib().mlbm_lattice_sync(self.handle))

    def time_steps(self, n: int) -> float:
        """Milliseconds for n steps (CUDA events on the lattice's stream)."""
        ms = ctypes.c_double()
        _check(lib().mlbm_lattice_time_steps(self.handle, int(n), ctypes.byref(ms)))
        return ms.value

    def set_populations(self, f):
        a = _f64(np.asarray(f).reshape(-1, 9))
        _check(lib().mlbm_lattice_set_populations(self.handle, _ptr(a)))

    def get_populations(self) -> np.ndarray:
        a = np.empty((self.nx * self.ny, 9))
        _check(lib().mlbm_lattice_get_populations(self.handle, _ptr(a)))
        return a

    def force(self) -> tuple:
        fx, fy = ctypes.c_double(), ctypes.c_double()
        _check(lib().mlbm_lattice_force(self.handle, ctypes.byref(fx), ctypes.byref(fy)))
        return fx.value, fy.value
