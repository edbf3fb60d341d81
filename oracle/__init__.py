"""FP64 CPU oracle of the meshless LBM step -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA path:
the heavy loops are in `mlbm_oracle.c` (plain C, double precision), the glue
and the observables here are plain numpy.  See the C file's header for the
equation-by-equation map to the paper (arXiv 2312.14789).

Main entry points
  Operator(workload, K, s, ...)      stencils, bounce-back links and the
                                     per-direction weights w_i^k of Eq. (12)
  bgk_step(op, f, tau, g)            one MLBM step (BGK / TRT), state f[n][9]
  mlbm1_step(op, ru, g)              one MLBM1 step (tau = 1), state (rho,u,v)[n]
  equilibrium(rho, ux, uy)           Eq. (7) for all nodes -> [n][9]
  macroscopics(f, g)                 rho, u of a post-collision state
  force_bgk / force_mlbm1            momentum exchange on the solids
  mean_velocity, permeability, tortuosity, strouhal, memory model
  steady_mean_step, paper_time_step   the steady criterion of Sec. 3.2
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

c_double_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the C oracle in-tree (gcc, no fused multiply-add contraction)."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liboracle.so")
    src = os.path.join(_HERE, "mlbm_oracle.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            L.oracle_feq.restype = dbl
            L.oracle_feq.argtypes = [i32, dbl, dbl, dbl]
            L.oracle_source.restype = dbl
            L.oracle_source.argtypes = [i32, dbl, dbl, dbl, dbl, dbl]
            L.oracle_omega.restype = dbl
            L.oracle_omega.argtypes = [i32]
            for nm in ("oracle_ex", "oracle_ey", "oracle_opp"):
                getattr(L, nm).restype = i32
                getattr(L, nm).argtypes = [i32]
            L.oracle_moments.restype = None
            L.oracle_moments.argtypes = [vp, dbl, dbl, vp, vp, vp]
            L.oracle_collide.restype = None
            L.oracle_collide.argtypes = [vp, dbl, dbl, dbl, dbl, vp]
            L.oracle_knn.restype = i32
            L.oracle_knn.argtypes = [vp, i64, vp, i32, i32, i32, vp, i64, vp, vp]
            L.oracle_wls_matrix.restype = i32
            L.oracle_wls_matrix.argtypes = [vp, i32, dbl, dbl, vp]
            L.oracle_lagrange_detect.restype = i32
            L.oracle_lagrange_detect.argtypes = [vp, i32, dbl, vp, vp, vp, vp, vp, vp]
            L.oracle_bc_links.restype = i32
            L.oracle_bc_links.argtypes = [dbl, dbl, dbl, vp, vp, vp, i32, vp, vp]
            L.oracle_assemble.restype = None
            L.oracle_assemble.argtypes = [i64, vp, i32, vp, vp, vp, vp, dbl, dbl, i32, i32, i32, dbl, vp, vp,
                                          vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.oracle_rbf_weights.restype = i32
            L.oracle_rbf_weights.argtypes = [vp, i32, dbl, dbl, vp]
            L.oracle_rbf_lagrangian.restype = None
            L.oracle_rbf_lagrangian.argtypes = [i64, vp, vp, i64, vp, i32, i32, dbl, i32, i32, vp, vp, vp, vp, i32,
                                                vp, i32, vp, vp, vp]
            L.oracle_mlbm_step.restype = None
            L.oracle_mlbm_step.argtypes = [i64, vp, i64, vp, i32, vp, vp, vp, vp, vp, dbl, dbl, dbl, dbl, vp]
            L.oracle_mlbm1_step.restype = None
            L.oracle_mlbm1_step.argtypes = [i64, vp, i64, vp, i32, vp, vp, vp, vp, vp, dbl, dbl, vp]
            L.oracle_force_bgk.restype = None
            L.oracle_force_bgk.argtypes = [i64, vp, i32, vp, vp, vp, vp, vp, vp, dbl, vp, vp]
            L.oracle_force_mlbm1.restype = None
            L.oracle_force_mlbm1.argtypes = [i64, vp, i32, vp, vp, vp, vp, vp, vp, dbl, dbl, dbl, vp, vp]
            _LIB = L
    return _LIB


def _p(a):
    return a.ctypes.data if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# D2Q9 constants read from the C oracle (one definition only)
def lattice_constants():
    L = lib()
    E = np.array([[L.oracle_ex(k), L.oracle_ey(k)] for k in range(9)], dtype=np.int64)
    W = np.array([L.oracle_omega(k) for k in range(9)])
    OPP = np.array([L.oracle_opp(k) for k in range(9)], dtype=np.int64)
    return E, W, OPP


# --------------------------------------------------------------------------
# point-wise closed forms
# --------------------------------------------------------------------------
def feq(k: int, rho: float, ux: float, uy: float) -> float:
    """Eq. (7) for one direction."""
    return lib().oracle_feq(int(k), float(rho), float(ux), float(uy))


def source(k: int, rho: float, ux: float, uy: float, gx: float, gy: float) -> float:
    return lib().oracle_source(int(k), float(rho), float(ux), float(uy), float(gx), float(gy))


def equilibrium(rho, ux, uy) -> np.ndarray:
    """Eq. (7) at every node: [n][9] (vectorised restatement via the C scalar)."""
    rho = np.atleast_1d(np.asarray(rho, np.float64))
    ux = np.broadcast_to(np.asarray(ux, np.float64), rho.shape)
    uy = np.broadcast_to(np.asarray(uy, np.float64), rho.shape)
    out = np.empty((rho.size, 9))
    f = lib().oracle_feq
    for i in range(rho.size):
        r, a, b = float(rho.flat[i]), float(ux.flat[i]), float(uy.flat[i])
        for k in range(9):
            out[i, k] = f(k, r, a, b)
    return out


def collide(f9, tau_p, tau_m, gx, gy) -> np.ndarray:
    f9 = _c(f9, np.float64)
    out = np.empty(9)
    lib().oracle_collide(_p(f9), float(tau_p), float(tau_m), float(gx), float(gy), _p(out))
    return out


def macroscopics(f, g=(0.0, 0.0)):
    """rho and u of a post-collision state f[n][9]: rho = sum f (collision keeps
    it), rho u = sum f e - rho g / 2 (collision added the full force F, the
    state's velocity is the one used in that collision)."""
    E, _, _ = lattice_constants()
    f = np.asarray(f, np.float64)
    rho = f.sum(axis=1)
    ux = (f @ E[:, 0]) / rho - 0.5 * g[0]
    uy = (f @ E[:, 1]) / rho - 0.5 * g[1]
    return rho, ux, uy


# --------------------------------------------------------------------------
# stencils and the streaming operator
# --------------------------------------------------------------------------
def knn(xy, box, periodic, K, targets=None):
    xy = _c(xy, np.float64)
    box = _c(box, np.float64)
    tg = None if targets is None else _c(targets, np.int64)
    nt = len(xy) if tg is None else len(tg)
    idx = np.empty((nt, K), np.int64)
    off = np.empty((nt, K, 2), np.float64)
    st = lib().oracle_knn(_p(xy), len(xy), _p(box), int(periodic[0]), int(periodic[1]), int(K),
                          _p(tg), nt, _p(idx), _p(off))
    if st:
        raise ValueError("oracle_knn: K larger than the node count")
    return idx, off


def wls_matrix(off, s, sigma_factor):
    """Returns (status, M[6][K]) for one stencil's offsets off[K][2]."""
    off = _c(off, np.float64)
    K = off.shape[0]
    M = np.empty((6, K))
    st = lib().oracle_wls_matrix(_p(off), K, float(s), float(sigma_factor), _p(M))
    return st, M


def rbf_weights(off, d):
    """RBF-FD weights (cubic polyharmonic spline with quadratic augmentation)
    of the stencil offsets off[K][2] for the value at the point d = (dx, dy)."""
    off = _c(off, np.float64)
    K = off.shape[0]
    w = np.empty(K)
    st = lib().oracle_rbf_weights(_p(off), K, float(d[0]), float(d[1]), _p(w))
    if st:
        raise ValueError(f"RBF-FD system singular (status {st})")
    return w


def lagrange_detect(off, s=1.0, link=None, q=None, bb_mode=1, tol=1e-9):
    """Returns (found, slot[9], h, centre direction m) for one stencil."""
    off = _c(off, np.float64)
    E, _, _ = lattice_constants()
    link = np.zeros(9, np.int32) if link is None else np.asarray(link)
    q = np.zeros(9) if q is None else np.asarray(q)
    dx = np.zeros(9); dy = np.zeros(9); use = np.zeros(9, np.int32)
    for k in range(1, 9):
        if link[k]:
            if bb_mode == 0:
                continue
            t = 1.0 - 2.0 * q[k]
            dx[k], dy[k] = t * s * E[k]
        else:
            dx[k], dy[k] = -s * E[k]
        use[k] = 1
    slot = np.empty(9, np.int32)
    h = np.zeros(1)
    c = np.zeros(1, np.int32)
    ok = lib().oracle_lagrange_detect(_p(off), off.shape[0], float(tol), _p(dx), _p(dy), _p(use),
                                      _p(slot), _p(h), _p(c))
    return bool(ok), slot, float(h[0]), int(c[0])


def bc_links(x, y, s, box, side, disks):
    box = _c(box, np.float64)
    side = _c(side, np.int32)
    disks = _c(np.asarray(disks).reshape(-1, 3), np.float64)
    link = np.zeros(9, np.int32)
    q = np.zeros(9)
    st = lib().oracle_bc_links(float(x), float(y), float(s), _p(box), _p(side),
                               _p(disks) if len(disks) else None, len(disks), _p(link), _p(q))
    return st, link, q


class Operator:
    """Stencils + bounce-back links + per-direction weights (Eq. (12)) for a
    workload, either for all nodes or for a subset `targets`."""

    def __init__(self, w, K, s, sigma_factor=0.7071067811865476, bb_mode=1, use_lagrange=True,
                 lag_tol=1e-9, targets=None, interp="wls", n_l=25, k_max=None):
        """interp: "wls" (least squares over the node's K-stencil), "rbf"
        (RBF-FD over the node's K-stencil) or "rbf_points" (RBF-FD with the
        n_l nearest nodes of every departure point, Sec. 2.2; the stencil
        becomes the union of those, k_max slots)."""
        self.w = w
        self.K, self.s, self.bb_mode = int(K), float(s), int(bb_mode)
        self.sigma_factor = float(sigma_factor)
        self.targets = None if targets is None else _c(targets, np.int64)
        self.nt = w.n if self.targets is None else len(self.targets)
        periodic = (w.sides[0] == 0, w.sides[2] == 0)
        self.idx, self.off = knn(w.xy, w.box, periodic, K, self.targets)
        nt, K = self.nt, self.K
        self.kind = np.zeros(nt, np.int32)
        self.M = np.zeros((nt, 6, K))
        self.lag_slot = np.zeros((nt, 9), np.int32)
        self.lag_h = np.zeros(nt)
        self.lag_center = np.zeros(nt, np.int32)
        self.link = np.zeros((nt, 9), np.int32)
        self.q = np.zeros((nt, 9))
        self.W = np.zeros((nt, 9, K))
        self.src = np.zeros((nt, 9), np.int32)
        self.status = np.zeros(nt, np.int32)
        box = _c(w.box, np.float64)
        side = _c(w.sides, np.int32)
        disks = _c(np.asarray(w.disks).reshape(-1, 3), np.float64)
        cls = _c(w.node_class, np.uint8)
        xy = _c(w.xy, np.float64)
        lib().oracle_assemble(nt, _p(self.targets), K, _p(self.idx), _p(self.off), _p(xy), _p(cls),
                              self.s, self.sigma_factor, self.bb_mode, int(bool(use_lagrange)),
                              {"wls": 0, "rbf": 1, "rbf_points": 0}[interp],
                              float(lag_tol), _p(box), _p(side), _p(disks) if len(disks) else None,
                              len(disks), _p(self.kind), _p(self.M), _p(self.lag_slot), _p(self.lag_h),
                              _p(self.lag_center), _p(self.link), _p(self.q), _p(self.W), _p(self.src),
                              _p(self.status))
        self.eq_val = _c(w.eq_values, np.float64)
        self.node_class = cls
        self.area = _c(w.area, np.float64)
        self.idx_own = self.idx
        if interp == "rbf_points":
            kmax = int(k_max or 4 * K)
            idx2 = np.empty((nt, kmax), np.int64)
            W2 = np.empty((nt, 9, kmax))
            lib().oracle_rbf_lagrangian(nt, _p(self.targets), _p(xy), w.n, _p(box), int(periodic[0]),
                                        int(periodic[1]), self.s, int(n_l), K, _p(self.idx),
                                        _p(_c(self.kind, np.int32)), _p(_c(self.link, np.int32)), _p(self.q),
                                        self.bb_mode, _p(self.W), kmax, _p(idx2), _p(W2), _p(self.status))
            self.idx, self.W, self.K = idx2, W2, kmax

    @property
    def target_ids(self):
        return np.arange(self.w.n) if self.targets is None else self.targets

    def check(self):
        bad = np.nonzero(self.status)[0]
        if len(bad):
            raise ValueError(f"oracle stencil assembly failed at {len(bad)} nodes, "
                             f"first node {self.target_ids[bad[0]]} status {self.status[bad[0]]}")
        return self


def bgk_step(op: Operator, f, tau, g=(0.0, 0.0), tau_minus=None) -> np.ndarray:
    """One MLBM step; f[n][9] post-collision at t -> targets' post-collision
    populations at t+1 ([nt][9])."""
    f = _c(f, np.float64)
    out = np.empty((op.nt, 9))
    tm = tau if tau_minus is None else tau_minus
    lib().oracle_mlbm_step(len(f), _p(f), op.nt, _p(op.targets), op.K, _p(op.idx), _p(op.W), _p(op.src),
                           _p(op.node_class), _p(op.eq_val), float(tau), float(tm), float(g[0]),
                           float(g[1]), _p(out))
    return out


def mlbm1_step(op: Operator, ru, g=(0.0, 0.0)) -> np.ndarray:
    """One MLBM1 step; ru[n][3] = (rho, ux, uy) at t -> targets' values at t+1."""
    ru = _c(ru, np.float64)
    out = np.empty((op.nt, 3))
    lib().oracle_mlbm1_step(len(ru), _p(ru), op.nt, _p(op.targets), op.K, _p(op.idx), _p(op.W),
                            _p(op.src), _p(op.node_class), _p(op.eq_val), float(g[0]), float(g[1]),
                            _p(out))
    return out


def run_bgk(op: Operator, f0, tau, g, steps, tau_minus=None):
    assert op.targets is None
    f = np.array(f0, np.float64)
    for _ in range(steps):
        f = bgk_step(op, f, tau, g, tau_minus)
    return f


def run_mlbm1(op: Operator, ru0, g, steps):
    assert op.targets is None
    ru = np.array(ru0, np.float64)
    for _ in range(steps):
        ru = mlbm1_step(op, ru, g)
    return ru


def force_bgk(op: Operator, f):
    f = _c(f, np.float64)
    fx, fy = np.zeros(1), np.zeros(1)
    lib().oracle_force_bgk(op.nt, _p(op.targets), op.K, _p(op.idx), _p(op.W), _p(op.src),
                           _p(_c(op.link, np.int32)), _p(f), _p(op.area), op.s, _p(fx), _p(fy))
    return float(fx[0]), float(fy[0])


def force_mlbm1(op: Operator, ru, g=(0.0, 0.0)):
    ru = _c(ru, np.float64)
    fx, fy = np.zeros(1), np.zeros(1)
    lib().oracle_force_mlbm1(op.nt, _p(op.targets), op.K, _p(op.idx), _p(op.W), _p(op.src),
                             _p(_c(op.link, np.int32)), _p(ru), _p(op.area), op.s, float(g[0]),
                             float(g[1]), _p(fx), _p(fy))
    return float(fx[0]), float(fy[0])


def wall_stress_force(op: Operator, ru, tau, nodes, normals, ds):
    """Force of the fluid on the walls by integrating the fluid stress along
    them (a reading: the paper is silent on how it evaluates the force of
    Sec. 3.1).  At each wall node i, with outward-from-solid unit normal n and
    wall length ds (node-spacing units), the traction is
        sigma n,  sigma = -(rho - 1)/3 I + rho nu (grad u + grad u^T),
    nu = (tau - 1/2)/3 (Eq. (6)), in lattice units of the streaming distance s;
    grad u comes from the node's own least-squares fit (rows 1 and 2 of its
    matrix M, which already carry the factor s of the lattice unit), and
    F = sum_i sigma_i n_i ds_i / s.  ru[n][3] = (rho, ux, uy) in the caller's
    order; the nodes must be least-squares nodes of `op`."""
    assert op.targets is None
    ru = np.asarray(ru, np.float64)
    nu = (float(tau) - 0.5) / 3.0
    F = np.zeros(2)
    for i, n, l in zip(np.asarray(nodes, np.int64), np.asarray(normals, np.float64), np.asarray(ds, np.float64)):
        if op.kind[i] != 0:
            raise ValueError(f"node {i} is not a least-squares node")
        j = op.idx_own[i]
        du = ru[j, 1] - ru[i, 1]
        dv = ru[j, 2] - ru[i, 2]
        ux_x, ux_y = op.M[i, 1] @ du, op.M[i, 2] @ du
        uy_x, uy_y = op.M[i, 1] @ dv, op.M[i, 2] @ dv
        rho = ru[i, 0]
        p = (rho - 1.0) / 3.0
        sxx = -p + 2.0 * rho * nu * ux_x
        syy = -p + 2.0 * rho * nu * uy_y
        sxy = rho * nu * (ux_y + uy_x)
        F += np.array([sxx * n[0] + sxy * n[1], sxy * n[0] + syy * n[1]]) * l / op.s
    return float(F[0]), float(F[1])


# --------------------------------------------------------------------------
# observables (Sec. 3.2, Eq. (23) and (25); Sec. 3.1 Strouhal number)
# --------------------------------------------------------------------------
def mean_velocity(ux, area, fluid_mask=None, total_area=None):
    """Area-weighted mean of u_x over the fluid nodes.  Returns (superficial,
    intrinsic): superficial divides by the whole box area (Darcy velocity),
    intrinsic by the fluid area.  Reading of Eq. (23), whose printed form is
    garbled: (1/phi) times the integral over the domain of u."""
    ux = np.asarray(ux, np.float64)
    area = np.asarray(area, np.float64)
    m = np.ones_like(ux, bool) if fluid_mask is None else fluid_mask
    s = float(np.sum(ux[m] * area[m]))
    fa = float(np.sum(area[m]))
    ta = fa if total_area is None else float(total_area)
    return s / ta, s / fa


def tortuosity(ux, uy, area):
    """Eq. (25): T_V = <|u|> / <u_x>, both area-weighted over the fluid."""
    ux, uy, area = (np.asarray(a, np.float64) for a in (ux, uy, area))
    return float(np.sum(np.hypot(ux, uy) * area) / np.sum(ux * area))


def permeability(u_superficial, tau, g):
    """Darcy: k = nu U_s / g with nu = c_s^2 (tau - 1/2) (Eq. (6))."""
    nu = (tau - 0.5) / 3.0
    return nu * u_superficial / g


def strouhal(cl, dt_per_sample, diameter_lb, u0, min_periods=2):
    """St = f d / U0 (Sec. 3.1) with f from the mean spacing of upward zero
    crossings of C_L - mean(C_L), linearly interpolated between samples."""
    c = np.asarray(cl, np.float64) - np.mean(cl)
    i = np.nonzero((c[:-1] < 0) & (c[1:] >= 0))[0]
    if len(i) < min_periods + 1:
        return float("nan")
    tz = (i + (-c[i]) / (c[i + 1] - c[i])) * dt_per_sample
    period = float(np.mean(np.diff(tz)))
    return (1.0 / period) * diameter_lb / u0


def paper_time_step(tau, s, box_side):
    """Physical time of one step in the units of Sec. 3.2 (sample side length
    1, kinematic viscosity 1): nu_phys = nu_lb dx^2 / dt with the streaming
    distance dx = s / box_side in those units and nu_lb = (tau - 1/2)/3
    (Eq. (6)), hence dt = nu_lb (s / box_side)^2."""
    return (tau - 0.5) / 3.0 * (s / box_side) ** 2


def steady_mean_step(mean_u, check, dn, dt, threshold):
    """The steady-state criterion of Sec. 3.2 applied to a record of the mean
    x-velocity: mean_u[j] is <u> at step j*check (j = 0, 1, ...).  At every
    recorded step t >= dn the relative rate of change over the previous dn
    steps is
        Delta u = (<u>(t) - <u>(t - dn)) / (<u>(t - dn) dt dn),
    the earlier mean <u>^n in the denominator as the paper prints it, taken in
    absolute value (reading: a mean that approaches its limit from above must
    not count as steady at once).  Returns the first such t with
    Delta u < threshold, or -1.  A zero earlier mean is never steady."""
    if dn % check:
        raise ValueError("dn must be a multiple of check")
    lag = dn // check
    for j in range(lag, len(mean_u)):
        then, now = float(mean_u[j - lag]), float(mean_u[j])
        if then == 0.0:
            continue
        rate = abs(now - then) / (abs(then) * dt * dn)
        if rate < threshold:
            return j * check
    return -1


def relative_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --------------------------------------------------------------------------
# memory model (Sec. 3.2, Eq. (26)-(28) and the table that follows them)
# --------------------------------------------------------------------------
def memory_lbm1(n_nodes, n_fields=3, c=8):
    """Eq. (26): M_LBM1 = N 2 N_f c (two time levels of N_f fields)."""
    return n_nodes * 2 * n_fields * c


def memory_mlbm1(n_rbffd, n_lag, n_fields=3, q=9, c=8, n_rbf=25, n_lagrange=9):
    """Eq. (27): [2 N_f N + 3/2 (25 N_RBF + 9 N_Lag)(q - 1)] c."""
    return (2 * n_fields * (n_rbffd + n_lag) + 1.5 * (n_rbf * n_rbffd + n_lagrange * n_lag) * (q - 1)) * c


def memory_ratio(n_rbffd, n_lag, n_lbm1, **kw):
    """Eq. (28): r_M = M_MLBM1 / M_LBM1."""
    return memory_mlbm1(n_rbffd, n_lag, **kw) / memory_lbm1(n_lbm1)
