"""Seeded synthetic workloads for the meshless LBM step.

Only geometry lives here: node positions, node classes, solid disks, the box
and its side types, prescribed boundary values (density and velocity for
equilibrium-overwrite nodes), node areas and plain random arrays.  No lattice
Boltzmann arithmetic (equilibria, weights, interpolation, collision) is
performed here, so both the CUDA path and the FP64 oracle can read the same
inputs without sharing any part of the method.

Workload shapes follow the paper's test cases:
  * periodic Poiseuille channel on a jittered grid (plain MLBM, Sec. 2.2);
  * cylinder in a channel with a refined scattered node set (Sec. 3.1);
  * porous box of random non-overlapping disks, periodic in x with walls at
    the top and bottom and wall nodes placed on the solid surfaces (Sec. 3.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

# node classes (also the values the C-ABI and the oracle accept)
FLUID, WALL, EQ = 0, 1, 2
# side types
PERIODIC, SOLID, OPEN = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


def build_sampler(force: bool = False) -> str:
    """Compile the Poisson-disk sampler (plain C) in-tree; return the .so path."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libpoisson.so")
    src = os.path.join(_HERE, "poisson.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build_sampler())
            lib.pd_sample.restype = ctypes.c_int64
            lib.pd_sample.argtypes = [
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
            _LIB = lib
    return _LIB


@dataclass
class Workload:
    """A node set plus everything the boundary treatment needs to know."""
    name: str
    xy: np.ndarray                 # (n, 2) float64 node positions
    node_class: np.ndarray         # (n,) uint8: FLUID / WALL / EQ
    box: tuple                     # (x0, y0, x1, y1)
    sides: tuple                   # (left, right, bottom, top): PERIODIC / SOLID / OPEN
    disks: np.ndarray              # (m, 3) float64: cx, cy, r (solid)
    eq_values: np.ndarray          # (n, 3) float64: rho, ux, uy for EQ nodes, zero elsewhere
    area: np.ndarray               # (n,) float64 node areas (same length unit as xy)
    h_ref: float = 1.0             # reference node spacing
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])

    def fluid_area(self) -> float:
        x0, y0, x1, y1 = self.box
        return float((x1 - x0) * (y1 - y0) - np.sum(np.pi * self.disks[:, 2] ** 2)) if len(self.disks) \
            else float((x1 - x0) * (y1 - y0))


def _sample(box, periodic, rgrid, disks, clear_frac, fixed, seed, max_out, k_tries=30):
    x0, y0, x1, y1 = box
    rgrid = np.ascontiguousarray(rgrid, dtype=np.float64)
    disks = np.ascontiguousarray(disks, dtype=np.float64).reshape(-1, 3)
    fixed = np.ascontiguousarray(fixed, dtype=np.float64).reshape(-1, 2)
    out = np.empty((max_out, 2), dtype=np.float64)
    n = _lib().pd_sample(x0, y0, x1, y1, int(periodic[0]), int(periodic[1]),
                         rgrid.ctypes.data, rgrid.shape[1], rgrid.shape[0],
                         disks.ctypes.data if len(disks) else None, len(disks), float(clear_frac),
                         fixed.ctypes.data if len(fixed) else None, len(fixed),
                         np.uint64(seed), k_tries, out.ctypes.data, max_out)
    if n < 0:
        raise RuntimeError("Poisson-disk sampler ran out of room; raise max_out")
    return out[:n].copy()


def fluid_voronoi_areas(xy, box, periodic, disks, spacing, fine=None):
    """Area of the part of each node's Voronoi cell that lies in the fluid:
    the box minus the solid disks is rastered on a regular grid (spacing
    `spacing`; `fine` = (x0, y0, x1, y1, spacing) rasters that window more
    finely), every fluid raster point goes to its nearest node (minimum image
    across periodic sides) and carries its raster cell's area."""
    from scipy.spatial import cKDTree
    x0, y0, x1, y1 = box
    lx, ly = x1 - x0, y1 - y0
    pts = np.asarray(xy, np.float64)
    shift = np.array([x0, y0])
    boxsize = None
    if periodic[0] or periodic[1]:
        boxsize = np.array([lx if periodic[0] else 1e30, ly if periodic[1] else 1e30])
        pts = np.mod(pts - shift, [lx if periodic[0] else 1e30, ly if periodic[1] else 1e30])
    else:
        pts = pts - shift
    tree = cKDTree(pts, boxsize=boxsize)
    area = np.zeros(len(pts))
    windows = []
    if fine is not None:
        windows.append(fine)
    windows.append((x0, y0, x1, y1, spacing))
    for wi, (wx0, wy0, wx1, wy1, d) in enumerate(windows):
        nx_, ny_ = max(1, int(np.ceil((wx1 - wx0) / d))), max(1, int(np.ceil((wy1 - wy0) / d)))
        dx, dy = (wx1 - wx0) / nx_, (wy1 - wy0) / ny_
        xs = wx0 + (np.arange(nx_) + 0.5) * dx
        for row in range(0, ny_, 256):
            ys = wy0 + (np.arange(row, min(ny_, row + 256)) + 0.5) * dy
            X, Y = np.meshgrid(xs, ys)
            m = np.ones(X.shape, bool)
            for cx, cy, r in np.asarray(disks).reshape(-1, 3):
                ddx = X - cx
                if periodic[0]:
                    ddx -= lx * np.rint(ddx / lx)
                m &= ddx * ddx + (Y - cy) ** 2 >= r * r
            if wi > 0 and fine is not None:
                fx0, fy0, fx1, fy1, _ = fine
                m &= ~((X >= fx0) & (X < fx1) & (Y >= fy0) & (Y < fy1))
            q = np.stack([X[m] - x0, Y[m] - y0], 1)
            if boxsize is not None:
                q = np.mod(q, [lx if periodic[0] else 1e30, ly if periodic[1] else 1e30])
            _, j = tree.query(q, workers=-1)
            area += np.bincount(j, minlength=len(pts)) * (dx * dy)
    return area


# --------------------------------------------------------------------------
# Plain grids
# --------------------------------------------------------------------------
def lattice(nx: int, ny: int, h: float = 1.0, walls_y: bool = False, name: str = "lattice") -> Workload:
    """Regular square lattice.  Doubly periodic, or periodic in x with wall
    nodes on rows y=0 and y=(ny-1)h when walls_y is set."""
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    xy = np.stack([ix.ravel() * h, iy.ravel() * h], axis=1).astype(np.float64)
    cls = np.zeros(len(xy), np.uint8)
    if walls_y:
        box = (0.0, 0.0, nx * h, (ny - 1) * h)
        sides = (PERIODIC, PERIODIC, SOLID, SOLID)
        cls[(iy.ravel() == 0) | (iy.ravel() == ny - 1)] = WALL
        area = np.full(len(xy), h * h)
        area[cls == WALL] = 0.5 * h * h
    else:
        box = (0.0, 0.0, nx * h, ny * h)
        sides = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
        area = np.full(len(xy), h * h)
    return Workload(name, xy, cls, box, sides, np.zeros((0, 3)), np.zeros((len(xy), 3)), area, h,
                    {"nx": nx, "ny": ny})


def lattice_channel(nx: int, ny: int, y_offset: float = 0.5, h: float = 1.0) -> Workload:
    """Regular lattice, periodic in x, rows at y = (j + y_offset) h for
    j = 0..ny-1, solid walls at y = 0 and y = (ny - 1 + 2 y_offset) h, so both
    walls sit y_offset*h from the outer rows (0.5: half-way between nodes;
    0: wall nodes on the walls)."""
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    xy = np.stack([ix.ravel() * h, (iy.ravel() + y_offset) * h], axis=1).astype(np.float64)
    cls = np.zeros(len(xy), np.uint8)
    if y_offset == 0.0:
        cls[(iy.ravel() == 0) | (iy.ravel() == ny - 1)] = WALL
    H = (ny - 1 + 2 * y_offset) * h
    return Workload(f"lattice_channel_{nx}x{ny}_o{y_offset:g}", xy, cls, (0.0, 0.0, nx * h, H),
                    (PERIODIC, PERIODIC, SOLID, SOLID), np.zeros((0, 3)), np.zeros((len(xy), 3)),
                    np.full(len(xy), h * h), h, {"nx": nx, "ny": ny, "H": H, "y_offset": y_offset})


def jittered_periodic(nx: int, ny: int, jitter: float = 0.2, seed: int = 0, h: float = 1.0) -> Workload:
    """Doubly periodic jittered grid: node (i, j) at h*(i + U(-j, j), j + U(-j, j))."""
    rng = np.random.default_rng(seed)
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    x = (ix.ravel() + rng.uniform(-jitter, jitter, ix.size)) * h
    y = (iy.ravel() + rng.uniform(-jitter, jitter, iy.size)) * h
    lx, ly = nx * h, ny * h
    xy = np.stack([np.mod(x, lx), np.mod(y, ly)], axis=1)
    cls = np.zeros(len(xy), np.uint8)
    return Workload(f"jittered_periodic_{nx}x{ny}_s{seed}", xy, cls, (0.0, 0.0, lx, ly),
                    (PERIODIC,) * 4, np.zeros((0, 3)), np.zeros((len(xy), 3)),
                    np.full(len(xy), h * h), h, {"nx": nx, "ny": ny, "jitter": jitter, "seed": seed})


def poiseuille_channel(nx: int = 40, ny: int = 50, jitter: float = 0.2, seed: int = 1,
                       h: float = 1.0) -> Workload:
    """Periodic-in-x channel with wall nodes on y=0 and y=(ny-1)h.

    Interior nodes are jittered by U(-jitter, jitter)h in both axes; the two
    wall rows only along x, so they stay on the walls.  40x50 with seed 1 is
    the plain-MLBM Poiseuille case (2000 nodes)."""
    rng = np.random.default_rng(seed)
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ix, iy = ix.ravel(), iy.ravel()
    jx = rng.uniform(-jitter, jitter, ix.size)
    jy = rng.uniform(-jitter, jitter, iy.size)
    wall = (iy == 0) | (iy == ny - 1)
    jy[wall] = 0.0
    lx = nx * h
    x = np.mod((ix + jx) * h, lx)
    y = (iy + jy) * h
    xy = np.stack([x, y], axis=1)
    cls = np.where(wall, WALL, FLUID).astype(np.uint8)
    area = np.full(len(xy), h * h)
    area[wall] = 0.5 * h * h
    return Workload(f"poiseuille_{nx}x{ny}_s{seed}", xy, cls, (0.0, 0.0, lx, (ny - 1) * h),
                    (PERIODIC, PERIODIC, SOLID, SOLID), np.zeros((0, 3)), np.zeros((len(xy), 3)),
                    area, h, {"nx": nx, "ny": ny, "jitter": jitter, "seed": seed, "H": (ny - 1) * h})


# --------------------------------------------------------------------------
# Cylinder in a channel
# --------------------------------------------------------------------------
def karman(seed: int = 2, D: float = 40.0, length_d: float = 22.0, height_d: float = 4.1,
           center_d: tuple = (2.0, 2.0), U0: float = 0.05, r_fine: float = 0.37, r_coarse: float = 0.74,
           fine_band_d: float = 1.5, blend_to_d: float = 4.0, scale: float = 1.0,
           lattice_beyond_d: float | None = None, areas: str = "voronoi",
           coarse_beyond_d: float | None = None, coarse_h: int = 2) -> Workload:
    """Channel length_d*D x height_d*D with a solid cylinder of diameter D.

    Lengths are in units of the reference spacing h_ref=1, so D is the number
    of spacings across the cylinder.  Scattered Poisson-disk nodes with radius
    r_fine within fine_band_d*D of the cylinder surface, blended linearly to
    r_coarse at blend_to_d*D.  The four straight sides carry equilibrium
    nodes on a regular row spaced r_coarse*1.19 apart: a parabolic inflow and
    outflow profile with maximum U0 on the left and right, zero velocity on
    the top and bottom, unit density everywhere.  No nodes closer than half
    the local radius to the cylinder surface apart from the wall nodes placed
    on it (arc spacing about 1.19 r_fine).  `scale` < 1 shrinks D and the
    channel together for small test cases.

    lattice_beyond_d (hybrid node set, Sec. 3.1's regular bulk with scattered
    refinement): nodes farther than lattice_beyond_d*D from the cylinder
    surface sit on the square lattice of unit spacing that also carries the
    side nodes (length and height are rounded to whole spacings); the
    scattered refinement fills the rest, its radius blended from r_fine
    (within min(fine_band_d, lattice_beyond_d/2)*D) to r_coarse at the
    lattice.  Requires r_coarse > 1/sqrt(2), so
    that no scattered node fits between lattice points.

    coarse_beyond_d (with lattice_beyond_d; the coarsened hybrid set of
    Sec. 3.1): beyond coarse_beyond_d*D from the surface only the lattice
    points whose coordinates are multiples of coarse_h remain (the sampling
    radius there is 0.75 coarse_h, so no scattered node fills the holes).

    areas: "voronoi" (default) gives each node the fluid part of its Voronoi
    cell (rastered), which weights the wall nodes on the cylinder surface by
    the half-cells they own; "spacing" gives each node the square of its
    local sampling radius, normalised to the fluid area."""
    D = D * scale
    lx, ly = length_d * D, height_d * D
    cx, cy, R = center_d[0] * D, center_d[1] * D, 0.5 * D
    # radius field on a grid
    nrx, nry = int(lx / 2) + 2, int(ly / 2) + 2
    gx, gy = np.meshgrid(np.linspace(0, lx, nrx), np.linspace(0, ly, nry), indexing="xy")
    dist = np.hypot(gx - cx, gy - cy) - R
    if lattice_beyond_d is not None:
        # the scattered refinement reaches the coarse radius where the lattice starts
        blend_to_d = lattice_beyond_d
        fine_band_d = min(fine_band_d, 0.5 * lattice_beyond_d)
    t = np.clip((dist - fine_band_d * D) / ((blend_to_d - fine_band_d) * D), 0.0, 1.0)
    rgrid = r_fine + t * (r_coarse - r_fine)
    if coarse_beyond_d is not None:
        if lattice_beyond_d is None or coarse_beyond_d <= lattice_beyond_d:
            raise ValueError("coarsening needs a hybrid set with coarse_beyond_d > lattice_beyond_d")
        rgrid = np.where(dist > coarse_beyond_d * D, 0.75 * coarse_h, rgrid)
    # equilibrium nodes on the four sides
    hb = r_coarse * 1.19
    if lattice_beyond_d is not None:
        if r_coarse <= 0.5 ** 0.5:
            raise ValueError("hybrid node sets need r_coarse > 1/sqrt(2)")
        lx, ly = float(round(lx)), float(round(ly))
        hb = 1.0
    nbx = int(round(lx / hb)); nby = int(round(ly / hb))
    xs = np.linspace(0.0, lx, nbx + 1)
    ys = np.linspace(0.0, ly, nby + 1)
    bottom = np.stack([xs, np.zeros_like(xs)], 1)
    top = np.stack([xs, np.full_like(xs, ly)], 1)
    left = np.stack([np.zeros(nby - 1), ys[1:-1]], 1)
    right = np.stack([np.full(nby - 1, lx), ys[1:-1]], 1)
    fixed = np.concatenate([bottom, top, left, right], 0)
    nf = len(fixed)
    # wall nodes on the cylinder surface, arc spacing ~ the fine spacing
    m = int(round(np.pi * 2 * R / (r_fine * 1.19)))
    ph = np.random.default_rng(seed).uniform(0, 2 * np.pi)
    a = ph + 2 * np.pi * np.arange(m) / m
    surface = np.stack([cx + R * np.cos(a), cy + R * np.sin(a)], 1)
    pre = [fixed, surface]
    if lattice_beyond_d is not None:
        gx_, gy_ = np.meshgrid(np.arange(1, int(lx)), np.arange(1, int(ly)), indexing="xy")
        lat = np.stack([gx_.ravel(), gy_.ravel()], 1).astype(np.float64)
        dlat = np.hypot(lat[:, 0] - cx, lat[:, 1] - cy) - R
        far = dlat > lattice_beyond_d * D
        if coarse_beyond_d is not None:
            on_coarse = (np.mod(lat[:, 0], coarse_h) == 0) & (np.mod(lat[:, 1], coarse_h) == 0)
            far &= (dlat <= coarse_beyond_d * D) | on_coarse
        pre.append(lat[far])
    pts = _sample((0.0, 0.0, lx, ly), (0, 0), rgrid, np.array([[cx, cy, R]]), 0.5,
                  np.concatenate(pre, 0), seed,
                  max_out=int(4 * lx * ly / r_fine ** 2) + sum(len(p) for p in pre) + 1000)
    n = len(pts)
    cls = np.zeros(n, np.uint8)
    cls[:nf] = EQ
    cls[nf:nf + m] = WALL
    eqv = np.zeros((n, 3))
    eqv[:nf, 0] = 1.0
    side_lr = np.zeros(n, bool)
    side_lr[len(bottom) + len(top):nf] = True
    yb = pts[:, 1]
    prof = 4.0 * U0 * yb * (ly - yb) / (ly * ly)
    eqv[side_lr, 1] = prof[side_lr]
    # local spacing^2 as node area, normalised to the fluid area
    fx = np.clip(pts[:, 0] / lx * (nrx - 1), 0, nrx - 1.000001)
    fy = np.clip(pts[:, 1] / ly * (nry - 1), 0, nry - 1.000001)
    r_at = rgrid[fy.astype(int), fx.astype(int)]
    if areas == "voronoi":
        reach = R + (fine_band_d + 0.5) * D
        fine = (max(0.0, cx - reach), max(0.0, cy - reach), min(lx, cx + reach), min(ly, cy + reach), 0.05)
        area = fluid_voronoi_areas(pts, (0.0, 0.0, lx, ly), (False, False), np.array([[cx, cy, R]]), 0.25, fine)
    else:
        area = r_at ** 2
        area *= (lx * ly - np.pi * R * R) / area.sum()
    name = f"karman_D{D:g}_s{seed}" + ("" if lattice_beyond_d is None else f"_hybrid{lattice_beyond_d:g}") + \
        ("" if coarse_beyond_d is None else f"_coarse{coarse_beyond_d:g}x{coarse_h}") + \
        ("" if areas == "spacing" else "_" + areas)
    return Workload(name, pts, cls, (0.0, 0.0, lx, ly), (OPEN,) * 4,
                    np.array([[cx, cy, R]]), eqv, area, 1.0,
                    {"D": D, "U0": U0, "H": ly, "L": lx, "seed": seed, "n_eq": nf, "n_wall": m,
                     "lattice_beyond_d": lattice_beyond_d, "coarse_beyond_d": coarse_beyond_d})


# --------------------------------------------------------------------------
# Porous box
# --------------------------------------------------------------------------
def _rsa_disks(rng, lx, ly, porosity, rmin, rmax, gap, wall_gap, max_tries=400000):
    """Random sequential addition of non-overlapping disks, periodic in x,
    kept wall_gap away from the walls at y=0 and y=ly, until the solid area
    fraction reaches 1 - porosity (or the tries run out)."""
    target = (1.0 - porosity) * lx * ly
    disks = []
    area = 0.0
    cx = np.zeros(0); cy = np.zeros(0); cr = np.zeros(0)
    tries = 0
    while area < target and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin, rmax)
        x = rng.uniform(0.0, lx)
        y = rng.uniform(r + wall_gap, ly - r - wall_gap)
        if len(cx):
            dx = np.abs(cx - x)
            dx = np.minimum(dx, lx - dx)
            dy = cy - y
            if np.any(dx * dx + dy * dy < (cr + r + gap) ** 2):
                continue
        disks.append((x, y, r))
        cx = np.append(cx, x); cy = np.append(cy, y); cr = np.append(cr, r)
        area += np.pi * r * r
    return np.array(disks, dtype=np.float64).reshape(-1, 3)


def porous(seed: int = 3, n_target: int = 1_000_000, porosity: float = 0.7, rmin: float = 8.0,
           rmax: float = 16.0, h: float = 1.0, gap: float = 2.0, r_pd: float = 0.84,
           side: float | None = None, areas: str = "uniform") -> Workload:
    """Square box of random non-overlapping solid disks (radii U(rmin, rmax) in
    units of h), periodic in x, solid walls at y=0 and y=L.  Wall nodes sit on
    every solid surface (arc spacing about h); fluid nodes are Poisson-disk
    samples of radius r_pd*h that keep r_pd*h from the wall nodes.  The side
    length is chosen so the fluid holds about n_target nodes.  areas:
    "uniform" (fluid area / n for every node) or "voronoi" (the fluid part of
    each node's Voronoi cell, rastered at 0.2h; wall nodes own about half a
    cell)."""
    rng = np.random.default_rng(seed)
    density = 0.68 / (r_pd * h) ** 2          # nodes per unit area for Bridson sampling
    if side is None:
        side = float(np.sqrt(n_target / (porosity * density)))
    lx = ly = side
    disks = _rsa_disks(rng, lx, ly, porosity, rmin * h, rmax * h, gap * h, 2.0 * h)
    fixed = []
    for (x, y, r) in disks:
        m = max(8, int(round(2 * np.pi * r / h)))
        ph = rng.uniform(0, 2 * np.pi)
        a = ph + 2 * np.pi * np.arange(m) / m
        px = np.mod(x + r * np.cos(a), lx)
        fixed.append(np.stack([px, y + r * np.sin(a)], 1))
    nw = int(round(lx / h))
    xs = (np.arange(nw) + rng.uniform(0, 1)) * (lx / nw)
    xs = np.mod(xs, lx)
    fixed.append(np.stack([xs, np.zeros(nw)], 1))
    fixed.append(np.stack([xs, np.full(nw, ly)], 1))
    fixed = np.concatenate(fixed, 0)
    rgrid = np.full((2, 2), r_pd * h)
    # the top wall row sits at y = ly, outside the half-open sampling box: keep
    # it as a fixed point by sampling in a box that includes it
    pts = _sample((0.0, 0.0, lx, ly * (1 + 1e-12) + 1e-9), (1, 0), rgrid, disks, 0.25, fixed, seed,
                  max_out=int(2.0 * lx * ly * density) + len(fixed) + 1000)
    n = len(pts)
    cls = np.zeros(n, np.uint8)
    cls[:len(fixed)] = WALL
    fluid_area = lx * ly - np.sum(np.pi * disks[:, 2] ** 2)
    if areas == "voronoi":
        area = fluid_voronoi_areas(pts, (0.0, 0.0, lx, ly), (True, False), disks, 0.2 * h)
    else:
        area = np.full(n, fluid_area / n)
    phi = fluid_area / (lx * ly)
    return Workload(f"porous_n{n}_s{seed}" + ("" if areas == "uniform" else "_" + areas), pts, cls,
                    (0.0, 0.0, lx, ly), (PERIODIC, PERIODIC, SOLID, SOLID),
                    disks, np.zeros((n, 3)), area, h,
                    {"seed": seed, "porosity": float(phi), "n_disks": len(disks), "L": lx,
                     "mean_d": float(2 * disks[:, 2].mean()) if len(disks) else 0.0})


def porous_batch_specs(n_samples: int = 64, first_seed: int = 1000) -> list:
    """The batched porous configuration: sample i (seed first_seed + i) draws
    its node count from U(50k, 400k) and its porosity from U(0.5, 0.85) with
    its own seed; its streaming distance cycles through {1, 1/2, 1/4} and its
    body force through {1e-6, 5e-6, 2e-5} (Darcy and inertial samples mixed).
    tau = 1 (MLBM1) for every sample."""
    out = []
    for i in range(n_samples):
        rng = np.random.default_rng(first_seed + i)
        n = int(rng.uniform(50_000, 400_000))
        phi = float(rng.uniform(0.5, 0.85))
        out.append({"seed": first_seed + i, "n_target": n, "porosity": phi,
                    "s": [1.0, 0.5, 0.25][i % 3], "g": [1e-6, 5e-6, 2e-5][i % 3]})
    return out


def porous_from_spec(spec: dict) -> Workload:
    """porous() for one spec of porous_batch_specs (or any dict with seed,
    n_target and porosity).  Porosity below ~0.55 is out of reach for
    non-overlapping disks with a 2-spacing gap, so those samples use a gap of
    1; the sampler keeps the porosity it reached."""
    gap = spec.get("gap", 1.0 if spec["porosity"] < 0.6 else 2.0)
    return porous(seed=int(spec["seed"]), n_target=int(spec["n_target"]), porosity=float(spec["porosity"]),
                  gap=gap)


def generate(specs: list, procs: int | None = None) -> list:
    """porous_from_spec over many specs in a spawn-started process pool (safe
    to use before or after CUDA is initialised in the calling process)."""
    import multiprocessing as mp
    import os
    procs = procs or min(16, os.cpu_count() or 4, len(specs))
    if procs <= 1 or len(specs) <= 1:
        return [porous_from_spec(s) for s in specs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(porous_from_spec, specs)


def cylinder_array(side: float = 40.0, radius: float = 8.0, h: float = 1.0, seed: int = 0,
                   r_pd: float = 0.84, areas: str = "voronoi") -> Workload:
    """One solid disk of the given radius at the centre of a doubly periodic
    square cell of the given side: a square array of cylinders with solid
    area fraction c = pi r^2 / side^2.  Wall nodes sit on the circle (arc
    spacing about h); fluid nodes are Poisson-disk samples of radius r_pd*h.
    areas: "voronoi" (fluid part of each node's Voronoi cell, rastered at
    0.2h) or "uniform"."""
    rng = np.random.default_rng(seed)
    c = side / 2.0
    disks = np.array([[c, c, radius]])
    m = max(8, int(round(2 * np.pi * radius / h)))
    a = rng.uniform(0, 2 * np.pi) + 2 * np.pi * np.arange(m) / m
    fixed = np.stack([c + radius * np.cos(a), c + radius * np.sin(a)], 1)
    density = 0.68 / (r_pd * h) ** 2
    box = (0.0, 0.0, side, side)
    pts = _sample(box, (1, 1), np.full((2, 2), r_pd * h), disks, 0.25, fixed, seed,
                  max_out=int(2.0 * side * side * density) + m + 1000)
    n = len(pts)
    cls = np.zeros(n, np.uint8)
    cls[:m] = WALL
    fluid_area = side * side - np.pi * radius ** 2
    if areas == "voronoi":
        area = fluid_voronoi_areas(pts, box, (True, True), disks, 0.2 * h)
    else:
        area = np.full(n, fluid_area / n)
    return Workload(f"cylarray_L{side:g}_r{radius:g}_s{seed}", pts, cls, box,
                    (PERIODIC, PERIODIC, PERIODIC, PERIODIC), disks, np.zeros((n, 3)), area, h,
                    {"seed": seed, "solid_fraction": float(np.pi * radius ** 2 / side ** 2), "L": side})


def karman_lattice(d_lb: float, u0: float = 0.05, length_d: float = 22.0, height_d: float = 4.1,
                   center_d: tuple = (2.0, 2.0)):
    """The vortex-street channel of `karman` on a regular lattice (the lattice
    LBM comparison of Sec. 3.1): D = d_lb lattice spacings, cells (ny, nx)
    with class 0 fluid, 1 solid (cell centre inside the cylinder), 2
    equilibrium (the four sides: parabolic inflow and outflow with maximum u0,
    rest on the top and bottom, unit density).  Returns (cell, eq_values
    [ny][nx][3] = rho, ux, uy)."""
    nx, ny = int(round(length_d * d_lb)), int(round(height_d * d_lb))
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cx, cy, r = center_d[0] * d_lb, center_d[1] * d_lb, 0.5 * d_lb
    cell = np.zeros((ny, nx), np.uint8)
    cell[(x - cx) ** 2 + (y - cy) ** 2 < r * r] = 1
    top_bottom = (y == 0) | (y == ny - 1)
    left_right = (x == 0) | (x == nx - 1)
    cell[top_bottom | left_right] = 2
    eqv = np.zeros((ny, nx, 3))
    eqv[..., 0] = 1.0
    h = ny - 1.0
    eqv[..., 1] = np.where(left_right & ~top_bottom, 4.0 * u0 * y * (h - y) / (h * h), 0.0)
    return cell, eqv


def wall_geometry(w: Workload, tol: float = 1e-6):
    """Wall nodes on the solid disks and on the straight solid sides of a node
    set, with the unit normal pointing out of the solid into the fluid and the
    length of wall each node stands for (half the gaps to its two neighbours
    along the same surface).  Returns (nodes int64[m], normals[m][2], ds[m]).
    Geometry only: used to integrate a wall traction along the surfaces."""
    x0, y0, x1, y1 = w.box
    lx, ly = x1 - x0, y1 - y0
    per_x, per_y = w.sides[0] == PERIODIC, w.sides[2] == PERIODIC
    wall = np.nonzero(w.node_class == WALL)[0]
    nodes, nrm, ds = [], [], []
    for (cx, cy, r) in np.asarray(w.disks, np.float64).reshape(-1, 3):
        d = w.xy[wall] - np.array([cx, cy])
        if per_x:
            d[:, 0] -= lx * np.round(d[:, 0] / lx)
        if per_y:
            d[:, 1] -= ly * np.round(d[:, 1] / ly)
        on = np.abs(np.hypot(d[:, 0], d[:, 1]) - r) <= tol * max(1.0, r)
        if not on.any():
            continue
        th = np.arctan2(d[on, 1], d[on, 0])
        o = np.argsort(th)
        ids, th = wall[on][o], th[o]
        if len(th) == 1:
            gaps = np.array([2 * np.pi])
        else:
            nxt = np.roll(th, -1) - th
            nxt[-1] += 2 * np.pi
            gaps = 0.5 * (nxt + np.roll(nxt, 1))
        nodes.append(ids)
        nrm.append(np.stack([np.cos(th), np.sin(th)], 1))
        ds.append(gaps * r)
    # straight solid sides: (side index, coordinate axis, wall position, normal)
    for side, axis, pos, nv in ((2, 1, y0, (0.0, 1.0)), (3, 1, y1, (0.0, -1.0)),
                                (0, 0, x0, (1.0, 0.0)), (1, 0, x1, (-1.0, 0.0))):
        if w.sides[side] != SOLID:
            continue
        on = np.abs(w.xy[wall, axis] - pos) <= tol * max(1.0, abs(pos))
        if not on.any():
            continue
        t = w.xy[wall[on], 1 - axis]
        o = np.argsort(t)
        ids, t = wall[on][o], t[o]
        length = lx if axis == 1 else ly
        periodic = per_x if axis == 1 else per_y
        if periodic:
            nxt = np.roll(t, -1) - t
            nxt[-1] += length
            gaps = 0.5 * (nxt + np.roll(nxt, 1))
        else:
            lo, hi = (x0, x1) if axis == 1 else (y0, y1)
            edges = np.concatenate([[lo], 0.5 * (t[1:] + t[:-1]), [hi]])
            gaps = np.diff(edges)
        nodes.append(ids)
        nrm.append(np.tile(np.array(nv), (len(ids), 1)))
        ds.append(gaps)
    if not nodes:
        return np.zeros(0, np.int64), np.zeros((0, 2)), np.zeros(0)
    return (np.concatenate(nodes).astype(np.int64), np.concatenate(nrm, 0), np.concatenate(ds))


# --------------------------------------------------------------------------
# Random arrays (initial perturbations, feature noise); no physics
# --------------------------------------------------------------------------
def uniform_noise(shape, seed: int, amp: float = 1.0) -> np.ndarray:
    """U(-amp, amp) float64 array from a seeded generator."""
    return np.random.default_rng(seed).uniform(-amp, amp, size=shape)


def normal_noise(shape, seed: int, std: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).normal(0.0, std, size=shape)
