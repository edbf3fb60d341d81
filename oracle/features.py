"""FP64 CPU oracle of the warm-start geometry features -- TEST INFRASTRUCTURE ONLY.

Sixteen numbers per node from the node position and the solid geometry
(disks, their periodic images, solid box sides), with a length scale L and a
ray length ell = min(8L, min(Lx, Ly)/2):

  0      clamp(d1/L, 0, 4), d1 = distance to the nearest solid surface
  1, 2   unit vector from that surface point to the node (zero without solids)
  3      clamp(d2/L, 0, 4), d2 = distance to the second nearest solid object
  4..7   free path along +x, -x, +y, -y (distance to the first solid met by
         the ray, at most ell) over L
  8      clamp(f(+y) f(-y)/L^2, 0, 16)
  9      clamp((f(+y) + f(-y))/L, 0, 8)
  10..13 1 - (solid area inside the circle of radius rho_j around the node)
         / (pi rho_j^2), rho_j = min(c_j L, min(Lx, Ly)/2), c_j = 1, 2, 4, 8
  14     1 - sum(pi r^2) / (Lx Ly)
  15     4 (y-y0)(y1-y)/Ly^2

Objects: every disk with the images ix, iy in {-1, 0, 1} (around the
minimum-image displacement) along each axis whose two sides are periodic,
then the solid sides (left, right, bottom, top).  With no object d1 = d2 =
4L.  Ties: the first object in that order gives the direction.  A ray meets
a disk where it enters it; an entry behind the start by more than 1e-4 r (a
node on the surface looking out of the solid) does not count.

The solid area inside a circle is the sum over objects of the closed-form
circle-circle intersection (lens) and circle/half-plane (segment) areas.
Plain numpy, vectorised over nodes only.  Pins: brute-force area counts on a
fine grid, brute-force nearest-surface distances and ray marches,
closed-form special cases (tests/test_oracle_features.py).
"""
from __future__ import annotations

import numpy as np

PERIODIC, SOLID = 0, 1
RADIUS_FACTORS = (1.0, 2.0, 4.0, 8.0)
NR = len(RADIUS_FACTORS)


def lens_area(d, a, b):
    """Area of the intersection of circles of radii a and b whose centres are
    d apart (arrays broadcast)."""
    d, a, b = np.broadcast_arrays(np.asarray(d, float), np.asarray(a, float), np.asarray(b, float))
    out = np.zeros(d.shape)
    apart = d >= a + b
    inside = (~apart) & (d <= np.abs(a - b))
    m = np.minimum(a, b)
    out[inside] = np.pi * m[inside] ** 2
    part = ~(apart | inside)
    dd, aa, bb = d[part], a[part], b[part]
    # half-angles subtended at each centre by the common chord (law of cosines)
    alpha = np.arccos(np.clip((dd ** 2 + aa ** 2 - bb ** 2) / (2 * dd * aa), -1, 1))
    beta = np.arccos(np.clip((dd ** 2 + bb ** 2 - aa ** 2) / (2 * dd * bb), -1, 1))
    # two circular sectors minus the kite between the centres and the chord ends
    kite = aa * dd * np.sin(alpha)
    out[part] = aa ** 2 * alpha + bb ** 2 * beta - kite
    return out


def segment_area(h, a):
    """Area of the part of a circle of radius a lying beyond a line at signed
    distance h from its centre."""
    h, a = np.broadcast_arrays(np.asarray(h, float), np.asarray(a, float))
    out = np.zeros(h.shape)
    full = h <= -a
    out[full] = np.pi * a[full] ** 2
    part = (h > -a) & (h < a)
    hh, aa = h[part], a[part]
    theta = np.arccos(hh / aa)            # half-angle of the chord
    out[part] = aa ** 2 * theta - hh * np.sqrt(aa ** 2 - hh ** 2)
    return out


def _ray_hits(along, across, r):
    """Distance from the node to where a ray along +axis enters a disk whose
    centre sits at (-along, -across) relative to the node in the ray frame
    (along = node - centre on the ray axis); inf where the ray misses."""
    half = np.sqrt(np.maximum(r * r - across ** 2, 0.0))      # half-chord at that offset
    entry = -along - half                                     # centre position minus half-chord
    ok = (np.abs(across) <= r) & (entry >= -1e-4 * r)
    return np.where(ok, np.maximum(entry, 0.0), np.inf)


def features(xy, box, sides, disks, L):
    """Features [n][16] (float64) of the nodes xy[n][2]."""
    xy = np.asarray(xy, float).reshape(-1, 2)
    disks = np.asarray(disks if disks is not None else np.zeros((0, 3)), float).reshape(-1, 3)
    x0, y0, x1, y1 = (float(v) for v in box)
    lx, ly = x1 - x0, y1 - y0
    perx = sides[0] == PERIODIC and sides[1] == PERIODIC
    pery = sides[2] == PERIODIC and sides[3] == PERIODIC
    rho = [min(c * L, 0.5 * min(lx, ly)) for c in RADIUS_FACTORS]
    ell = min(8.0 * L, 0.5 * min(lx, ly))
    x, y = xy[:, 0], xy[:, 1]
    n = len(xy)

    # candidate objects in the fixed order: (distance to surface, unit vector)
    dists, dirs = [], []
    solid_area = np.zeros((NR, n))
    free = np.full((4, n), ell)            # +x, -x, +y, -y
    for cx, cy, r in disks:
        dx0, dy0 = x - cx, y - cy
        if perx:
            dx0 = dx0 - lx * np.rint(dx0 / lx)
        if pery:
            dy0 = dy0 - ly * np.rint(dy0 / ly)
        for ix in ((-1, 0, 1) if perx else (0,)):
            for iy in ((-1, 0, 1) if pery else (0,)):
                dx, dy = dx0 + ix * lx, dy0 + iy * ly
                dist = np.hypot(dx, dy)
                safe = np.where(dist > 0, dist, 1.0)
                dists.append(dist - r)
                dirs.append(np.stack([np.where(dist > 0, dx / safe, 0.0), np.where(dist > 0, dy / safe, 0.0)], 1))
                # a ray along -x is a ray along +x in the mirrored frame
                free[0] = np.minimum(free[0], _ray_hits(dx, dy, r))
                free[1] = np.minimum(free[1], _ray_hits(-dx, dy, r))
                free[2] = np.minimum(free[2], _ray_hits(dy, dx, r))
                free[3] = np.minimum(free[3], _ray_hits(-dy, dx, r))
                for j in range(NR):
                    solid_area[j] += lens_area(dist, rho[j], r)
    walls = [(x - x0, (1.0, 0.0), 1), (x1 - x, (-1.0, 0.0), 0), (y - y0, (0.0, 1.0), 3), (y1 - y, (0.0, -1.0), 2)]
    for k, (h, nrm, ray) in enumerate(walls):
        if sides[k] != SOLID:
            continue
        dists.append(h)
        dirs.append(np.tile(np.array(nrm), (n, 1)))
        free[ray] = np.minimum(free[ray], np.maximum(h, 0.0))
        for j in range(NR):
            solid_area[j] += segment_area(h, rho[j])

    F = np.zeros((n, 16))
    if dists:
        D = np.stack(dists, 0)                        # [objects][n]
        first = np.argmin(D, axis=0)                  # first minimum in object order
        d1 = D[first, np.arange(n)]
        Dm = D.copy()
        Dm[first, np.arange(n)] = np.inf
        d2 = Dm.min(axis=0)
        direc = np.stack(dirs, 0)[first, np.arange(n)]
    else:
        d1 = np.full(n, np.inf)
        d2 = np.full(n, np.inf)
        direc = np.zeros((n, 2))
    d1 = np.where(np.isfinite(d1), d1, 4 * L)
    d2 = np.where(np.isfinite(d2), d2, 4 * L)
    F[:, 0] = np.clip(d1 / L, 0, 4)
    F[:, 1:3] = direc
    F[:, 3] = np.clip(d2 / L, 0, 4)
    F[:, 4:8] = free.T / L
    F[:, 8] = np.minimum(free[2] * free[3] / L ** 2, 16)
    F[:, 9] = np.minimum((free[2] + free[3]) / L, 8)
    for j in range(NR):
        F[:, 10 + j] = 1.0 - solid_area[j] / (np.pi * rho[j] ** 2)
    F[:, 14] = 1.0 - np.sum(np.pi * disks[:, 2] ** 2) / (lx * ly)
    F[:, 15] = 4.0 * (y - y0) * (y1 - y) / ly ** 2
    return F
