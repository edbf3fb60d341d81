"""Pins of the geometry-feature oracle: closed-form areas against brute-force
counts on fine grids, nearest-surface distances against brute force over
sampled surface points (periodic images written out explicitly), and special
cases with closed forms."""
import numpy as np
import pytest

from oracle import features as F
from paper_2312_14789_gb300 import inputs as I


def _grid_count(inside, x0, x1, y0, y1, m=1600):
    xs = x0 + (np.arange(m) + 0.5) * (x1 - x0) / m
    ys = y0 + (np.arange(m) + 0.5) * (y1 - y0) / m
    X, Y = np.meshgrid(xs, ys)
    return inside(X, Y).sum() * (x1 - x0) * (y1 - y0) / m ** 2


@pytest.mark.parametrize("d,a,b", [(0.0, 2.0, 1.0), (0.5, 2.0, 1.0), (1.5, 2.0, 1.0), (2.7, 2.0, 1.0),
                                   (3.5, 2.0, 1.0), (1.0, 1.0, 1.0), (0.3, 0.5, 3.0), (2.9, 0.5, 3.0)])
def test_lens_area_brute_force(d, a, b):
    exact = float(F.lens_area(d, a, b))
    r = max(a, b)
    est = _grid_count(lambda X, Y: (X ** 2 + Y ** 2 <= a * a) & ((X - d) ** 2 + Y ** 2 <= b * b),
                      -r, d + r, -r, r)
    assert abs(exact - est) <= 2e-3 * np.pi * min(a, b) ** 2 + 1e-12


@pytest.mark.parametrize("h", [-2.5, -1.2, -0.3, 0.0, 0.4, 1.7, 2.0, 3.0])
def test_segment_area_brute_force(h):
    a = 2.0
    exact = float(F.segment_area(h, a))
    est = _grid_count(lambda X, Y: (X ** 2 + Y ** 2 <= a * a) & (X >= h), -a, a, -a, a)
    assert abs(exact - est) <= 2e-3 * np.pi * a * a


def _small_porous():
    # a small periodic-in-x porous box with solid top and bottom walls
    return I.porous(seed=7, n_target=6000, porosity=0.7)


def test_local_porosity_brute_force():
    w = _small_porous()
    L = 12.0
    rng = np.random.default_rng(0)
    pick = rng.choice(w.n, 6, replace=False)
    Fx = F.features(w.xy[pick], w.box, w.sides, w.disks, L)
    x0, y0, x1, y1 = w.box
    lx, ly = x1 - x0, y1 - y0
    for row, i in enumerate(pick):
        px, py = w.xy[i]
        for j, c in enumerate(F.RADIUS_FACTORS):
            rho = min(c * L, 0.5 * min(lx, ly))

            def solid(X, Y):
                inside = (X - px) ** 2 + (Y - py) ** 2 <= rho * rho
                s = (Y < y0) | (Y > y1)                 # beyond the solid bottom / top walls
                for cx, cy, r in w.disks:
                    for k in (-1, 0, 1):                # explicit periodic copies in x
                        s |= (X - (cx + k * lx)) ** 2 + (Y - cy) ** 2 <= r * r
                return inside & s
            est = _grid_count(solid, px - rho, px + rho, py - rho, py + rho, m=900)
            phi = 1.0 - est / (np.pi * rho * rho)
            assert abs(Fx[row, 10 + j] - phi) <= 6e-3, (i, j, Fx[row, 10 + j], phi)


def test_nearest_surface_brute_force():
    w = _small_porous()
    L = 12.0
    rng = np.random.default_rng(1)
    pick = rng.choice(w.n, 40, replace=False)
    Fx = F.features(w.xy[pick], w.box, w.sides, w.disks, L)
    x0, y0, x1, y1 = w.box
    lx = x1 - x0
    t = np.linspace(0, 2 * np.pi, 4000, endpoint=False)
    pts = []
    for cx, cy, r in w.disks:
        for k in (-1, 0, 1):
            pts.append(np.stack([cx + k * lx + r * np.cos(t), cy + r * np.sin(t)], 1))
    xs = np.linspace(x0 - lx, x1 + lx, 60000)
    pts.append(np.stack([xs, np.full_like(xs, y0)], 1))
    pts.append(np.stack([xs, np.full_like(xs, y1)], 1))
    P = np.concatenate(pts, 0)
    for row, i in enumerate(pick):
        d = np.sqrt(((P - w.xy[i]) ** 2).sum(1)).min()
        assert abs(min(d / L, 4.0) - Fx[row, 0]) <= 0.02 / L, (i, d, Fx[row, 0] * L)
        # the surface point the direction points back to lies on a solid surface
        if Fx[row, 0] < 4.0:
            q = w.xy[i] - Fx[row, 0] * L * Fx[row, 1:3]
            dq = np.sqrt(((P - q) ** 2).sum(1)).min()
            assert dq <= 0.02
            assert abs(np.hypot(Fx[row, 1], Fx[row, 2]) - 1.0) <= 1e-12


def test_channel_closed_form():
    # plain channel: no disks, periodic in x, walls at y = 0 and y = H
    H, L = 40.0, 10.0
    ell = min(8 * L, 0.5 * H)
    y = np.array([0.0, 3.0, 10.0, 20.0, 37.5])
    xy = np.stack([np.full_like(y, 5.0), y], 1)
    Fx = F.features(xy, (0, 0, 100.0, H), (0, 0, 1, 1), None, L)
    d1, d2 = np.minimum(y, H - y), np.maximum(y, H - y)
    assert np.allclose(Fx[:, 0], np.minimum(d1 / L, 4))
    assert np.allclose(Fx[:, 3], np.minimum(d2 / L, 4))
    assert np.allclose(Fx[:, 2], np.where(y <= H / 2, 1.0, -1.0)) and np.allclose(Fx[:, 1], 0)
    up, down = np.minimum(H - y, ell), np.minimum(y, ell)
    assert np.allclose(Fx[:, 4:6], ell / L)
    assert np.allclose(Fx[:, 6], up / L) and np.allclose(Fx[:, 7], down / L)
    assert np.allclose(Fx[:, 8], np.minimum(up * down / L ** 2, 16))
    assert np.allclose(Fx[:, 9], np.minimum((up + down) / L, 8))
    # porosity within rho of a wall: circle minus segment beyond the wall
    rho = L
    for k, yy in enumerate(y):
        h = min(yy, H - yy)
        seg = 0.0 if h >= rho else rho * rho * np.arccos(h / rho) - h * np.sqrt(rho * rho - h * h)
        assert abs(Fx[k, 10] - (1 - seg / (np.pi * rho * rho))) <= 1e-12
    assert np.allclose(Fx[:, 14], 1.0)
    assert np.allclose(Fx[:, 15], 4 * y * (H - y) / H ** 2)


def test_no_solid_and_disk_inside_circle():
    L = 5.0
    xy = np.array([[10.0, 10.0], [30.0, 12.0]])
    Fx = F.features(xy, (0, 0, 100.0, 100.0), (0, 0, 0, 0), None, L)
    assert np.allclose(Fx[:, [0, 3]], 4) and np.allclose(Fx[:, 1:3], 0)
    assert np.allclose(Fx[:, 4:8], 8.0) and np.allclose(Fx[:, 8:10], [16, 8])
    assert np.allclose(Fx[:, 10:15], 1.0)
    # one disk of radius 1 at distance 3 from the node along +x: wholly inside
    # the circles of radius >= 4 (L, 2L, 4L, 8L -> min(., 50)); the +x ray
    # enters it at distance 2, the other rays miss it
    disks = np.array([[13.0, 10.0, 1.0]])
    Fx = F.features(xy[:1], (0, 0, 100.0, 100.0), (0, 0, 0, 0), disks, L)
    assert abs(Fx[0, 0] - 2.0 / L) <= 1e-12 and np.allclose(Fx[0, 1:3], [-1, 0])
    assert abs(Fx[0, 4] - 2.0 / L) <= 1e-12 and np.allclose(Fx[0, 5:8], 8.0)
    for j, c in enumerate(F.RADIUS_FACTORS):
        rho = min(c * L, 50.0)
        assert abs(Fx[0, 10 + j] - (1 - 1.0 / rho ** 2)) <= 1e-12
    assert abs(Fx[0, 14] - (1 - np.pi / 1e4)) <= 1e-15


def test_periodic_image_nearest():
    # a disk near the right edge is nearest to a node near the left edge
    # through its periodic image; the box is not square
    box, sides = (0.0, 0.0, 50.0, 20.0), (0, 0, 0, 0)
    disks = np.array([[48.0, 10.0, 1.5]])
    Fx = F.features(np.array([[1.0, 10.0]]), box, sides, disks, 2.0)
    assert abs(Fx[0, 0] - (3.0 - 1.5) / 2.0) <= 1e-12
    assert np.allclose(Fx[0, 1:3], [1.0, 0.0])


def test_global_porosity_matches_sampler():
    w = _small_porous()
    Fx = F.features(w.xy[:3], w.box, w.sides, w.disks, 12.0)
    assert np.allclose(Fx[:, 14], w.meta["porosity"], rtol=0, atol=1e-12)


def test_doubly_periodic_brute_force():
    # small non-square box periodic in x and y; every image within two box
    # lengths is written out explicitly
    box, sides = (0.0, 0.0, 30.0, 22.0), (0, 0, 0, 0)
    lx, ly = 30.0, 22.0
    disks = np.array([[4.0, 19.0, 3.0], [21.0, 6.0, 4.5]])
    L = 2.5
    rng = np.random.default_rng(3)
    xy = np.stack([rng.uniform(0, lx, 12), rng.uniform(0, ly, 12)], 1)
    Fx = F.features(xy, box, sides, disks, L)
    centres = [(cx + i * lx, cy + j * ly, r) for cx, cy, r in disks for i in range(-2, 3) for j in range(-2, 3)]
    for k, (px, py) in enumerate(xy):
        ds = sorted(np.hypot(px - cx, py - cy) - r for cx, cy, r in centres)
        if ds[0] < 0:
            continue                                  # node inside a disk: not a fluid node
        assert abs(Fx[k, 0] - min(ds[0] / L, 4)) <= 1e-12
        assert abs(Fx[k, 3] - min(ds[1] / L, 4)) <= 1e-12
        for j, c in enumerate(F.RADIUS_FACTORS):
            rho = min(c * L, 0.5 * min(lx, ly))

            def solid(X, Y):
                s = np.zeros(X.shape, bool)
                for cx, cy, r in centres:
                    s |= (X - cx) ** 2 + (Y - cy) ** 2 <= r * r
                return s & ((X - px) ** 2 + (Y - py) ** 2 <= rho * rho)
            est = _grid_count(solid, px - rho, px + rho, py - rho, py + rho, m=700)
            assert abs(Fx[k, 10 + j] - (1 - est / (np.pi * rho * rho))) <= 6e-3


def test_vertical_channel_closed_form():
    # walls on the left and right, periodic in y
    W, L = 30.0, 6.0
    x = np.array([0.0, 4.0, 15.0, 26.0, 30.0])
    xy = np.stack([x, np.full_like(x, 7.0)], 1)
    Fx = F.features(xy, (0, 0, W, 80.0), (1, 1, 0, 0), None, L)
    d1, d2 = np.minimum(x, W - x), np.maximum(x, W - x)
    assert np.allclose(Fx[:, 0], np.minimum(d1 / L, 4)) and np.allclose(Fx[:, 3], np.minimum(d2 / L, 4))
    assert np.allclose(Fx[:, 1], np.where(x <= W / 2, 1.0, -1.0)) and np.allclose(Fx[:, 2], 0)


def test_free_path_ray_march():
    # march each ray in small steps until it is inside a solid (disk images
    # written out, walls) or has gone ell
    w = _small_porous()
    L = 12.0
    x0, y0, x1, y1 = w.box
    lx, ly = x1 - x0, y1 - y0
    ell = min(8 * L, 0.5 * min(lx, ly))
    rng = np.random.default_rng(5)
    pick = rng.choice(w.n, 40, replace=False)
    Fx = F.features(w.xy[pick], w.box, w.sides, w.disks, L)
    C = np.array([(cx + k * lx, cy, r) for cx, cy, r in w.disks for k in (-1, 0, 1)])
    step = 2e-3
    t = np.arange(1, int(ell / step) + 1) * step
    for row, i in enumerate(pick):
        px, py = w.xy[i]
        for ray, (ex, ey) in enumerate([(1, 0), (-1, 0), (0, 1), (0, -1)]):
            X, Y = px + ex * t, py + ey * t
            solid = (Y < y0) | (Y > y1)
            for cx, cy, r in C:
                solid |= (X - cx) ** 2 + (Y - cy) ** 2 < r * r
            hit = t[np.argmax(solid)] if solid.any() else ell
            assert abs(Fx[row, 4 + ray] * L - min(hit, ell)) <= 2 * step + 1e-9, (i, ray, Fx[row, 4 + ray] * L, hit)
