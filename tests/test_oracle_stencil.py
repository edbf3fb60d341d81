"""Pins of the oracle's stencil machinery: neighbour search, weighted least
squares, biquadratic Lagrange weights and the bounce-back link geometry.

Independent checks: scipy's k-d tree (periodic boxsize) for the neighbour
sets, numpy's SVD least squares for the fit, exact polynomial reproduction,
and hand-worked segment/solid intersections.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle as O
from paper_2312_14789_gb300 import inputs as I


@pytest.mark.parametrize("K", [6, 9, 12, 16])
def test_knn_matches_kdtree_periodic(K):
    w = I.jittered_periodic(17, 13, 0.3, seed=4)
    idx, off = O.knn(w.xy, w.box, (True, True), K)
    tree = cKDTree(w.xy, boxsize=[w.box[2], w.box[3]])
    d, j = tree.query(w.xy, k=K)
    for i in range(w.n):
        assert set(idx[i]) == set(j[i])
        r = np.hypot(off[i, :, 0], off[i, :, 1])
        assert np.allclose(np.sort(r), d[i], rtol=0, atol=1e-12)
    assert np.all(idx[:, 0] == np.arange(w.n))  # self first (distance 0)


def test_knn_nonperiodic_and_targets():
    w = I.poiseuille_channel(12, 9, 0.2, seed=3)
    tg = np.array([0, 5, 50, 107])
    idx, off = O.knn(w.xy, w.box, (True, False), 10, targets=tg)
    lx = w.box[2]
    for t, i in enumerate(tg):
        dx = w.xy[:, 0] - w.xy[i, 0]
        dx = np.where(dx >= lx / 2, dx - lx, np.where(dx < -lx / 2, dx + lx, dx))
        d2 = dx ** 2 + (w.xy[:, 1] - w.xy[i, 1]) ** 2
        order = np.lexsort((np.arange(w.n), d2))[:10]
        assert np.array_equal(idx[t], order)


def test_knn_ties_broken_by_node_id():
    w = I.lattice(8, 8)
    idx, off = O.knn(w.xy, w.box, (True, True), 12)
    # node 0: self, 4 at distance 1, 4 at sqrt 2, then 3 of the 4 at distance 2,
    # the three with the lowest ids
    d2 = (off[0] ** 2).sum(1)
    assert np.array_equal(d2, [0, 1, 1, 1, 1, 2, 2, 2, 2, 4, 4, 4])
    rel = (w.xy - w.xy[0] + 4) % 8 - 4
    four = np.nonzero((rel ** 2).sum(1) == 4)[0]
    assert list(idx[0][9:]) == sorted(four)[:3]


def _rand_stencil(rng, K):
    off = rng.uniform(-1.5, 1.5, size=(K, 2))
    off[0] = 0.0
    return off


@pytest.mark.parametrize("K", [7, 9, 12, 16])
def test_wls_matches_svd_least_squares(K):
    rng = np.random.default_rng(K)
    for trial in range(5):
        off = _rand_stencil(rng, K)
        s = 0.7
        st, M = O.wls_matrix(off, s, 0.7071067811865476)
        assert st == 0
        rK = np.hypot(off[:, 0], off[:, 1]).max()
        sig = 0.7071067811865476 * rK
        wt = np.exp(-(off ** 2).sum(1) / sig ** 2)
        P = np.stack([np.ones(K), off[:, 0], off[:, 1], off[:, 0] ** 2, off[:, 0] * off[:, 1],
                      off[:, 1] ** 2], 1)
        f = rng.standard_normal(K)
        c, *_ = np.linalg.lstsq(P * np.sqrt(wt)[:, None], f * np.sqrt(wt), rcond=None)
        # M is stored in streaming-distance units: row i scaled by s^deg(i)
        scale = np.array([1, s, s, s * s, s * s, s * s])
        assert np.allclose(M @ f, c * scale, rtol=1e-10, atol=1e-12)


def test_wls_reproduces_quadratics_and_interpolates_with_six_points():
    rng = np.random.default_rng(1)
    for K in (6, 12, 16):
        off = _rand_stencil(rng, K)
        s = 0.9
        st, M = O.wls_matrix(off, s, 0.7071067811865476)
        assert st == 0
        a = rng.standard_normal(6)
        poly = lambda x, y: a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y
        f = poly(off[:, 0], off[:, 1])
        for d in rng.uniform(-1, 1, size=(5, 2)):
            p = np.array([1, d[0] / s, d[1] / s, (d[0] / s) ** 2, d[0] * d[1] / s ** 2, (d[1] / s) ** 2])
            assert abs(p @ M @ f - poly(*d)) < 1e-11
        if K == 6:  # square system: the fit interpolates any data
            g = rng.standard_normal(6)
            for j in range(6):
                d = off[j]
                p = np.array([1, d[0] / s, d[1] / s, (d[0] / s) ** 2, d[0] * d[1] / s ** 2, (d[1] / s) ** 2])
                assert abs(p @ M @ g - g[j]) < 1e-10


def test_wls_degenerate_stencil_is_rejected():
    off = np.stack([np.linspace(-1, 1, 9), np.zeros(9)], 1)  # collinear
    st, _ = O.wls_matrix(off, 1.0, 0.7071067811865476)
    assert st == 2


def test_lagrange_detection_and_weights():
    w = I.lattice(6, 6, h=0.5)
    idx, off = O.knn(w.xy, w.box, (True, True), 12)
    ok, slot, h, c = O.lagrange_detect(off[14], s=0.5)
    assert ok and h == 0.5 and c == 0
    for b in (-1, 0, 1):
        for a in (-1, 0, 1):
            assert np.allclose(off[14][slot[(b + 1) * 3 + a + 1]], [a * h, b * h])
    wj = I.jittered_periodic(6, 6, 0.2, seed=2)
    idx2, off2 = O.knn(wj.xy, wj.box, (True, True), 12)
    assert not O.lagrange_detect(off2[14])[0]


def test_lagrange_weights_reproduce_biquadratics_and_are_one_hot_on_nodes():
    w = I.lattice(7, 7)
    for s in (1.0, 0.37):
        op = O.Operator(w, K=12, s=s).check()
        assert np.all(op.kind == 1)
        rng = np.random.default_rng(3)
        c = rng.standard_normal(9)
        t = 20
        E, _, _ = O.lattice_constants()
        x0 = w.xy[t]
        for k in range(1, 9):
            wk = op.W[t, k]
            assert abs(wk.sum() - 1) < 1e-14
            off = op.off[t]
            bq = lambda x, y: sum(c[3 * i + j] * x ** i * y ** j for i in range(3) for j in range(3))
            val = wk @ bq(off[:, 0], off[:, 1])
            d = -s * E[k]
            assert abs(val - bq(*d)) < 1e-12
            if s == 1.0:
                assert np.sum(wk == 1.0) == 1 and np.sum(wk != 0.0) == 1


def test_bc_links_walls_and_disk():
    box = (0.0, 0.0, 10.0, 10.0)
    side = (0, 0, 1, 1)
    # node 0.3 above the bottom wall: directions with e_y = +1 cross at q = 0.3/s
    st, link, q = O.bc_links(5.0, 0.3, 1.0, box, side, np.zeros((0, 3)))
    assert st == 0
    assert list(np.nonzero(link)[0]) == [2, 5, 6]
    assert np.allclose(q[[2, 5, 6]], 0.3)
    # node on the wall: q = 0 for the same directions, none for tangential ones
    st, link, q = O.bc_links(5.0, 0.0, 0.5, box, side, np.zeros((0, 3)))
    assert list(np.nonzero(link)[0]) == [2, 5, 6] and np.all(q[[2, 5, 6]] == 0)
    # disk at (5, 5) radius 1; node at (6.5, 5): e_1 = (1, 0) departs towards -x
    disks = np.array([[5.0, 5.0, 1.0]])
    st, link, q = O.bc_links(6.5, 5.0, 1.0, box, side, disks)
    assert link[1] == 1 and abs(q[1] - 0.5) < 1e-15
    assert link[3] == 0
    # diagonal e_5 = (1, 1) from (6.2, 5): points (6.2 - t, 5 - t) relative to
    # the centre are (1.2 - t, -t); |.|^2 = 1 gives 2t^2 - 2.4t + 0.44 = 0
    st, link, q = O.bc_links(6.2, 5.0, 1.0, box, side, disks)
    tq = (2.4 - np.sqrt(2.4 ** 2 - 8 * 0.44)) / 4
    assert link[5] == 1 and abs(q[5] - tq) < 1e-14
    assert link[8] == 1 and abs(q[8] - tq) < 1e-14   # e_8 = (1, -1), mirror image
    assert abs(q[1] - 0.2) < 1e-14
    # node on the disk surface
    st, link, q = O.bc_links(6.0, 5.0, 0.5, box, side, disks)
    assert link[1] == 1 and q[1] == 0.0 and link[3] == 0
    # periodic image of a disk across x = 0
    disks = np.array([[0.5, 5.0, 1.0]])
    st, link, q = O.bc_links(9.0, 5.0, 1.0, box, side, disks)
    assert link[3] == 1 and abs(q[3] - 0.5) < 1e-15
    # node inside a solid
    st, link, q = O.bc_links(0.5, 5.0, 1.0, box, side, disks)
    assert st == 3
