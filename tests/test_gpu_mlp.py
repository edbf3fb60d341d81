"""GPU parity of the warm-start network and features against the FP64 oracles.

Forward and gradients: the oracle runs with the kernels' BF16 rounding points
(features, weights, hidden activations, output and hidden errors rounded to
BF16, everything else exact), so the only difference left is FP32
accumulation order and the rare BF16 rounding flip it causes.  Element by
element, per output column and per parameter tensor:
  * every element within 5e-3 of the column's / tensor's largest magnitude
    (one BF16 flip of a hidden value moves an output by about 2^-8 times one
    weight times that value, a few 1e-4 of the scale, while a wrong row, a
    transposed weight block or a dropped term moves elements by O(scale));
  * at least 99.5% of the elements within 1e-4 of that scale plus 1e-3 of
    their own magnitude (the FP32 accumulation order alone);
and the relative L2 error of each column / tensor at most 1e-3.
"""
import numpy as np
import pytest

from oracle import features as OF
from oracle import mlp as OM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_14789_gb300 import mlbm
    return mlbm


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-300))


def _assert_elementwise(a, b, what):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape, what
    scale = float(np.max(np.abs(b))) if b.size else 0.0
    d = np.abs(a - b)
    worst = int(np.argmax(d)) if d.size else 0
    assert np.all(d <= 5e-3 * scale), (what, worst, float(d.flat[worst]), scale)
    tight = d <= 1e-4 * scale + 1e-3 * np.abs(b)
    assert tight.mean() >= 0.995, (what, float(tight.mean()))
    assert _rel(a, b) <= 1e-3, (what, _rel(a, b))


def _params(seed, bias_scale=0.1, n_out=2):
    rng = np.random.default_rng(seed + 100)
    p = OM.init_params(seed, n_out)
    for l in range(1, 8, 2):
        p[l] = bias_scale * rng.standard_normal(p[l].shape)
    return p


def _to_f32(params):
    """FP32 copy of the oracle's parameters (what the kernels hold) and its
    FP64 image for the oracle."""
    flat = OM.pack(params).astype(np.float32)
    return flat, OM.unpack(flat.astype(np.float64), params[-1].size)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("n_out", [2, 3])
@pytest.mark.parametrize("n", [1, 15, 16, 17, 64, 65, 1037, 20011])
def test_forward_matches_oracle(M, n, n_out):
    flat, p64 = _to_f32(_params(1, n_out=n_out))
    net = M.Mlp(3, n_out)
    net.set_params(flat)
    X = np.random.default_rng(n).normal(size=(n, 16))
    Xd = _dev(X)
    Yd = torch.empty((n, n_out), dtype=torch.float32, device="cuda")
    net.forward(Xd.data_ptr(), n, Yd.data_ptr())
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy()
    Yo, _ = OM.forward(p64, X.astype(np.float32).astype(np.float64), bf16_round=True)
    for j in range(n_out):
        _assert_elementwise(Y[:, j], Yo[:, j], f"output column {j}")


def test_forward_empty(M):
    net = M.Mlp(3)
    net.forward(0, 0, 0)


@pytest.mark.parametrize("n_out", [2, 3])
@pytest.mark.parametrize("n", [1, 17, 64, 65, 3001, 40000])
def test_gradients_match_oracle(M, n, n_out):
    flat, p64 = _to_f32(_params(2, n_out=n_out))
    net = M.Mlp(3, n_out)
    net.set_params(flat)
    rng = np.random.default_rng(7 + n)
    X = rng.normal(size=(n, 16)).astype(np.float32)
    T = rng.normal(size=(n, n_out)).astype(np.float32)
    Xd, Td = _dev(X), _dev(T)
    G = torch.empty(net.param_count(), dtype=torch.float32, device="cuda")
    loss = net.gradients(Xd.data_ptr(), Td.data_ptr(), n, G.data_ptr())
    g_gpu = OM.unpack(G.cpu().numpy().astype(np.float64), n_out)
    g_or = OM.gradients(p64, X.astype(np.float64), T.astype(np.float64), bf16_round=True)
    l_or = OM.loss(p64, X.astype(np.float64), T.astype(np.float64), bf16_round=True)
    assert abs(loss - l_or) <= 1e-3 * l_or
    for k, (a, b) in enumerate(zip(g_gpu, g_or)):
        _assert_elementwise(a, b, f"parameter tensor {k}")


def test_gradients_reproducible(M):
    flat, _ = _to_f32(_params(4))
    net = M.Mlp(3)
    net.set_params(flat)
    rng = np.random.default_rng(11)
    n = 50000
    Xd, Td = _dev(rng.normal(size=(n, 16))), _dev(rng.normal(size=(n, 2)))
    G1 = torch.empty(net.param_count(), dtype=torch.float32, device="cuda")
    G2 = torch.empty_like(G1)
    l1 = net.gradients(Xd.data_ptr(), Td.data_ptr(), n, G1.data_ptr())
    l2 = net.gradients(Xd.data_ptr(), Td.data_ptr(), n, G2.data_ptr())
    assert l1 == l2 and torch.equal(G1, G2)


def test_adam_steps_match_oracle(M):
    params = _params(5)
    flat, p64 = _to_f32(params)
    net = M.Mlp(3)
    net.set_params(flat)
    rng = np.random.default_rng(12)
    n = 3000
    X = rng.normal(size=(n, 16)).astype(np.float32).astype(np.float64)
    T = rng.normal(size=(n, 2)).astype(np.float32).astype(np.float64)
    Xd, Td = _dev(X), _dev(T)
    lr = 1e-3
    m = [np.zeros_like(a) for a in p64]
    v = [np.zeros_like(a) for a in p64]
    p = p64
    for t in (1, 2):
        g = OM.gradients(p, X, T, bf16_round=True)
        p_new, m, v = OM.adam_step(p, g, m, v, t, lr)
        net.train(Xd.data_ptr(), Td.data_ptr(), n, n, 1, lr, 0)
        got = OM.unpack(net.get_params().astype(np.float64))
        for k in range(len(p)):
            sel = np.abs(g[k]) > 1e-4 * np.abs(g[k]).max()
            # the step is lr * m_hat / (sqrt(v_hat) + eps): an O(lr) move per
            # entry, FP32 master weights
            err = np.abs((got[k] - p[k]) - (p_new[k] - p[k]))[sel]
            assert err.max() <= 2e-2 * lr + 1e-7, (t, k, err.max())
        p = got                          # continue from the kernel's parameters


def test_training_lowers_loss(M):
    teacher = _params(6, bias_scale=0.05)
    rng = np.random.default_rng(13)
    n = 8192
    X = rng.normal(size=(n, 16))
    T, _ = OM.forward(teacher, X)
    Xd, Td = _dev(X), _dev(T)
    net = M.Mlp(21)
    l0 = net.gradients(Xd.data_ptr(), Td.data_ptr(), n)
    net.train(Xd.data_ptr(), Td.data_ptr(), n, 1024, 600, 2e-3, 99)
    l1 = net.gradients(Xd.data_ptr(), Td.data_ptr(), n)
    assert l1 < 0.1 * l0, (l0, l1)


def test_bad_arguments(M):
    net = M.Mlp(1)
    with pytest.raises(M.MlbmError):
        net.forward(0, -1, 0)
    with pytest.raises(ValueError):
        net.set_params(np.zeros(3, np.float32))
    with pytest.raises(M.MlbmError):
        net.train(0, 0, 10, 10, 1, 1e-3, 0)


# ------------------------------------------------------------------ features
def _feature_cases():
    from paper_2312_14789_gb300 import inputs as I
    w = I.porous(seed=7, n_target=6000, porosity=0.7)
    yield "porous", w.xy, w.box, w.sides, w.disks, 12.0
    rng = np.random.default_rng(2)
    xy = np.stack([rng.uniform(0, 30, 500), rng.uniform(0, 22, 500)], 1)
    yield "doubly_periodic", xy, (0, 0, 30.0, 22.0), (0, 0, 0, 0), np.array([[4.0, 19.0, 3.0], [21.0, 6.0, 4.5]]), 2.5
    xy = np.stack([rng.uniform(0, 30, 300), rng.uniform(0, 80, 300)], 1)
    yield "vertical_channel", xy, (0, 0, 30.0, 80.0), (1, 1, 0, 0), None, 6.0
    yield "no_solid", xy, (0, 0, 30.0, 80.0), (0, 0, 0, 0), None, 6.0


def _compare_features(got, ref, L):
    """FP32 features against the FP64 oracle: every entry within 5e-5 except
    where the choice itself is ambiguous at FP32 resolution (the nearest of
    two nearly equidistant objects decides the direction; a ray grazing a
    disk decides hit or miss); those may differ in at most 0.2 % of the rows."""
    err = np.abs(got - ref)
    tol = 5e-5
    ambiguous_dir = np.abs(ref[:, 3] - ref[:, 0]) * L < 1e-3      # d2 - d1 in length units
    bad = err > tol
    bad[ambiguous_dir, 1:3] = False
    ray_cols = [4, 5, 6, 7, 8, 9]
    ray_rows = bad[:, ray_cols].any(axis=1)
    assert ray_rows.mean() <= 2e-3, (ray_rows.sum(), len(ray_rows))
    bad[:, ray_cols] = False
    assert not bad.any(), (np.argwhere(bad)[:5], err[bad][:5])


@pytest.mark.parametrize("case", list(range(4)))
def test_features_match_oracle(M, case):
    name, xy, box, sides, disks, L = list(_feature_cases())[case]
    n = len(xy)
    Xd = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    M.features_device(xy, box, sides, disks, L, Xd.data_ptr())
    got = Xd.cpu().numpy().astype(np.float64)
    ref = OF.features(xy, box, sides, disks, L)
    _compare_features(got, ref, L)


def test_features_full_size_sampled(M):
    from paper_2312_14789_gb300 import inputs as I
    w = I.porous(seed=20000, n_target=200_000, porosity=0.7)
    L = w.meta["mean_d"] / 2
    Xd = torch.empty((w.n, 16), dtype=torch.float32, device="cuda")
    M.features_for(w, L, Xd.data_ptr())
    pick = np.random.default_rng(0).choice(w.n, 3000, replace=False)
    pick = np.concatenate([pick, [0, w.n - 1]])
    got = Xd.cpu().numpy()[pick].astype(np.float64)
    ref = OF.features(w.xy[pick], w.box, w.sides, w.disks, L)
    _compare_features(got, ref, L)


# ---------------------------------------------------------------- warm start
def _small_ctx(M, seed=7, model=1):
    from paper_2312_14789_gb300 import inputs as I
    w = I.porous(seed=seed, n_target=6000, porosity=0.7)
    st = M.build_stencils_for(w, K=16, s=1.0, bb_mode=M.BB_INTERPOLATED)
    p = M.Params(model, 1.0 if model == 1 else 0.8, 0.0, 0.0, 0.0)
    return w, st, p


def test_warm_start_sets_prediction(M):
    for model in (1, 0):
        w, st, p = _small_ctx(M, model=model)
        ctx = M.init(st, p)
        net = M.Mlp(5)
        L = w.meta["mean_d"] / 2
        Xd = torch.empty((w.n, 16), dtype=torch.float32, device="cuda")
        M.features_for(w, L, Xd.data_ptr())
        Yd = torch.empty((w.n, 2), dtype=torch.float32, device="cuda")
        net.forward(Xd.data_ptr(), w.n, Yd.data_ptr())
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy().astype(np.float64)
        scale = 1e-3 / max(np.abs(Y).max(), 1e-30)
        assert M.warm_start(ctx, net, Xd.data_ptr(), scale) == 0
        ru = M.get_fields(ctx)
        assert np.allclose(ru[:, 0], 1.0, rtol=0, atol=1e-6)
        assert np.allclose(ru[:, 1:], scale * Y, rtol=1e-5, atol=1e-9)


def test_warm_start_density_keeps_mass(M):
    w, st, p = _small_ctx(M, seed=9)
    ctx = M.init(st, p)
    net = M.Mlp(5, 3)
    Xd = torch.empty((w.n, 16), dtype=torch.float32, device="cuda")
    M.features_for(w, 10.0, Xd.data_ptr())
    Yd = torch.empty((w.n, 3), dtype=torch.float32, device="cuda")
    net.forward(Xd.data_ptr(), w.n, Yd.data_ptr())
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.float64)
    su = 1e-3 / np.abs(Y[:, :2]).max()
    sr = 1e-4 / np.abs(Y[:, 2]).max()
    assert M.warm_start(ctx, net, Xd.data_ptr(), su, sr) == 0
    ru = M.get_fields(ctx)
    drho = sr * Y[:, 2].astype(np.float32).astype(np.float64)
    drho -= np.sum(drho * w.area) / np.sum(w.area)
    assert np.allclose(ru[:, 0] - 1.0, drho, rtol=0, atol=2e-9)
    assert abs(np.sum((ru[:, 0] - 1.0) * w.area)) <= 1e-9 * np.sum(w.area)
    assert np.allclose(ru[:, 1:], su * Y[:, :2], rtol=1e-5, atol=1e-9)
    with pytest.raises(M.MlbmError):
        M.warm_start(ctx, net, Xd.data_ptr(), su)          # 3 outputs need a density scale


def test_warm_start_cold_fallback(M):
    from paper_2312_14789_gb300 import inputs as I
    ws = [I.porous(seed=s, n_target=4000, porosity=0.7) for s in (8, 9)]
    sts = [M.build_stencils_for(w, K=16, s=1.0, bb_mode=M.BB_INTERPOLATED) for w in ws]
    ps = [M.Params(1, 1.0, 0.0, 1e-6, 0.0)] * 2
    ctx = M.batch_init(sts, ps)
    n = sum(w.n for w in ws)
    Xd = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    M.features_for(ws[0], 10.0, Xd[:ws[0].n].data_ptr())
    M.features_for(ws[1], 10.0, Xd[ws[0].n:].data_ptr())
    net = M.Mlp(5)
    Yd = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    net.forward(Xd.data_ptr(), n, Yd.data_ptr())
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.float64)
    s0 = 1e-3 / np.abs(Y).max()
    # the second sample's scale takes speeds far above 0.3: it starts from rest
    assert M.warm_start(ctx, net, Xd.data_ptr(), [s0, 1e6]) == 1
    ru = M.get_fields(ctx)
    n0 = ws[0].n
    assert np.allclose(ru[:n0, 1:], s0 * Y[:n0], rtol=1e-5, atol=1e-9)
    assert np.all(ru[n0:, 1:] == 0.0) and np.allclose(ru[:, 0], 1.0)
    with pytest.raises(M.MlbmError):
        M.warm_start(ctx, net, Xd.data_ptr(), [np.nan, 1.0])


def test_steady_check_interval(M):
    # the criterion evaluated every 100 steps against the snapshot of 1000
    # steps earlier stops within one window of the every-window evaluation,
    # at a multiple of 100, never later
    w, st, p = _small_ctx(M, seed=11)
    p = M.Params(1, 1.0, 0.0, 1e-6, 0.0)
    a = M.init(st, p)
    t1 = M.run_to_steady(a, 1e-7, 1000, 100_000)
    b = M.init(st, p)
    t2 = M.run_to_steady(b, 1e-7, 1000, 100_000, check=100)
    assert t2 % 100 == 0 and t1 - 1000 < t2 <= t1, (t1, t2)
    c = M.batch_init([st], [p])
    t3 = M.batch_run_to_steady(c, 1e-7, 1000, 100_000, check=100)
    assert t3[0] == t2
    with pytest.raises(M.MlbmError):
        M.run_to_steady(M.init(st, p), 1e-7, 1000, 10_000, check=300)
