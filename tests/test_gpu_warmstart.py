"""What the learned warm start gains: a network trained (on the GPU, by the
library's kernels) on small solved porous samples starts held-out samples
closer to their steady state (velocity and density), so they reach it in
fewer steps than from rest, and the converged permeability agrees with the
cold start's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_warm_start_reaches_steady_state_sooner():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_14789_gb300 import mlbm
    from paper_2312_14789_gb300 import warmstart as W

    nodes = 12_000
    ws_train = W.make_samples(range(10000, 10016), nodes)
    ws_test = W.make_samples(range(20000, 20004), nodes)
    par = lambda ws: [mlbm.Params(mlbm.MODEL_TAU1, 1.0, 0.0, 1e-6, 0.0) for _ in ws]

    sts = W.build(ws_train)
    ps = par(ws_train)
    ru, steps, _, _ = W.solve(sts, ps)
    X = W.features(ws_train)
    T = torch.from_numpy(W.targets(ws_train, ru, ps, 3)).cuda()
    net = mlbm.Mlp(1, 3)
    l0 = net.gradients(X.data_ptr(), T.data_ptr(), X.shape[0])
    W.train(net, X, T, 3000, batch=16384)
    l1 = net.gradients(X.data_ptr(), T.data_ptr(), X.shape[0])
    assert l1 < 0.2 * l0

    sts = W.build(ws_test)
    ps = par(ws_test)
    Xt = W.features(ws_test)
    ru_c, st_c, _, k_c = W.solve(sts, ps)
    ru_w, st_w, _, k_w = W.solve(sts, ps, init=W.warm_init(net, Xt, ws_test, ps))
    st_c, st_w = np.asarray(st_c, float), np.asarray(st_w, float)
    # every held-out sample converges sooner from the learned start
    assert np.all(st_w < st_c), (st_w, st_c)
    assert st_w.mean() <= 0.85 * st_c.mean(), (st_w, st_c)
    # and to the same permeability
    assert np.max(np.abs(k_w - k_c) / np.abs(k_c)) <= 1e-4
    # the learned initial field is much closer to the steady field than rest is
    Yd = torch.empty((Xt.shape[0], 3), dtype=torch.float32, device="cuda")
    net.forward(Xt.data_ptr(), Xt.shape[0], Yd.data_ptr())
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.float64)
    o = 0
    for w, p in zip(ws_test, ps):
        sc = W.velocity_scale(p.gx, p.tau, W.length_scale(w))
        u = ru_c[o:o + w.n, 1:]
        assert np.linalg.norm(sc * Y[o:o + w.n, :2] - u) <= 0.8 * np.linalg.norm(u)
        o += w.n
