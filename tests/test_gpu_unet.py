"""Warm-start network on the GPU against the float64 oracle: forward output,
every layer's gradients, one Adam step, and the warm start's fallback rule."""
import numpy as np
import pytest

import workloads
from oracle import joseph, unet as U

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


def _net(sl, H, W, n, seed):
    net = sl.UNet(H, W, max_batch=n)
    params = workloads.unet_init(seed, sl.UNET_LAYERS)
    # non-zero biases so that every bias path is exercised
    rng = np.random.default_rng(seed)
    params = {k: (w, (0.05 * rng.standard_normal(b.shape)).astype(np.float32))
              for k, (w, b) in params.items()}
    net.set_params(sl.flatten_params(params))
    return net, params


def test_layer_tables_agree(sl):
    assert [(a, tuple(b), c) for a, b, c in sl.UNET_LAYERS] == [(a, tuple(b), c) for a, b, c in U.LAYERS]
    assert sl.UNet(16, 16).nparams == U.param_count()


@pytest.mark.parametrize("H,W,n", [(16, 16, 2), (64, 40, 1), (24, 56, 3)])
def test_forward_matches_oracle(sl, H, W, n):
    net, params = _net(sl, H, W, n, 5)
    x = np.random.default_rng(1).standard_normal((n, 1, H, W)).astype(np.float32)
    want, _ = U.forward(U.weights_for_forward(params), x.astype(np.float64))
    xd = torch.tensor(x.ravel(), device="cuda")
    yd = torch.empty_like(xd)
    net.forward(xd, yd)
    torch.cuda.synchronize()
    got = yd.cpu().numpy().reshape(want.shape)
    assert np.max(np.abs(got - want)) <= 1e-4 * np.max(np.abs(want))
    net.close()


def _decision_margins(wts, x):
    """Smallest margin of the discrete decisions of the forward pass:
    |pre-activation| / (sum |w||x| + |b|) over every ReLU, and the relative gap
    between the two largest values of every max-pool window.  The gradients of
    the two sides can only agree where each decision is taken alike in float32
    and float64, i.e. where these margins are far above float32 rounding of
    the sums (at most K * 6e-8 for K <= 2304 terms)."""
    c = U.forward(wts, x)[1]
    inputs = {"enc1a": c["x"], "enc1b": c["enc1a"], "enc2a": c["p1"], "enc2b": c["enc2a"],
              "enc3a": c["p2"], "enc3b": c["enc3a"], "bota": c["p3"], "botb": c["bota"],
              "dec3a": c["c3"], "dec3b": c["dec3a"], "dec2a": c["c2"], "dec2b": c["dec2a"],
              "dec1a": c["c1"], "dec1b": c["dec1a"]}
    relu_min = np.inf
    for name, inp in inputs.items():
        w, b = wts[name]
        pre = U.conv3x3(inp, w, b)
        mag = U.conv3x3(np.abs(inp), np.abs(w), np.abs(b))
        relu_min = min(relu_min, np.min(np.abs(pre) / mag))
    pool_min = np.inf
    for name in ("enc1b", "enc2b", "enc3b"):
        e = c[name]
        n_, ch, h, w = e.shape
        win = np.sort(e.reshape(n_, ch, h // 2, 2, w // 2, 2).transpose(0, 1, 2, 4, 3, 5)
                      .reshape(n_, ch, h // 2, w // 2, 4), axis=-1)
        top = win[..., 3] > 0
        gap = (win[..., 3] - win[..., 2])[top] / win[..., 3][top]
        pool_min = min(pool_min, gap.min(initial=np.inf))
    return relu_min, pool_min


def test_gradients_and_adam_step_match_oracle(sl):
    # 8 x 8 (levels 8, 4, 2, 1) with weights seed 3: every ReLU and pooling
    # decision has a margin above 2e-5 (checked below), so both sides route
    # the gradient alike
    H = W = 8
    n = 1
    net, params = _net(sl, H, W, n, 3)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((n, 1, H, W)).astype(np.float32)
    t = (0.5 * rng.standard_normal((n, 1, H, W))).astype(np.float32)
    wts = U.weights_for_forward(params)
    relu_min, pool_min = _decision_margins(wts, x.astype(np.float64))
    assert relu_min > 2e-5 and pool_min > 1e-4, (relu_min, pool_min)
    y, cache = U.forward(wts, x.astype(np.float64))
    loss_o, dy = U.mse(y, t.astype(np.float64))
    g_o = U.backward(wts, cache, dy)
    xd = torch.tensor(x.ravel(), device="cuda")
    td = torch.tensor(t.ravel(), device="cuda")
    lr = 1e-3
    loss_g = net.train_step(xd, td, lr)
    assert abs(loss_g - loss_o) <= 1e-5 * loss_o
    g_g = sl.unflatten_params(net.get_grads())
    for name, _, _ in U.LAYERS:
        for which in (0, 1):
            a, b = g_g[name][which].astype(np.float64), g_o[name][which]
            assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-12, (name, which)
    # Adam: the first step moves each entry by lr * sign(g); compare where the
    # sign of the gradient is not decided by rounding
    p_o, _, _ = U.train_step(params, U.zero_state(params), x.astype(np.float64), t.astype(np.float64), lr)
    p_g = sl.unflatten_params(net.get_params())
    for name, _, _ in U.LAYERS:
        for which in (0, 1):
            go = g_o[name][which]
            clear = np.abs(go) > 1e-3 * np.max(np.abs(go))
            d = np.abs(p_g[name][which].astype(np.float64) - p_o[name][which].astype(np.float64))
            assert np.max(d[clear], initial=0.0) <= 1e-6, (name, which)
            assert np.max(d) <= 2.0 * lr + 1e-6
    net.close()


def test_training_reduces_loss(sl):
    H = W = 32
    n = 4
    net, _ = _net(sl, H, W, n, 8)
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.standard_normal(n * H * W).astype(np.float32), device="cuda")
    t = torch.tanh(x) * 0.5
    losses = [net.train_step(x, t, 1e-3) for _ in range(30)]
    assert losses[-1] < 0.3 * losses[0]
    net.close()


def test_backproject_data_matches_oracle(sl):
    N, V, D = 24, 18, 35
    g = joseph.Geometry(N, V, D)
    b = np.random.default_rng(4).standard_normal(g.m)
    s = sl.Slim(N, V, D, D, 2, 1e-2, 1)
    s.set_data(b)
    out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    s.backproject_data(out)
    want = joseph.full_matrix(g).T @ b
    assert np.max(np.abs(out.cpu().numpy() - want)) <= 1e-5 * np.max(np.abs(want))
    s.close()


def test_warm_start_uses_or_rejects_the_guess(sl):
    N, V, D = 32, 20, 47
    g = joseph.Geometry(N, V, D)
    A = joseph.full_matrix(g)
    net = sl.UNet(N, N)
    flat = np.zeros(net.nparams, dtype=np.float32)
    flat[-1] = 1.0                       # bias of the final 1x1 conv: the network outputs 1
    net.set_params(flat)
    s_out = 0.25
    for sign, want_used in ((1.0, True), (-1.0, False)):
        b = sign * (A @ np.full(g.n, s_out))
        s = sl.Slim(N, V, D, D, 2, 1e-2, 1)
        s.set_data(b)
        s.set_x(np.full(g.n, 7.0))
        used, ratio = s.warm_start(net, 1.0, s_out)
        x = s.get_x()
        assert used == want_used
        if want_used:
            assert ratio < 1e-6 and np.allclose(x, s_out)
        else:
            assert abs(ratio - 2.0) < 1e-9 and not x.any()
        s.close()
    net.close()
