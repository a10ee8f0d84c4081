"""Pins of the warm-start network oracle: brute-force layers on tiny inputs,
adjoint identities, central finite differences, closed forms of the loss and
of the first Adam step."""
import numpy as np
import pytest

import workloads
from oracle import unet as U

RNG = np.random.default_rng(12345)


def test_round_bf16_ties_and_carry():
    one = np.float32(1.0)
    half_ulp = np.float32(1.0 + 2.0 ** -8)        # exactly between 1 and 1 + 2^-7
    above = np.float32(1.0 + 3 * 2.0 ** -8)        # between 1 + 2^-7 and 1 + 2^-6: tie -> even
    got = U.round_bf16(np.array([one, half_ulp, above, -half_ulp, np.float32(3.0)]))
    assert got.tolist() == [1.0, 1.0, 1.0 + 2.0 ** -6, -1.0, 3.0]
    # carry into the exponent: the largest value below 2 rounds up to 2
    assert U.round_bf16(np.array([np.float32(2.0 - 2.0 ** -23)]))[0] == 2.0


def _conv_brute(x, w, b):
    n, c, h, wd = x.shape
    o = w.shape[0]
    y = np.zeros((n, o, h, wd))
    for a in range(n):
        for oo in range(o):
            for i in range(h):
                for j in range(wd):
                    s = b[oo]
                    for cc in range(c):
                        for u in range(3):
                            for v in range(3):
                                ii, jj = i + u - 1, j + v - 1
                                if 0 <= ii < h and 0 <= jj < wd:
                                    s += w[oo, cc, u, v] * x[a, cc, ii, jj]
                    y[a, oo, i, j] = s
    return y


def test_conv3x3_matches_brute_force_and_delta_kernel():
    x = RNG.standard_normal((2, 2, 4, 5))
    w = RNG.standard_normal((3, 2, 3, 3))
    b = RNG.standard_normal(3)
    assert np.allclose(U.conv3x3(x, w, b), _conv_brute(x, w, b), rtol=0, atol=1e-12)
    d = np.zeros((2, 2, 3, 3))
    d[0, 0, 1, 1] = d[1, 1, 1, 1] = 1.0
    assert np.array_equal(U.conv3x3(x, d, np.zeros(2)), x)
    # a kernel tap at (0, 0) reads the pixel up-left: shift down-right with zero fill
    s = np.zeros((1, 1, 3, 3))
    s[0, 0, 0, 0] = 1.0
    y = U.conv3x3(x[:, :1], s, np.zeros(1))
    assert np.array_equal(y[:, :, 1:, 1:], x[:, :1, :-1, :-1]) and not y[:, :, 0, :].any()


def _directional(f, x, d, eps=1e-6):
    return (f(x + eps * d) - f(x - eps * d)) / (2 * eps)


def test_conv3x3_backward_finite_differences():
    x = RNG.standard_normal((2, 3, 5, 4))
    w = RNG.standard_normal((4, 3, 3, 3))
    b = RNG.standard_normal(4)
    dy = RNG.standard_normal((2, 4, 5, 4))
    dx, dw, db = U.conv3x3_backward(x, w, dy)
    for arg, grad, f in ((x, dx, lambda t: np.sum(dy * U.conv3x3(t, w, b))),
                         (w, dw, lambda t: np.sum(dy * U.conv3x3(x, t, b))),
                         (b, db, lambda t: np.sum(dy * U.conv3x3(x, w, t)))):
        d = RNG.standard_normal(arg.shape)
        assert abs(_directional(f, arg, d) - np.sum(grad * d)) <= 1e-6 * max(1.0, abs(np.sum(grad * d)))


def test_maxpool_values_ties_and_backward():
    x = np.array([[[[1., 5., 2., 2.], [3., 4., 2., 2.], [0., -1., 7., 1.], [-2., -3., 7., 0.]]]])
    y, arg = U.maxpool2(x)
    assert y[0, 0].tolist() == [[5., 2.], [0., 7.]]
    assert arg[0, 0].tolist() == [[1, 0], [0, 0]]          # ties: first in row-major order
    dx = U.maxpool2_backward(arg, np.array([[[[1., 2.], [3., 4.]]]]))
    want = np.zeros((4, 4))
    want[0, 1], want[0, 2], want[2, 0], want[2, 2] = 1., 2., 3., 4.
    assert np.array_equal(dx[0, 0], want)


def test_tconv2x2_brute_force_and_adjoint():
    x = RNG.standard_normal((2, 3, 3, 2))
    w = RNG.standard_normal((3, 4, 2, 2))
    b = RNG.standard_normal(4)
    y = U.tconv2x2(x, w, b)
    brute = np.zeros((2, 4, 6, 4))
    for n in range(2):
        for o in range(4):
            for i in range(6):
                for j in range(4):
                    brute[n, o, i, j] = b[o] + sum(w[c, o, i % 2, j % 2] * x[n, c, i // 2, j // 2]
                                                   for c in range(3))
    assert np.allclose(y, brute, rtol=0, atol=1e-12)
    dy = RNG.standard_normal(y.shape)
    dx, dw, db = U.tconv2x2_backward(x, w, dy)
    # adjoint: <T x, dy> = <x, T^* dy> for the bias-free map
    assert np.isclose(np.sum(U.tconv2x2(x, w, np.zeros(4)) * dy), np.sum(x * dx), rtol=1e-12)
    d = RNG.standard_normal(w.shape)
    f = lambda t: np.sum(dy * U.tconv2x2(x, t, b))
    assert abs(_directional(f, w, d) - np.sum(dw * d)) <= 1e-6 * max(1.0, abs(np.sum(dw * d)))
    assert np.allclose(db, dy.sum(axis=(0, 2, 3)))


def test_conv1x1_and_mse():
    x = RNG.standard_normal((2, 3, 2, 2))
    w = RNG.standard_normal((1, 3))
    b = np.array([0.5])
    y = U.conv1x1(x, w, b)
    assert np.allclose(y[:, 0], 0.5 + sum(w[0, c] * x[:, c] for c in range(3)))
    t = RNG.standard_normal(y.shape)
    loss, g = U.mse(y, t)
    assert np.isclose(loss, np.mean((y - t) ** 2)) and np.allclose(g, 2 * (y - t) / y.size)
    dy = RNG.standard_normal(y.shape)
    dx, dw, db = U.conv1x1_backward(x, w, dy)
    d = RNG.standard_normal(x.shape)
    f = lambda s: np.sum(dy * U.conv1x1(s, w, b))
    assert abs(_directional(f, x, d) - np.sum(dx * d)) < 1e-7


def test_adam_first_step_and_quadratic():
    g = np.array([3.0, -0.5, 1e-3])
    p, m, v = U.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=0.0)
    assert np.allclose(p, -0.1 * np.sign(g))           # m_hat / sqrt(v_hat) = sign(g) at t = 1
    # minimises a convex quadratic
    A = np.diag([1.0, 10.0])
    p, m, v = np.array([1.0, 1.0]), np.zeros(2), np.zeros(2)
    for t in range(1, 3001):
        p, m, v = U.adam(p, A @ p, m, v, t, lr=0.01)
    assert np.linalg.norm(p) < 1e-3


def test_parameter_count():
    # weights 1,923,392 (summed by hand over the 18 layers) + biases 1,633
    assert U.param_count() == 1925025


def test_network_gradient_finite_differences():
    params = workloads.unet_init(7, U.LAYERS)
    wts = {k: (np.asarray(w, np.float64), np.asarray(b, np.float64) + 0.01)
           for k, (w, b) in params.items()}
    x = RNG.standard_normal((1, 1, 8, 8))
    y, c = U.forward(wts, x)
    assert y.shape == (1, 1, 8, 8)
    dy = RNG.standard_normal(y.shape)
    g = U.backward(wts, c, dy)
    for name in ("enc1a", "enc3b", "botb", "up3", "dec2a", "up1", "dec1b", "out"):
        w, b = wts[name]
        for which, arr in ((0, w), (1, b)):
            e = tuple(int(RNG.integers(0, s)) for s in arr.shape)
            eps = 1e-6

            def loss(delta):
                a = arr.copy()
                a[e] += delta
                ww = dict(wts)
                ww[name] = (a, b) if which == 0 else (w, a)
                return float(np.sum(dy * U.forward(ww, x)[0]))

            fd = (loss(eps) - loss(-eps)) / (2 * eps)
            an = g[name][which][e]
            assert abs(fd - an) <= 1e-5 * max(1e-3, abs(an)), (name, which, e, fd, an)


def test_train_step_reduces_loss():
    params = workloads.unet_init(3, U.LAYERS)
    state = U.zero_state(params)
    x = RNG.standard_normal((2, 1, 8, 8))
    t = np.tanh(x)
    losses = []
    for _ in range(12):
        params, state, loss = U.train_step(params, state, x, t, lr=1e-3)
        losses.append(loss)
    assert losses[-1] < 0.5 * losses[0]
    assert all(w.dtype == np.float32 for w, _ in params.values())
