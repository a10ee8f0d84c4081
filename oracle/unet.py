"""U-Net that maps A^T b to an initial guess x_0 (the learned warm start).

Test infrastructure: the float64 oracle of the network, its gradients and its
optimiser.  Nothing outside tests/, the smoke check and the bench's CPU leg
imports this module.

The paper starts its iterations from x_0 = 0 (Sec. 4); a learned x_0 is an
extension beyond the paper, not one of its methods.  Architecture:
  encoder  three levels of [conv3x3 + ReLU, conv3x3 + ReLU] with 32, 64, 128
           channels, each followed by a 2x2 max-pool;
  bottom   [conv3x3 + ReLU] x 2 with 256 channels;
  decoder  three levels of [2x2 stride-2 transposed conv, concatenation with
           the encoder output of that level (upsampled channels first), then
           conv3x3 + ReLU twice] with 128, 64, 32 channels;
  output   1x1 conv to one channel.
Tensors are NCHW.  The forward pass uses weights rounded to bfloat16 from a
float32 master copy (round to nearest even); Adam (Kingma and Ba, 2015)
updates the master copy.  Everything here computes in float64.

Layer definitions (zero padding for the 3x3 convolution):
  conv3x3    y[n,o,i,j] = b[o] + sum_{c,u,v} w[o,c,u,v] x[n,c,i+u-1,j+v-1]
  tconv2x2   y[n,o,2i+u,2j+v] = b[o] + sum_c w[c,o,u,v] x[n,c,i,j]
  maxpool2   y[n,c,i,j] = max of x[n,c,2i:2i+2,2j:2j+2]; the gradient goes to
             the first maximum in row-major order of the window
  conv1x1    y[n,o,i,j] = b[o] + sum_c w[o,c] x[n,c,i,j]
  loss       mean of (y - t)^2 over all elements
"""
from __future__ import annotations

import numpy as np

# (name, weight shape, kind); biases have the output-channel count
LAYERS = [
    ("enc1a", (32, 1, 3, 3), "conv"), ("enc1b", (32, 32, 3, 3), "conv"),
    ("enc2a", (64, 32, 3, 3), "conv"), ("enc2b", (64, 64, 3, 3), "conv"),
    ("enc3a", (128, 64, 3, 3), "conv"), ("enc3b", (128, 128, 3, 3), "conv"),
    ("bota", (256, 128, 3, 3), "conv"), ("botb", (256, 256, 3, 3), "conv"),
    ("up3", (256, 128, 2, 2), "tconv"),
    ("dec3a", (128, 256, 3, 3), "conv"), ("dec3b", (128, 128, 3, 3), "conv"),
    ("up2", (128, 64, 2, 2), "tconv"),
    ("dec2a", (64, 128, 3, 3), "conv"), ("dec2b", (64, 64, 3, 3), "conv"),
    ("up1", (64, 32, 2, 2), "tconv"),
    ("dec1a", (32, 64, 3, 3), "conv"), ("dec1b", (32, 32, 3, 3), "conv"),
    ("out", (1, 32), "conv1x1"),
]


def bias_size(shape, kind):
    return shape[1] if kind == "tconv" else shape[0]


def param_count():
    return sum(int(np.prod(s)) + bias_size(s, k) for _, s, k in LAYERS)


def round_bf16(a) -> np.ndarray:
    """float32 values rounded to bfloat16 (nearest, ties to even), as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# Layers
# ---------------------------------------------------------------------------
def conv3x3(x, w, b):
    n, c, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((n, w.shape[0], h, wd))
    for u in range(3):
        for v in range(3):
            y += np.einsum("nchw,oc->nohw", xp[:, :, u:u + h, v:v + wd], w[:, :, u, v])
    return y + b[None, :, None, None]


def conv3x3_backward(x, w, dy):
    n, c, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w, dtype=np.float64)
    for u in range(3):
        for v in range(3):
            dxp[:, :, u:u + h, v:v + wd] += np.einsum("nohw,oc->nchw", dy, w[:, :, u, v])
            dw[:, :, u, v] = np.einsum("nohw,nchw->oc", dy, xp[:, :, u:u + h, v:v + wd])
    return dxp[:, :, 1:h + 1, 1:wd + 1], dw, dy.sum(axis=(0, 2, 3))


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(y, dy):
    """Gradient through ReLU given its output y."""
    return dy * (y > 0.0)


def maxpool2(x):
    n, c, h, wd = x.shape
    win = x.reshape(n, c, h // 2, 2, wd // 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(
        n, c, h // 2, wd // 2, 4)
    arg = np.argmax(win, axis=-1)          # first maximum in row-major window order
    return np.take_along_axis(win, arg[..., None], axis=-1)[..., 0], arg


def maxpool2_backward(arg, dy):
    n, c, h2, w2 = dy.shape
    win = np.zeros((n, c, h2, w2, 4))
    np.put_along_axis(win, arg[..., None], dy[..., None], axis=-1)
    return win.reshape(n, c, h2, w2, 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(n, c, 2 * h2, 2 * w2)


def tconv2x2(x, w, b):
    n, c, h, wd = x.shape
    y = np.zeros((n, w.shape[1], 2 * h, 2 * wd))
    for u in range(2):
        for v in range(2):
            y[:, :, u::2, v::2] = np.einsum("nchw,co->nohw", x, w[:, :, u, v])
    return y + b[None, :, None, None]


def tconv2x2_backward(x, w, dy):
    dx = np.zeros_like(x, dtype=np.float64)
    dw = np.zeros_like(w, dtype=np.float64)
    for u in range(2):
        for v in range(2):
            d = dy[:, :, u::2, v::2]
            dx += np.einsum("nohw,co->nchw", d, w[:, :, u, v])
            dw[:, :, u, v] = np.einsum("nchw,nohw->co", x, d)
    return dx, dw, dy.sum(axis=(0, 2, 3))


def conv1x1(x, w, b):
    return np.einsum("nchw,oc->nohw", x, w) + b[None, :, None, None]


def conv1x1_backward(x, w, dy):
    return (np.einsum("nohw,oc->nchw", dy, w), np.einsum("nohw,nchw->oc", dy, x),
            dy.sum(axis=(0, 2, 3)))


def mse(y, t):
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) at step t >= 1; returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# Network
# ---------------------------------------------------------------------------
def weights_for_forward(params):
    """bfloat16-rounded weights (float64) from the float32 master copy; biases
    stay float32."""
    return {k: (round_bf16(w), np.asarray(b, dtype=np.float32).astype(np.float64))
            for k, (w, b) in params.items()}


def forward(wts, x):
    """y = U-Net(x) and the activations the backward pass needs."""
    c = {"x": x}

    def block(name_a, name_b, inp):
        a = relu(conv3x3(inp, *wts[name_a]))
        bb = relu(conv3x3(a, *wts[name_b]))
        c[name_a], c[name_b] = a, bb
        return bb

    e1 = block("enc1a", "enc1b", x)
    p1, c["arg1"] = maxpool2(e1)
    e2 = block("enc2a", "enc2b", p1)
    p2, c["arg2"] = maxpool2(e2)
    e3 = block("enc3a", "enc3b", p2)
    p3, c["arg3"] = maxpool2(e3)
    c["p1"], c["p2"], c["p3"] = p1, p2, p3
    bt = block("bota", "botb", p3)
    c3 = np.concatenate([tconv2x2(bt, *wts["up3"]), e3], axis=1)
    d3 = block("dec3a", "dec3b", c3)
    c2 = np.concatenate([tconv2x2(d3, *wts["up2"]), e2], axis=1)
    d2 = block("dec2a", "dec2b", c2)
    c1 = np.concatenate([tconv2x2(d2, *wts["up1"]), e1], axis=1)
    d1 = block("dec1a", "dec1b", c1)
    c["c3"], c["c2"], c["c1"] = c3, c2, c1
    y = conv1x1(d1, *wts["out"])
    return y, c


def backward(wts, c, dy):
    """Gradients of sum(dy * y) with respect to every weight and bias."""
    g = {}

    def block_back(name_a, name_b, inp, d):
        d = relu_backward(c[name_b], d)
        da, g_w, g_b = conv3x3_backward(c[name_a], wts[name_b][0], d)
        g[name_b] = (g_w, g_b)
        da = relu_backward(c[name_a], da)
        dx, g_w, g_b = conv3x3_backward(inp, wts[name_a][0], da)
        g[name_a] = (g_w, g_b)
        return dx

    dd1, g_w, g_b = conv1x1_backward(c["dec1b"], wts["out"][0], dy)
    g["out"] = (g_w, g_b)
    dc1 = block_back("dec1a", "dec1b", c["c1"], dd1)
    de1 = dc1[:, 32:]
    dd2, g_w, g_b = tconv2x2_backward(c["dec2b"], wts["up1"][0], dc1[:, :32])
    g["up1"] = (g_w, g_b)
    dc2 = block_back("dec2a", "dec2b", c["c2"], dd2)
    de2 = dc2[:, 64:]
    dd3, g_w, g_b = tconv2x2_backward(c["dec3b"], wts["up2"][0], dc2[:, :64])
    g["up2"] = (g_w, g_b)
    dc3 = block_back("dec3a", "dec3b", c["c3"], dd3)
    de3 = dc3[:, 128:]
    dbt, g_w, g_b = tconv2x2_backward(c["botb"], wts["up3"][0], dc3[:, :128])
    g["up3"] = (g_w, g_b)
    dp3 = block_back("bota", "botb", c["p3"], dbt)
    de3 = de3 + maxpool2_backward(c["arg3"], dp3)
    dp2 = block_back("enc3a", "enc3b", c["p2"], de3)
    de2 = de2 + maxpool2_backward(c["arg2"], dp2)
    dp1 = block_back("enc2a", "enc2b", c["p1"], de2)
    de1 = de1 + maxpool2_backward(c["arg1"], dp1)
    block_back("enc1a", "enc1b", c["x"], de1)
    return g


def train_step(params, state, x, target, lr):
    """Forward with bf16 weights, MSE loss, backward, Adam on the float32
    master copy.  params: {name: (w, b)} float32; state: {"t": int, "m": .., "v": ..}.
    Returns (params, state, loss) with float32 master values."""
    wts = weights_for_forward(params)
    y, c = forward(wts, x)
    loss, dy = mse(y, target)
    g = backward(wts, c, dy)
    t = state["t"] + 1
    out_p, m_new, v_new = {}, {}, {}
    for name, (w, b) in params.items():
        gw, gb = g[name]
        mw, mb = state["m"][name]
        vw, vb = state["v"][name]
        w2, mw2, vw2 = adam(np.asarray(w, np.float64), gw, mw, vw, t, lr)
        b2, mb2, vb2 = adam(np.asarray(b, np.float64), gb, mb, vb, t, lr)
        out_p[name] = (w2.astype(np.float32), b2.astype(np.float32))
        m_new[name] = (mw2, mb2)
        v_new[name] = (vw2, vb2)
    return out_p, {"t": t, "m": m_new, "v": v_new}, loss


def zero_state(params):
    z = {k: (np.zeros(w.shape), np.zeros(b.shape)) for k, (w, b) in params.items()}
    return {"t": 0, "m": z, "v": {k: (a.copy(), b.copy()) for k, (a, b) in z.items()}}
