"""The network's layers through the C ABI against the float64 oracle's layer
functions, at sizes that span several tiles of the tensor-core GEMM with
ragged edges in every dimension, one to 72 k-slabs, and split-K weight
gradients.

Bounds: each output is compared with the sum of the magnitudes of its terms
(the same contraction on |x|, |w|).  The forward pass and the input gradient
carry activations as three bfloat16 terms (float32 accuracy) and weights as
bfloat16 values, so they are held to 1e-5 of that magnitude; the weight
gradient multiplies two 2-term operands (2^-16 relative per product) and is
held to 1e-4 of it."""
import numpy as np
import pytest

from oracle import unet as U

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def sl():
    from paper_1912_07962_gb300 import build, slim
    build.build()
    return slim


def _dev(a):
    """NCHW (or any) float64 array -> contiguous float32 CUDA tensor."""
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _cnhw(a):
    return np.ascontiguousarray(a.transpose(1, 0, 2, 3))


def _nchw(t, shape_cnhw):
    return t.cpu().numpy().astype(np.float64).reshape(shape_cnhw).transpose(1, 0, 2, 3)


def _check(got, want, mag, rel, what):
    bad = np.abs(got - want) > rel * mag + 1e-30
    assert not bad.any(), (what, float(np.max(np.abs(got - want) / (mag + 1e-30))))


# (n, c_in, H, W, c_out): ragged in every dimension; one channel in (K = 9);
# the deepest layer's K = 2304 on a 6 x 10 grid; a level-1-like case whose
# weight gradient is split four ways
# channel counts that are multiples of 8 take the convolution from pre-split
# planes (forward: c_in; input gradient: c_out), the others the gathering
# kernel; (2, 24, 13, 21, 40) has both on the planes path with ragged output
# channels (40 of a 64-wide tile, 24 of 32) and K = 216 / 360, which end in
# part-filled 64-wide slices
CONV_CASES = [(3, 37, 20, 27, 70), (1, 1, 8, 8, 32), (1, 256, 6, 10, 256), (2, 32, 48, 48, 64),
              (2, 24, 13, 21, 40)]


@pytest.mark.parametrize("n,ci,H,W,co", CONV_CASES)
def test_conv3x3_forward_and_gradients(sl, n, ci, H, W, co):
    rng = np.random.default_rng(n * 1000 + ci)
    x = rng.standard_normal((n, ci, H, W))
    w = U.round_bf16(rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci)))
    b = 0.1 * rng.standard_normal(co)
    dy = rng.standard_normal((n, co, H, W))
    for relu in (0, 1):
        y = torch.empty(co * n * H * W, dtype=torch.float32, device="cuda")
        sl.unet_conv3x3(_dev(_cnhw(x)), n, ci, H, W, _dev(w), _dev(b), co, relu, y)
        torch.cuda.synchronize()
        pre = U.conv3x3(x, w, b)
        want = U.relu(pre) if relu else pre
        mag = U.conv3x3(np.abs(x), np.abs(w), np.abs(b))
        _check(_nchw(y, (co, n, H, W)), want, mag, 1e-5, ("forward", relu))
    dx_o, dw_o, db_o = U.conv3x3_backward(x, w, dy)
    dx_mag, dw_mag, db_mag = U.conv3x3_backward(np.abs(x), np.abs(w), np.abs(dy))
    dw0 = rng.standard_normal(w.shape)          # the gradients accumulate
    db0 = rng.standard_normal(co)
    dw = _dev(dw0)
    db = _dev(db0)
    dx = torch.full((ci * n * H * W,), np.nan, dtype=torch.float32, device="cuda")
    sl.unet_conv3x3_grad(_dev(_cnhw(x)), _dev(_cnhw(dy)), n, ci, H, W, _dev(w), co, dw, db, dx)
    torch.cuda.synchronize()
    _check(dw.cpu().numpy().astype(np.float64).reshape(w.shape) - dw0, dw_o, dw_mag, 1e-4, "dw")
    _check(db.cpu().numpy().astype(np.float64) - db0, db_o, db_mag, 1e-5, "db")
    _check(_nchw(dx, (ci, n, H, W)), dx_o, dx_mag, 1e-5, "dx")


# (n, c_in, H, W, c_out) of the input grid; the last case splits dW 3 ways
TCONV_CASES = [(3, 45, 7, 9, 38), (1, 256, 4, 4, 128), (2, 64, 40, 40, 32)]


@pytest.mark.parametrize("n,ci,H,W,co", TCONV_CASES)
def test_tconv2x2_forward_and_gradients(sl, n, ci, H, W, co):
    rng = np.random.default_rng(7 * n + ci)
    x = rng.standard_normal((n, ci, H, W))
    w = U.round_bf16(rng.standard_normal((ci, co, 2, 2)) * np.sqrt(1.0 / ci))
    b = 0.1 * rng.standard_normal(co)
    dy = rng.standard_normal((n, co, 2 * H, 2 * W))
    y = torch.full((co * n * 4 * H * W,), np.nan, dtype=torch.float32, device="cuda")
    sl.unet_tconv2x2(_dev(_cnhw(x)), n, ci, H, W, _dev(w), _dev(b), co, y)
    torch.cuda.synchronize()
    want = U.tconv2x2(x, w, b)
    mag = U.tconv2x2(np.abs(x), np.abs(w), np.abs(b))
    _check(_nchw(y, (co, n, 2 * H, 2 * W)), want, mag, 1e-5, "forward")
    dx_o, dw_o, db_o = U.tconv2x2_backward(x, w, dy)
    dx_mag, dw_mag, db_mag = U.tconv2x2_backward(np.abs(x), np.abs(w), np.abs(dy))
    dw0 = rng.standard_normal(w.shape)
    dw = _dev(dw0)
    db = torch.zeros(co, dtype=torch.float32, device="cuda")
    dx = torch.full((ci * n * H * W,), np.nan, dtype=torch.float32, device="cuda")
    sl.unet_tconv2x2_grad(_dev(_cnhw(x)), _dev(_cnhw(dy)), n, ci, H, W, _dev(w), co, dw, db, dx)
    torch.cuda.synchronize()
    _check(dw.cpu().numpy().astype(np.float64).reshape(w.shape) - dw0, dw_o, dw_mag, 1e-4, "dw")
    _check(db.cpu().numpy().astype(np.float64), db_o, db_mag, 1e-5, "db")
    _check(_nchw(dx, (ci, n, H, W)), dx_o, dx_mag, 1e-5, "dx")


def test_weights_are_read_as_bfloat16(sl):
    # a weight halfway between two bfloat16 values goes to the even one
    n, ci, H, W, co = 1, 1, 8, 8, 1
    x = np.zeros((n, ci, H, W))
    x[0, 0, 4, 4] = 1.0
    w = np.zeros((co, ci, 3, 3))
    w[0, 0, 1, 1] = 1.0 + 2.0 ** -8             # tie: rounds to 1.0
    y = torch.empty(H * W, dtype=torch.float32, device="cuda")
    sl.unet_conv3x3(_dev(x), n, ci, H, W, _dev(w), None, co, 0, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().reshape(H, W)
    assert got[4, 4] == 1.0 and np.count_nonzero(got) == 1


def test_dx_skipped_when_null(sl):
    n, ci, H, W, co = 1, 4, 8, 8, 8
    rng = np.random.default_rng(5)
    x = _dev(rng.standard_normal(ci * n * H * W))
    dy = _dev(rng.standard_normal(co * n * H * W))
    w = _dev(U.round_bf16(rng.standard_normal(co * ci * 9)))
    dw = torch.zeros(co * ci * 9, dtype=torch.float32, device="cuda")
    sl.unet_conv3x3_grad(x, dy, n, ci, H, W, w, co, dw, None, None)
    torch.cuda.synchronize()
    assert torch.count_nonzero(dw).item() > 0
