"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module produces *inputs only*: phantoms (x_true), standard-normal noise
directions, the paper's small Gaussian test matrix, and the parameter sets of
the tomography workloads.  It holds none of the method's arithmetic: no
projector, no sampling of blocks, no step of the iteration.  Both the CUDA
library and the CPU oracle consume what it returns.

Phantoms stand in for the data the paper reconstructs (a walnut slice, Sec. 4.3,
and a modified 3D Shepp-Logan volume, Sec. 4.3), which are not available: they
are sums of random uniform ellipses (2D) or ellipsoids (3D) on [-1, 1]^d, sampled
at pixel centres.

The noise model is the paper's (Sec. 4.1): b = A x_true + eps with
||eps||_2 / ||A x_true||_2 equal to the noise level; `add_noise` composes that
from a clean projection and a standard-normal direction drawn here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Random streams: one numpy Generator per (seed, stream) pair.
STREAM_PHANTOM = 0
STREAM_NOISE = 1
STREAM_META = 4


def _gen(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


# --------------------------------------------------------------------------
# Phantoms
# --------------------------------------------------------------------------
def ellipse_params_2d(seed: int, count: int = 10) -> np.ndarray:
    """Rows (cx, cy, a, b, phi, rho): centres U(-0.7,0.7), semi-axes U(0.05,0.5),
    rotation U(0,pi), intensity U(0,1), drawn in that order per ellipse."""
    g = _gen(seed, STREAM_PHANTOM)
    out = np.empty((count, 6))
    for e in range(count):
        out[e, 0] = g.uniform(-0.7, 0.7)
        out[e, 1] = g.uniform(-0.7, 0.7)
        out[e, 2] = g.uniform(0.05, 0.5)
        out[e, 3] = g.uniform(0.05, 0.5)
        out[e, 4] = g.uniform(0.0, math.pi)
        out[e, 5] = g.uniform(0.0, 1.0)
    return out


def rasterize_ellipses_2d(N: int, params: np.ndarray) -> np.ndarray:
    """Sum of ellipse intensities at pixel centres; x[iy*N + ix], float64.

    Pixel (ix, iy) sits at normalised coordinates X = (ix-c)/(N/2),
    Y = (iy-c)/(N/2) with c = (N-1)/2.
    """
    c = (N - 1) / 2.0
    coords = (np.arange(N) - c) / (N / 2.0)
    X = coords[None, :]
    Y = coords[:, None]
    img = np.zeros((N, N))
    for cx, cy, a, b, phi, rho in params:
        Xp = X - cx
        Yp = Y - cy
        u = (Xp * math.cos(phi) + Yp * math.sin(phi)) / a
        v = (-Xp * math.sin(phi) + Yp * math.cos(phi)) / b
        img += rho * ((u * u + v * v) <= 1.0)
    return img.reshape(-1)


def phantom_2d(N: int, seed: int, count: int = 10) -> np.ndarray:
    """Seeded random-ellipse phantom of side N (n = N^2 pixels), float64."""
    return rasterize_ellipses_2d(N, ellipse_params_2d(seed, count))


def ellipsoid_params_3d(seed: int, count: int = 20) -> np.ndarray:
    """Rows (cx, cy, cz, a, b, c, q0, q1, q2, q3, rho): centres U(-0.7,0.7)^3,
    semi-axes U(0.05,0.5)^3, orientation from a normalised Gaussian quaternion,
    intensity U(0,1)."""
    g = _gen(seed, STREAM_PHANTOM)
    out = np.empty((count, 11))
    for e in range(count):
        out[e, 0:3] = g.uniform(-0.7, 0.7, size=3)
        out[e, 3:6] = g.uniform(0.05, 0.5, size=3)
        q = g.standard_normal(4)
        out[e, 6:10] = q / np.linalg.norm(q)
        out[e, 10] = g.uniform(0.0, 1.0)
    return out


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def phantom_3d(N: int, seed: int, count: int = 20, dtype=np.float64) -> np.ndarray:
    """Seeded random-ellipsoid volume of side N; x[(iz*N + iy)*N + ix]."""
    c = (N - 1) / 2.0
    coords = (np.arange(N) - c) / (N / 2.0)
    vol = np.zeros((N, N, N), dtype=dtype)  # [iz, iy, ix]
    for row in ellipsoid_params_3d(seed, count):
        cen, ax, q, rho = row[0:3], row[3:6], row[6:10], row[10]
        R = _quat_to_rot(q)
        rad = float(ax.max())
        # bounding box in index space (the ellipsoid lies in the ball of radius max axis)
        lo = [max(0, int(math.floor((cen[d] - rad) * (N / 2.0) + c))) for d in range(3)]
        hi = [min(N - 1, int(math.ceil((cen[d] + rad) * (N / 2.0) + c))) for d in range(3)]
        if any(lo[d] > hi[d] for d in range(3)):
            continue
        xs = coords[lo[0]:hi[0] + 1] - cen[0]
        ys = coords[lo[1]:hi[1] + 1] - cen[1]
        zs = coords[lo[2]:hi[2] + 1] - cen[2]
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        # body-frame coordinates: R^T (p - centre)
        u = (R[0, 0] * X + R[1, 0] * Y + R[2, 0] * Z) / ax[0]
        v = (R[0, 1] * X + R[1, 1] * Y + R[2, 1] * Z) / ax[1]
        w = (R[0, 2] * X + R[1, 2] * Y + R[2, 2] * Z) / ax[2]
        inside = (u * u + v * v + w * w) <= 1.0
        vol[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += (rho * inside).astype(dtype)
    return vol.reshape(-1)


# --------------------------------------------------------------------------
# Noise
# --------------------------------------------------------------------------
def noise_direction(m: int, seed: int) -> np.ndarray:
    """Standard-normal vector e ~ N(0, I_m), float64."""
    return _gen(seed, STREAM_NOISE).standard_normal(m)


def add_noise(clean: np.ndarray, e: np.ndarray, level: float) -> np.ndarray:
    """b = clean + level * ||clean|| * e / ||e||  (noise level as in Sec. 4.1)."""
    clean = np.asarray(clean, dtype=np.float64)
    return clean + level * np.linalg.norm(clean) * (e / np.linalg.norm(e))


# --------------------------------------------------------------------------
# The paper's illustrative Gaussian example (Sec. 4.1)
# --------------------------------------------------------------------------
def gaussian_problem(seed: int, m: int = 1000, n: int = 100, level: float = 0.01):
    """A ~ N(0,1)^{m x n}, x_true = 1, 1% white noise.  Returns (A, x_true, b)."""
    g = _gen(seed, STREAM_PHANTOM)
    A = g.standard_normal((m, n))
    x_true = np.ones(n)
    b = add_noise(A @ x_true, noise_direction(m, seed), level)
    return A, x_true, b


# --------------------------------------------------------------------------
# Workload parameter sets
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Tomo2D:
    name: str
    N: int              # image side, n = N^2
    n_views: int        # angles uniform in [0, pi)
    det: int            # detector bins per view at unit spacing
    ell: int            # rows per block
    r: int              # memory
    lam: float          # damping lambda = 1/alpha
    seed: int
    epochs: int = 20
    noise: float = 0.01
    n_ellipses: int = 10

    @property
    def n(self) -> int:
        return self.N * self.N

    @property
    def m(self) -> int:
        return self.n_views * self.det

    @property
    def p(self) -> int:
        return (self.r + 1) * self.ell


# 64x64 image, 60 angles x 91 bins, one view per block, r=3, lambda=1e-2, 20 epochs.
C1 = Tomo2D("plain-fp64-64x64", N=64, n_views=60, det=91, ell=91, r=3, lam=1e-2, seed=1)
# 256x256 image, 180 angles x 363 bins, one view per block, r=5, lambda=1e-3.
C2 = Tomo2D("precision-256x256", N=256, n_views=180, det=363, ell=363, r=5, lam=1e-3, seed=2)


def tomo_inputs_2d(cfg: Tomo2D):
    """(x_true, e) for a 2D workload: phantom and the noise direction."""
    return phantom_2d(cfg.N, cfg.seed, cfg.n_ellipses), noise_direction(cfg.m, cfg.seed)


@dataclasses.dataclass
class Tomo3D:
    name: str
    N: int
    n_views: int
    det_u: int
    det_v: int
    ell: int
    r: int
    lam: float
    seed: int
    noise: float = 0.01
    n_ellipsoids: int = 20

    @property
    def n(self) -> int:
        return self.N ** 3

    @property
    def m(self) -> int:
        return self.n_views * self.det_u * self.det_v


# 256^3 volume, 360 views on a 256 (rows) x 368 (columns) detector, l=2048 random rays, r=4.
C4 = Tomo3D("streaming-256^3", N=256, n_views=360, det_u=368, det_v=256, ell=2048, r=4,
            lam=1e-3, seed=4)

STREAM_FRAMES = 6


def random_frames(n_views: int, seed: int) -> np.ndarray:
    """View frames of the random-direction 3D geometry (Sec. 4.3: projection
    images taken from directions uniform on the unit sphere).  Rows
    (d, u, v), 9 float64 values each: d a normalised standard-normal 3-vector;
    u, v an orthonormal detector basis perpendicular to d: u from the
    coordinate axis least aligned with d by one Gram-Schmidt step, v = d x u."""
    g = _gen(seed, STREAM_FRAMES)
    out = np.empty((n_views, 9))
    for a in range(n_views):
        d = g.standard_normal(3)
        d /= np.linalg.norm(d)
        e = np.zeros(3)
        e[int(np.argmin(np.abs(d)))] = 1.0
        u = e - (e @ d) * d
        u /= np.linalg.norm(u)
        v = np.cross(d, u)
        out[a] = np.concatenate([d, u, v])
    return out


# The 3D geometry of Sec. 4.3 (random directions) at 256^3: 360 random view
# directions on a 368 x 368 detector (the cube's shadow is up to 443 wide; the
# corners are clipped), l = 2048 random rays from the arrived views, r = 4.
C4R = Tomo3D("random-directions-256^3", N=256, n_views=360, det_u=368, det_v=368, ell=2048,
             r=4, lam=1e-3, seed=5)


def batch_mix(count: int = 96, meta_seed: int = 3):
    """Parameters of the batched workload: per problem (N, n_views, det, ell, r, lam, seed).

    Sides from {128,192,256,384,512}, views U{90..360}, bins ceil(sqrt(2)*N),
    ell U{128..512}, r U{2..8}, lambda log-uniform in [1e-4, 1e-2]."""
    g = _gen(meta_seed, STREAM_META)
    sides = [128, 192, 256, 384, 512]
    out = []
    for i in range(count):
        N = sides[int(g.integers(0, len(sides)))]
        views = int(g.integers(90, 361))
        det = int(math.ceil(math.sqrt(2.0) * N))
        ell = int(g.integers(128, 513))
        r = int(g.integers(2, 9))
        lam = float(10.0 ** g.uniform(-4.0, -2.0))
        out.append(Tomo2D(f"batch-{i}", N=N, n_views=views, det=det, ell=ell, r=r, lam=lam,
                          seed=1000 + i))
    return out


# ---------------------------------------------------------------------------
# Warm-start network: initial weights and the train / held-out seeds
# ---------------------------------------------------------------------------
STREAM_NET = 5
WARM_TRAIN_SEEDS = range(10000, 12000)     # 2000 training phantoms
WARM_TEST_SEEDS = range(20000, 20200)      # 200 held-out phantoms


def unet_init(seed: int, layers):
    """Initial float32 weights of the warm-start U-Net: He-normal (standard
    deviation sqrt(2 / fan_in)), zero biases.  `layers` is a list of
    (name, weight shape, kind) in the network's order; kind "tconv" has its
    output channels second and fan_in = in_channels * 4."""
    g = _gen(seed, STREAM_NET)
    out = {}
    for name, shape, kind in layers:
        if kind == "tconv":
            fan_in, nb = shape[0] * shape[2] * shape[3], shape[1]
        else:
            fan_in, nb = int(np.prod(shape[1:])), shape[0]
        w = (g.standard_normal(shape) * math.sqrt(2.0 / fan_in)).astype(np.float32)
        out[name] = (w, np.zeros(nb, dtype=np.float32))
    return out
