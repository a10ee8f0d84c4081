"""Joseph ray-driven rows of the parallel-beam forward model A (oracle side).

The paper's tomography experiments use parallel-beam rays (Sec. 4.3) whose
blocks are one projection image each and whose rows are generated rather than
stored (Sec. 4.2: "function evaluations can be used").  The paper names no
projector; this is Joseph's method (P. M. Joseph, IEEE TMI 1(3), 1982): march
the ray one pixel row (or column) at a time along its dominant axis and
interpolate linearly between the two nearest pixel centres on that row, each
tap weighted by the path length per step.

Definition (float64, every operation rounded once; no fused multiply-add):

  2D image, N x N, x[iy*N + ix]; pixel centre (ix - cc, iy - cc), cc = (N-1)/2.
  View a: theta_a = a*pi/A_v unless angles are given; co = cos(theta), si = sin(theta)
  (host libm, shared as data).  Bin d: t = d - (D-1)/2.  Ray = {p : p.(co, si) = t}.
  Row-stepping iff |co| >= |si|, with rc = 1/co; else column-stepping with rc = 1/si.
  ia = |rc| is the path length per step.
  Row-stepping, for iy = 0..N-1:
      y  = iy - cc;  u = t - y*si;  fx = u*rc + cc
      j0 = floor(fx);  w1 = fx - j0
      tap (j0,   iy) weight (1 - w1)*ia;   tap (j0+1, iy) weight w1*ia
  Column-stepping is the same with (x, co) and (y, si) exchanged:
      xx = ix - cc;  u = t - xx*co;  fy = u*rc + cc;  i0 = floor(fy); ...
  Taps outside [0, N-1] and taps of weight exactly 0 are dropped.

  3D volume N^3, x[(iz*N + iy)*N + ix]; views rotate about z; detector column
  uu (t = uu - (Du-1)/2) and row v (z_v = v - (Dv-1)/2).  The in-plane march is
  the 2D one; along z, fz = z_v + cc, k0 = floor(fz), wz = fz - k0, and each
  in-plane tap w splits into w*(1 - wz) at slice k0 and w*wz at slice k0+1.
  Ray id = (a*Dv + v)*Du + uu; 2D ray id = a*D + d.

  3D with random directions (Sec. 4.3: projection images from directions
  uniform on the sphere): view a has a frame (d, u, v) given as data, d the
  unit ray direction and (u, v) an orthonormal detector basis perpendicular
  to it.  Ray (a, v, uu) passes through p0 = t_u u + t_v v (t_u = uu -
  (Du-1)/2, t_v = v - (Dv-1)/2; componentwise t_u*u_c + t_v*v_c) in
  coordinates centred on the volume.  March along k = argmax_c |d_c| (first on
  ties), the other axes (i, j) in increasing order; inv = 1/d_k and ia = |inv|
  per view (shared as data).  For slice s = 0..N-1:
      tau = ((s - cc) - p0_k)*inv
      fi = (p0_i + tau*d_i) + cc;  i0 = floor(fi);  wi = fi - i0   (same for j)
      taps (i0, j0) ((1-wi)*(1-wj))*ia, (i0+1, j0) (wi*(1-wj))*ia,
           (i0, j0+1) ((1-wi)*wj)*ia, (i0+1, j0+1) (wi*wj)*ia
  at axis-k coordinate s, in that order; taps outside the volume or of weight
  exactly 0 are dropped.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


class Geometry:
    """Parallel-beam geometry: 2D when det_v == 1 and dim == 2, else 3D."""

    def __init__(self, N: int, n_views: int, det_u: int, det_v: int = 1, dim: int = 2,
                 angles=None, frames=None):
        self.N, self.n_views, self.det_u, self.det_v, self.dim = N, n_views, det_u, det_v, dim
        # 3D random directions: per view (d, u, v) and the march axis, 1/d_k
        self.frames = None if frames is None else np.asarray(frames, dtype=np.float64)
        if self.frames is not None:
            if dim != 3 or self.frames.shape != (n_views, 9):
                raise ValueError("frames: 3D, one (d, u, v) row per view")
            self.axis = [int(np.argmax(np.abs(f[:3]))) for f in self.frames]
            self.inv = [1.0 / f[k] for f, k in zip(self.frames, self.axis)]
        if dim == 2 and det_v != 1:
            raise ValueError("2D geometry has det_v == 1")
        if angles is None:
            angles = [a * math.pi / n_views for a in range(n_views)]
        self.angles = [float(t) for t in angles]
        self.cos = [math.cos(t) for t in self.angles]
        self.sin = [math.sin(t) for t in self.angles]
        self.row_step = [abs(c) >= abs(s) for c, s in zip(self.cos, self.sin)]
        self.rc = [1.0 / (c if rs else s) for c, s, rs in zip(self.cos, self.sin, self.row_step)]
        self.ia = [abs(v) for v in self.rc]
        self.rays_per_view = det_u * det_v
        self.n = N ** dim
        self.m = n_views * self.rays_per_view

    def view_rays(self, a: int) -> np.ndarray:
        return np.arange(a * self.rays_per_view, (a + 1) * self.rays_per_view)


def _inplane_taps(g: Geometry, a: int, du: int):
    """In-plane Joseph taps of bin du in view a: (ix, iy, w) arrays, step order, a then b."""
    N = g.N
    cc = (N - 1) / 2.0
    t = du - (g.det_u - 1) / 2.0
    steps = np.arange(N, dtype=np.float64)
    s_int = np.arange(N, dtype=np.int64)
    co, si, rc, ia = g.cos[a], g.sin[a], g.rc[a], g.ia[a]
    pos = steps - cc                               # y (row-stepping) or xx (column-stepping)
    if g.row_step[a]:
        u = t - pos * si
    else:
        u = t - pos * co
    f = u * rc + cc
    j0f = np.floor(f)
    w1 = f - j0f
    wa = (1.0 - w1) * ia
    wb = w1 * ia
    j0 = j0f.astype(np.int64)
    minor = np.stack([j0, j0 + 1], axis=1).reshape(-1)      # interpolated index
    major = np.stack([s_int, s_int], axis=1).reshape(-1)    # stepped index
    w = np.stack([wa, wb], axis=1).reshape(-1)
    keep = (minor >= 0) & (minor < N) & (w != 0.0)
    minor, major, w = minor[keep], major[keep], w[keep]
    if g.row_step[a]:
        return minor, major, w      # ix = minor, iy = major
    return major, minor, w          # ix = major, iy = minor


def _frame_taps(g: Geometry, ray: int):
    """Taps of one ray of the random-direction 3D geometry (voxel, weight)."""
    N = g.N
    a, rem = divmod(int(ray), g.rays_per_view)
    iv, iu = divmod(rem, g.det_u)
    f = g.frames[a]
    d, u, v = f[0:3], f[3:6], f[6:9]
    tu = iu - (g.det_u - 1) / 2.0
    tv = iv - (g.det_v - 1) / 2.0
    p0 = [tu * u[c] + tv * v[c] for c in range(3)]
    k = g.axis[a]
    i, j = [c for c in range(3) if c != k]
    inv = g.inv[a]
    ia = abs(inv)
    cc = (N - 1) / 2.0
    s = np.arange(N, dtype=np.int64)
    tau = ((s.astype(np.float64) - cc) - p0[k]) * inv
    fi = (p0[i] + tau * d[i]) + cc
    fj = (p0[j] + tau * d[j]) + cc
    i0f, j0f = np.floor(fi), np.floor(fj)
    wi, wj = fi - i0f, fj - j0f
    i0, j0 = i0f.astype(np.int64), j0f.astype(np.int64)
    w = np.stack([((1.0 - wi) * (1.0 - wj)) * ia, (wi * (1.0 - wj)) * ia,
                  ((1.0 - wi) * wj) * ia, (wi * wj) * ia], axis=1).reshape(-1)
    ci = np.stack([i0, i0 + 1, i0, i0 + 1], axis=1).reshape(-1)
    cj = np.stack([j0, j0, j0 + 1, j0 + 1], axis=1).reshape(-1)
    ck = np.repeat(s, 4)
    coord = np.zeros((3, ci.size), dtype=np.int64)
    coord[k], coord[i], coord[j] = ck, ci, cj
    keep = ((coord >= 0) & (coord < N)).all(axis=0) & (w != 0.0)
    idx = (coord[2] * N + coord[1]) * N + coord[0]
    return idx[keep], w[keep]


def ray_taps(g: Geometry, ray: int):
    """(pixel indices int64, weights float64) of one row of A."""
    if g.frames is not None:
        return _frame_taps(g, ray)
    if g.dim == 2:
        a, d = divmod(int(ray), g.det_u)
        ix, iy, w = _inplane_taps(g, a, d)
        return iy * g.N + ix, w
    N = g.N
    a, rem = divmod(int(ray), g.rays_per_view)
    v, du = divmod(rem, g.det_u)
    ix, iy, w = _inplane_taps(g, a, du)
    cc = (N - 1) / 2.0
    fz = (v - (g.det_v - 1) / 2.0) + cc
    k0f = math.floor(fz)
    wz = fz - k0f
    k0 = int(k0f)
    idx, wt = [], []
    # per in-plane tap: slice k0 then slice k0+1
    w_lo = w * (1.0 - wz)
    w_hi = w * wz
    base = iy * N + ix
    lo = np.stack([(k0 * N * N) + base, ((k0 + 1) * N * N) + base], axis=1).reshape(-1)
    ww = np.stack([w_lo, w_hi], axis=1).reshape(-1)
    kk = np.stack([np.full_like(base, k0), np.full_like(base, k0 + 1)], axis=1).reshape(-1)
    keep = (kk >= 0) & (kk < N) & (ww != 0.0)
    idx, wt = lo[keep], ww[keep]
    return idx, wt


def rows(g: Geometry, ray_ids) -> sp.csr_matrix:
    """The rows of A for the given ray ids, stacked in that order (len(ray_ids) x n)."""
    indptr = [0]
    cols, vals = [], []
    for ray in ray_ids:
        idx, w = ray_taps(g, ray)
        cols.append(idx)
        vals.append(w)
        indptr.append(indptr[-1] + len(idx))
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = np.concatenate(vals) if vals else np.zeros(0)
    return sp.csr_matrix((vals, cols, np.array(indptr)), shape=(len(ray_ids), g.n))


def full_matrix(g: Geometry) -> sp.csr_matrix:
    return rows(g, range(g.m))
