"""Pins for the random-direction 3D Joseph rows (Sec. 4.3's geometry: views
from directions uniform on the sphere).

* Directions in the xy-plane with the detector basis (co, si, 0), (0, 0, 1)
  give the rows of the rotate-about-z geometry (an independent code path,
  pinned on its own) to rounding.
* Rays along z with a detector of N x N unit bins at the voxel centres are
  line sums: A x = sum over z of x.
* The reversed direction (-d, same u, v) is the same line: bit-identical taps.
* A ray through the centre stays inside the volume: its weights sum to
  N / |d_k| (each slice's bilinear weights sum to 1/|d_k|).
* Exchanging two axes of the frames (d, u, v) and of the volume gives the
  same rows with the voxel indices exchanged (the march axis and the
  interpolation axes are bookkept by value, not by position).
* The frames of the input generator are orthonormal and uniform on the sphere
  in the mean.
"""
import math

import numpy as np

import workloads
from oracle import joseph


def test_inplane_directions_match_the_rotation_geometry():
    N, V, Du, Dv = 8, 7, 12, 8
    angles = [a * math.pi / V for a in range(V)]
    frames = np.array([[-math.sin(t), math.cos(t), 0.0, math.cos(t), math.sin(t), 0.0,
                        0.0, 0.0, 1.0] for t in angles])
    g_rot = joseph.Geometry(N, V, Du, Dv, dim=3, angles=angles)
    g_dir = joseph.Geometry(N, V, Du, Dv, dim=3, frames=frames)
    A = joseph.full_matrix(g_rot).toarray()
    B = joseph.full_matrix(g_dir).toarray()
    assert np.abs(A - B).max() <= 1e-13 * np.abs(A).max()
    assert (np.abs(A) > 1e-12).sum() > 1000


def test_axis_aligned_rays_are_line_sums():
    N = 6
    frames = np.array([[0.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0]])
    g = joseph.Geometry(N, 1, N, N, dim=3, frames=frames)
    x = np.random.default_rng(0).standard_normal(N ** 3)
    y = joseph.full_matrix(g) @ x
    want = x.reshape(N, N, N).sum(axis=0).reshape(-1)   # ray (v, u) -> y index v, x index u
    assert np.array_equal(y, want) or np.abs(y - want).max() <= 1e-14 * np.abs(want).max()
    A = joseph.full_matrix(g)
    assert A.nnz == N ** 3 and np.all(A.data == 1.0)


def test_reversed_direction_is_the_same_ray():
    fr = workloads.random_frames(6, 3)
    rev = fr.copy()
    rev[:, :3] *= -1.0
    g1 = joseph.Geometry(10, 6, 14, 13, dim=3, frames=fr)
    g2 = joseph.Geometry(10, 6, 14, 13, dim=3, frames=rev)
    for ray in range(0, g1.m, 5):
        i1, w1 = joseph.ray_taps(g1, ray)
        i2, w2 = joseph.ray_taps(g2, ray)
        o1, o2 = np.lexsort((w1, i1)), np.lexsort((w2, i2))
        assert np.array_equal(i1[o1], i2[o2]) and np.array_equal(w1[o1], w2[o2])


def test_central_ray_weights_sum_to_the_path_per_slice():
    N = 12
    fr = workloads.random_frames(20, 4)
    g = joseph.Geometry(N, 20, 5, 5, dim=3, frames=fr)   # odd detector: bin (2, 2) at p0 = 0
    for a in range(20):
        ray = a * g.rays_per_view + 2 * 5 + 2
        _, w = joseph.ray_taps(g, ray)
        want = N * abs(g.inv[a])
        assert abs(w.sum() - want) <= 1e-12 * want, a


def test_frames_are_orthonormal_and_uniform():
    fr = workloads.random_frames(4000, 9)
    d, u, v = fr[:, :3], fr[:, 3:6], fr[:, 6:9]
    for q in (d, u, v):
        assert np.abs(np.linalg.norm(q, axis=1) - 1.0).max() < 1e-14
    assert np.abs((d * u).sum(1)).max() < 1e-14 and np.abs((d * v).sum(1)).max() < 1e-14
    assert np.abs((u * v).sum(1)).max() < 1e-14
    # uniform on the sphere: mean 0, E[d d^T] = I/3 (4000 samples: 4 sigma bounds)
    assert np.abs(d.mean(axis=0)).max() < 4 * math.sqrt(1 / 3 / 4000)
    assert np.abs(d.T @ d / 4000 - np.eye(3) / 3).max() < 0.03


def test_exchanging_two_axes_permutes_the_voxels():
    N, V, Du, Dv = 7, 8, 11, 10
    fr = workloads.random_frames(V, 13)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        sw = fr.copy()
        for base in (0, 3, 6):       # exchange components a and b of d, u and v
            sw[:, [base + a, base + b]] = sw[:, [base + b, base + a]]
        g1 = joseph.Geometry(N, V, Du, Dv, dim=3, frames=fr)
        g2 = joseph.Geometry(N, V, Du, Dv, dim=3, frames=sw)
        # voxel (x, y, z) of g1 is voxel (x, y, z) with coordinates a, b exchanged in g2
        idx = np.arange(N ** 3)
        c = np.stack([idx % N, (idx // N) % N, idx // (N * N)])
        c[[a, b]] = c[[b, a]]
        perm = (c[2] * N + c[1]) * N + c[0]
        A1 = joseph.full_matrix(g1).toarray()
        A2 = joseph.full_matrix(g2).toarray()
        assert np.abs(A1 - A2[:, perm]).max() <= 1e-14 * np.abs(A1).max(), (a, b)
