// The random-direction 3D geometry (Sec. 4.3: projection images taken from
// directions uniform on the unit sphere).  View a has a frame (d, u, v): d
// the unit ray direction, (u, v) an orthonormal detector basis.  Ray
// (a, v, uu) passes through p0 = t_u u + t_v v (t_u = uu - (Du-1)/2,
// t_v = v - (Dv-1)/2) in coordinates centred on the volume.  Joseph's method
// marches it along k = argmax |d_c| (first on ties): at slice s of axis k,
//   tau = ((s - cc) - p0_k) / d_k,  f_c = (p0_c + tau d_c) + cc  (c = i, j),
// and the four bilinear taps around (f_i, f_j) carry the weights
// (1-w_i)(1-w_j), w_i(1-w_j), (1-w_i)w_j, w_i w_j times |1/d_k|, in that
// order, each operation rounded once; taps outside the volume or of weight 0
// are dropped.  Rays of different views cross every slice, so the Gram matrix
// of a window of random rays is dense in general: its entries come from a
// voxel -> ray list of the new block, and the damped solve is the tiled one.
#pragma once
#include <cuda_runtime.h>

#include "slim_device.cuh"
#include "slim_rays.cuh"

namespace slim {

struct FrameGeom {
  double d[3], u[3], v[3];   // ray direction, detector axes
  double inv, ia;            // 1/d_k and |1/d_k| (host division, shared as data)
  int k, i, j;               // march axis; the other two, increasing
  int pad_;
};

// Host: the frame of one view from its (d, u, v) row of 9 values.
FrameGeom make_frame_geom(const double* row9);

struct FrameArgs {
  const FrameGeom* frames;   // [n_views]
  int* vhead;                // [n] voxel -> last entry of the new block there (-1: none)
  int* vnext;                // [ell * taps] next entry at the same voxel
};

// March the new block's rays (ring slot of the step, taps 4 per slice),
// r_k = A_k x - b_k into the right-hand side, and list the block's entries by
// voxel.  The scatter clears the lists' heads afterwards (vhead as its map).
template <typename T> cudaError_t launch_forward_frames(const RayArgs& a, const FrameArgs& f,
                                                        const T* x, const T* b, cudaStream_t s);
// G[q][new] and G[new][q] for every ring row q through the voxel lists.
cudaError_t launch_gram_frames(const RayArgs& a, const FrameArgs& f, cudaStream_t s);
// y[i] = A_{ids[i]} x (ids null: ray i) and x += A_ids^T y.
template <typename T> cudaError_t launch_project_frames(const FrameGeom* frames, int N, int Du,
                                                        int Dv, const int* ids, long long count,
                                                        const T* x, T* y, cudaStream_t s);
template <typename T> cudaError_t launch_backproject_frames(const FrameGeom* frames, int N, int Du,
                                                            int Dv, const int* ids,
                                                            long long count, const T* y, T* x,
                                                            cudaStream_t s);

}  // namespace slim
