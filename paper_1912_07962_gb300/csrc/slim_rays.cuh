// Random-ray blocks (Sec. 1's W_k selecting ell arbitrary rows): 2D blocks of
// random rays, and the 3D streaming form (views arrive in angle order, each
// block draws rays from the views seen so far; Sec. 4.3).
#pragma once
#include <cuda_runtime.h>

#include "slim_device.cuh"

namespace slim {

struct RayArgs {
  StepInfo* info;
  long long* done;
  const ViewGeom* views;
  int N, Du, Dv, n_views, dim;       // dim 3: det_v == N, ray (a, v, u) lies in z-slice v
  long long n, m;
  int ell, nslots, r, p, taps;       // taps = 2N per ray
  unsigned magic_n;                  // ceil(2^32 / N) (N = 1: 2^32 - 1), exact division by N
  int lanes;                         // threads per ray of the march: 8, 16 or 32
  int short_window;                  // pair Gram: windows of more steps go to the whole warp
  int kind, steps_per_view;          // 1: i.i.d. over all rays; 2: over arrived views
  unsigned long long seed;
  double lam;
  int ramp;
  int decay_after;             // 1/k decay of the damping after this step (0: none)
  int* ring_ids;                     // [p]
  int* ring_pix;                     // [p*taps] voxel index or -1
  double* ring_w;                    // [p*taps]
  double* rhs;                       // [p] (2D: [P])
  double* z;                         // [p] (2D: [P])
  int* status;
  // 2D: dense Gram in ring order
  double* G;
  int P;
  // 3D: per-slice lists of ring rows
  int S, cap;
  int* slice_cnt;                    // [S]
  int* slice_rows;                   // [S*cap]
  int dense;                         // 1: the tiled solve over P rows (2D, 3D random directions)
  int distinct;                      // 1: the ell rays of a block are distinct (Floyd)
};

template <typename T> cudaError_t launch_sample_rays(const RayArgs& a, cudaStream_t s);
template <typename T> cudaError_t launch_forward_rays(const RayArgs& a, T* x, const T* b,
                                                      cudaStream_t s);
// 2D: G[new, q] and G[q, new] for every ring row q, from pairwise ray overlaps.
cudaError_t launch_gram_pairs(const RayArgs& a, cudaStream_t s);
// 3D: group ring rows by z-slice, then per slice form lambda_k I + G_s from
// pairwise overlaps, factor it (float64 Cholesky) and solve for z.
cudaError_t launch_slice_collect(const RayArgs& a, cudaStream_t s);
cudaError_t launch_slice_solve(const RayArgs& a, cudaStream_t s);
size_t slice_solve_smem(int cap);
cudaError_t prepare_slice_solve(int cap);   // opt in to its shared memory (once)

// y[i] = A_{ray i} x for the rays ids[i] (nullptr: ray i), any dim.
template <typename T> cudaError_t launch_project_rays(const ViewGeom* views, int N, int Du, int Dv,
                                                      const int* ids, long long count, const T* x,
                                                      T* y, cudaStream_t s);

}  // namespace slim
