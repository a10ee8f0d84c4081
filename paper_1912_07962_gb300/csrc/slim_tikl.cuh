// slimTik with a lower-bidiagonal L (Eq. slimTik, C_k = L^T L): the kernels
// that apply W = C^{-1} = L^{-1} L^{-T} on the image vector.
//
// L acts on the image vector x (length n) as (L x)_i = d0_i x_i + d1_i x_{i-1}
// (d1_0 unused), so C = L^T L is tridiagonal and W v is two first-order
// recurrences: L^T t = v backward (t_j = (v_j - d1_{j+1} t_{j+1}) / d0_j),
// then L u = t forward (u_i = (t_i - d1_i u_{i-1}) / d0_i).  Each recurrence
// runs in one CTA as a chunked affine scan: every thread composes the affine
// map of its chunk, one thread chains the chunk maps, every thread re-runs
// its chunk from its incoming value.
//
// The Woodbury form of the step with this W (the algebra of the diagonal
// case, W general):
//   (mu_k I + M_k W M_k^T) z = c - (beta/mu_k) M_k x_{k-1},
//   x_k = (1 - eta beta/mu_k) x_{k-1} - eta W M_k^T z.
#pragma once
#include <cuda_runtime.h>

#include "slim_kernels.cuh"

namespace slim {

struct TiklArgs {
  const double* d0inv;   // [n] 1 / d0
  const double* d1;      // [n] sub-diagonal of L (d1[0] unused)
  double* U;             // [ell * n] W a_i^T for the new block's rows, row i at U + i n
  double* UT;            // [n * ell] the same, pixel-major (UT[pix * ell + i])
  double* v;             // [n] work vector of the update
};

// Gram rows of the new block: G[q][new_i] = G[new_i][q] = a_q W a_i^T for every
// ring row q (ring order, P x P).  Uses the new block's taps in the ring.
template <typename T>
cudaError_t launch_tikl_gram(const StepArgs<T>& a, const TiklArgs& t, cudaStream_t s);
// x -= eta W M_k^T z (after slimTik's scaling of x, when that applies).
template <typename T>
cudaError_t launch_tikl_update(const StepArgs<T>& a, const TiklArgs& t, cudaStream_t s);

}  // namespace slim
