// Pipelined form of the view-block iteration.
//
// The system lambda_k I + M_k M_k^T of Eq. (B_k) depends only on the blocks
// drawn (tau_{k-r} .. tau_k), never on the iterate, so its Gram rows and its
// factorisation can be prepared ahead of the update of x.  The geometry
// chain of step j (draw tau_j, march its rays into the tap ring, add its row
// and column block to the Gram matrix, form and factor K_j) runs up to D
// steps ahead of the iterate chain of step k (r_k = A_k x - b_k, the damped
// solve with the prepared factor, x -= eta M_k^T z).
//
// Tap rows live in an extended ring of r+1+D blocks (block j in slot
// (j-1) mod (r+1+D)), and the Gram matrix is kept over the extended ring
// (order Pe = (r+1+D) ell).  The geometry chain of step j writes only slot
// (j-1) mod (r+1+D), which no iterate chain still in flight reads.  The
// factor, the solve vectors and the iterate-chain kernels keep the ring
// order of the plain form (block i at ring slot (i-1) mod (r+1)); a per-step
// map takes ring index q to its row of the extended ring.
#pragma once
#include <cuda_runtime.h>

#include "slim_device.cuh"

namespace slim {

template <typename T>
struct LaArgs {
  const ViewGeom* views;
  int N, D, n_views;
  long long n, m;
  int ell, r, nslots, eslots;    // nslots = r+1 ring slots, eslots = r+1+D extended slots
  int p, P, Pe, taps;            // (r+1) ell, padded order of the factor, eslots*ell, 2N
  unsigned long long seed;
  double lam, eta;
  int ramp;
  int decay_after;             // 1/k decay of the damping after this step (0: none)
  long long* gdone;              // geometry steps prepared (device counter)
  StepInfo* info_buf;            // [nbuf] per-buffer step values
  int nbuf;                      // D+1
  int* ring_ids;                 // [Pe]
  int* ring_pix;                 // [Pe*taps]
  double* ring_w;                // [Pe*taps]
  int* map_ray;                  // [2n] pixel -> ray of the block being added
  double* map_w;                 // [2n]
  double* G;                     // [Pe*Pe] Gram matrix over the extended ring
  double* rhs;                   // [P]
  double* z;                     // [P]
  T* x;
  const T* b;
  int* status;
  double tik_beta;               // slimTik: lam_tik^2 / M (0: slimLS)
  int tik_reading;               // Tikhonov count: 0 blocks of M_k, 1 r
  const double* cinv;            // [n] 1/c of C_k = diag(c); null: C_k = I
  int cyclic;                    // random cyclic order of the views (see StepArgs)
  int* perm;                     // [n_views]
  long long* perm_epoch;
};

// Geometry chain (stream of its own, one step at a time).
template <typename T> cudaError_t la_launch_sample(const LaArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t la_launch_taps(const LaArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t la_launch_gram(const LaArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t la_launch_map_clear(const LaArgs<T>& a, cudaStream_t s);
// Row of the factored matrix (blocks in chronological order, the newest last)
// -> extended row for the step held in `info` (-1: empty or padding).
cudaError_t la_launch_ext_map(const StepInfo* info, int ell, int nslots, int eslots, int p, int P,
                              int* ext, cudaStream_t s);
// L = lambda_k I + G gathered into ring order (lower triangle), precision TF.
template <typename TF> cudaError_t la_launch_form(const StepInfo* info, const int* ext,
                                                  const double* G, int Pe, TF* L, int P,
                                                  cudaStream_t s);
// Iterate chain.
template <typename T> cudaError_t la_launch_residual(const LaArgs<T>& a, const StepInfo* info,
                                                     cudaStream_t s);
cudaError_t la_launch_refine(const StepInfo* info, const int* ext, const double* G, int Pe,
                             const double* z, const double* rhs, double* res, int P,
                             cudaStream_t s);
template <typename T> cudaError_t la_launch_scatter(const LaArgs<T>& a, const int* ext,
                                                    cudaStream_t s);
// slimTik: rhs -= (beta/mu_k) M_k x over the factored rows, and
// x *= 1 - eta beta/mu_k before the scatter.
template <typename T> cudaError_t la_launch_tik_rhs(const LaArgs<T>& a, const int* ext,
                                                    const StepInfo* info, cudaStream_t s);
template <typename T> cudaError_t la_launch_tik_scale(const LaArgs<T>& a, const StepInfo* info,
                                                      cudaStream_t s);

}  // namespace slim
