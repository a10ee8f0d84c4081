// Host launchers of the per-step kernels (definitions in slim_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "slim_device.cuh"

namespace slim {

// Device-resident state of one iteration, as seen by the kernels.
template <typename T>
struct StepArgs {
  StepInfo* info;          // written by the sampler
  long long* done;         // steps completed so far (device counter)
  const ViewGeom* views;   // per-view geometry
  int N, D, n_views;       // image side, bins per view, views
  long long n, m;          // unknowns, rows
  int ell, nslots, r;      // rows per block, r+1 ring slots, memory
  int P, p, taps;          // padded order, (r+1)*ell, tap slots per ray (2N)
  unsigned long long seed;
  double lam, eta;
  int ramp;
  int* ring_ids;           // [p]        ray id per ring row, -1 if empty
  int* ring_pix;           // [p*taps]   pixel of each tap, -1 if none
  double* ring_w;          // [p*taps]   float64 tap weights
  int* map_ray;            // [2*n]      new block's ray at pixel (tap a | tap b), -1 if none
  double* map_w;           // [2*n]      its weight
  double* G;               // [P*P]      Gram matrix M M^T in ring order
  double* rhs;             // [P]        [0..r_k..0]
  double* z;               // [P]        solution
  T* x;                    // [n]
  const T* b;              // [m]
  int* status;
};

template <typename T> cudaError_t launch_sample(const StepArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_forward_residual(const StepArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_gram_update(const StepArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_scatter(const StepArgs<T>& a, cudaStream_t s);

// L = lambda_k I + G on the lower triangle, converted to TF (the factor precision).
template <typename TF> cudaError_t launch_form_k(const StepInfo* info, const double* G, TF* L,
                                                 int P, cudaStream_t s);

// res = rhs - lambda_k z - G z (float64); z += dz.
cudaError_t launch_refine_residual(const StepInfo* info, const double* G, const double* z,
                                   const double* rhs, double* res, int P, cudaStream_t s);
cudaError_t launch_axpy(double* z, const double* dz, int P, cudaStream_t s);

// y[i] = A_{ids[i]} x  (ids == nullptr: ray i), and x += A_ids^T y.
template <typename T> cudaError_t launch_project(const ViewGeom* views, int N, int D,
                                                 const int* ids, int count, const T* x, T* y,
                                                 cudaStream_t s);
template <typename T> cudaError_t launch_backproject(const ViewGeom* views, int N, int D,
                                                     const int* ids, int count, const T* y, T* x,
                                                     cudaStream_t s);

// out[0] += sum (x - ref)^2, out[1] += sum ref^2
template <typename T> cudaError_t launch_rel_err(const T* x, const double* ref, long long n,
                                                 double* out, cudaStream_t s);

}  // namespace slim
