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
  int decay_after;             // 1/k decay of the damping after this step (0: none)
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
  // stored rows of A (a_mode 1: float32 values, 2: bfloat16 values); null if
  // the rows are generated by the projector
  const int* csr_ptr;      // [m+1]
  const int* csr_col;      // [nnz]
  const void* csr_val;     // [nnz]
  int csr_bf16;
  // slimTik, Eq. (slimTik) with C_k = diag(c): beta = lam_tik^2 / M (0: slimLS),
  // the count c_k of Tikhonov rows (0: blocks of M_k, 1: r as printed), 1/c
  // per pixel (null: C_k = I)
  double tik_beta;
  int tik_reading;
  const double* cinv;
  // sg (B_k = alpha_k I): the scatter takes z = r_k / lambda_k on the block's rows
  int sg;
  // threads per ring row in the scatter: 8, 16 or 32 (32 for view blocks)
  int lanes;
  // view blocks in the random cyclic order (a permutation of the views per
  // epoch) instead of i.i.d. draws; the current epoch's permutation and its epoch
  int cyclic;
  int* perm;               // [n_views]
  long long* perm_epoch;   // -1 before the first
};

// Sliced ELLPACK with slices of 32 lines (SELL-32): line l of slice s has its
// entry k at slice_ptr[s] + 32 k + (l mod 32); short lines are padded with
// index 0 and value 0.
struct Sell {
  long long lines = 0;      // rows (or columns) covered
  long long stored = 0;     // entries including padding
  int* slice_ptr = nullptr; // [slices+1] offsets of the slices
  int* idx = nullptr;       // [stored]
  void* val = nullptr;      // [stored]
};

// Stored A: CSR by rays and a CSC copy by pixels, values float32 or bfloat16.
struct CsrStore {
  long long nnz = 0;
  int bf16 = 0;
  int max_row = 0;          // bound on the entries of a row (2N)
  int max_col = 0;          // bound on the entries of a column (2 A_v)
  int* row_ptr = nullptr;   // [m+1]
  int* col = nullptr;       // [nnz]
  void* val = nullptr;      // [nnz]
  int* col_ptr = nullptr;   // [n+1]
  int* row = nullptr;       // [nnz]
  void* cval = nullptr;     // [nnz]
  // SELL-32 copy of the CSC for the transposed full pass: slices of 32
  // consecutive pixels, each pixel's entries in ray order
  Sell cols32;
};

// Build the stored rows of all m rays from the projector (values rounded to
// float32 or bfloat16), and the CSC copy.  Allocates the arrays in `st`.
cudaError_t build_csr(const ViewGeom* views, int N, int D, long long m, long long n, int bf16,
                      CsrStore* st, cudaStream_t s);
void free_csr(CsrStore* st);

// y[i] = A_{ids[i]} x over stored rows (ids == nullptr: all m rows), and
// x += A^T y over all rows using the CSC copy (ids == nullptr) or the rows.
template <typename T> cudaError_t launch_csr_project(const CsrStore& a, const int* ids, int count,
                                                     const T* x, T* y, cudaStream_t s);
template <typename T> cudaError_t launch_csr_backproject(const CsrStore& a, long long n,
                                                         const int* ids, int count, const T* y,
                                                         T* x, cudaStream_t s);

template <typename T> cudaError_t launch_sample(const StepArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_forward_residual(const StepArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_gram_update(const StepArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_scatter(const StepArgs<T>& a, cudaStream_t s);

// slimTik: rhs -= (beta/mu_k) M_k x over the window's rows, and
// x *= 1 - eta beta/mu_k (before the scatter adds -eta C^{-1} M_k^T z).
template <typename T> cudaError_t launch_tik_rhs(const StepArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_tik_scale(const StepArgs<T>& a, cudaStream_t s);

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
