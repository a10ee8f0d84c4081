// The online limited-memory BFGS comparator (Sec. 4.1's olbfgs): one step
//   g_k = A_k^T (A_k x_{k-1} - b_k),  x_k = x_{k-1} - eta alpha_k H_k g_k,
// alpha_k = 1/lambda_k, H_k the L-BFGS inverse built from the last tau pairs
// (s_j = x_j - x_{j-1}, y_j = A_j^T A_j s_j) from gamma_k I, gamma_k the mean
// of s^T y / y^T y over the stored pairs (H = I before the first pair); a pair
// with s^T y <= 0 is not stored.  The block's rows come from the tap ring
// (one block, r = 0).
#pragma once
#include <cuda_runtime.h>

#include "slim_device.cuh"

namespace slim {

constexpr int kOlbfgsMaxMem = 20;   // largest memory tau

template <typename T>
struct OlbfgsArgs {
  const StepInfo* info;   // lambda_k of the step
  int ell, taps, tau;     // rows of the block, tap slots per row, memory
  long long n;
  const int* ring_pix;    // [ell*taps] the block's taps
  const double* ring_w;   // [ell*taps]
  const double* rhs;      // [ell] r_k
  int* map_ray;           // [2n] pixel map of the block, cleared here
  double eta;
  T* x;                   // [n]
  double* g;              // [n] zero on entry and on exit
  double* S;              // [(tau+1)*n] pair vectors s, one slot per pair + a spare
  double* Y;              // [(tau+1)*n] y
  double* u;              // [ell] A_k s_new
  double* SY;             // [(tau+1)^2] s_i^T y_j (slot indices, i <= j chronologically)
  double* YY;             // [(tau+1)^2] y_i^T y_j
  int* state;             // [2 + tau] stored pairs m, spare slot, slots oldest first
  double* part;           // [grid * (2 kOlbfgsMaxMem + 2)] per-CTA partial sums
  unsigned* bar;          // [2] grid barrier
  int* status;
};

// Doubles of scratch for n unknowns, ell rows and memory tau on num_sms CTAs.
size_t olbfgs_scratch_count(long long n, int ell, int tau, int num_sms);
// Lay the scratch (zeroed by the caller) out into the args' pointers.
template <typename T>
void olbfgs_bind(OlbfgsArgs<T>* a, double* scratch, int num_sms);

// One cooperative launch, one CTA per SM.
template <typename T>
cudaError_t launch_olbfgs(const OlbfgsArgs<T>& a, int num_sms, cudaStream_t s);

}  // namespace slim
