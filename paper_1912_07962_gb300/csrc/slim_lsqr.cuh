// LSQR for the damped least-squares problem of one slimLS step, Eq. (slimLSstep):
//   s_k = argmin_s || [M_k; lambda_k^{1/2} I] s - [0; ...; r_k; ...; 0] ||,
// then x_k = x_{k-1} - eta s_k (Sec. 4.2; the paper solves this problem with
// LSQR for damped least squares).  M_k is read from the ring of the retained
// blocks' taps, matrix-free.
#pragma once
#include <cuda_runtime.h>

#include "slim_kernels.cuh"

namespace slim {

template <typename T>
struct LsqrArgs {
  const StepInfo* info;     // lambda_k of the step
  int p, taps;              // rows of the window, tap slots per row
  long long n;              // unknowns
  const int* ring_ids;      // [p] ray id of each row, -1 if the row is empty
  const int* ring_pix;      // [p*taps] pixel of each tap, -1 if none
  const double* ring_w;     // [p*taps] tap weights
  const double* c;          // [p] right-hand side [0; ...; r_k; ...; 0]
  double eta;
  int max_iter;
  double tol;               // stop when ||M^T r - lambda s|| <= tol ||M^T c|| (0: max_iter)
  T* x;                     // [n] x -= eta s at the end
  double* u;                // [p] scratch
  double* v;                // [n]
  double* w;                // [n]
  double* s;                // [n] the step s_k on exit
  double* tmp;              // [n] zero on entry and on exit (M^T u accumulates here)
  double* part;             // [2 * grid] per-CTA partial sums
  unsigned* bar;            // [2] grid barrier (count, generation), zero before the first use
  double* stats;            // [3] iterations, ||M^T r - lambda s|| estimate, ||M^T c||
  int* status;
  // slimTik with C_k = diag(c) (Eq. slimTik): LSQR runs on the window's
  // columns scaled by wh = c^{-1/2} with damping sqrt(mu_k) (info->lam_k) and
  // c = [0..r_k..0] - (beta/mu_k) M x; then x = (1 - eta beta/mu_k) x - eta wh s
  // (info->tik_c = beta/mu_k).  wh null: C = I.
  const double* wh;         // [n] c^{-1/2}, or null
  double* vs;               // [n] wh * v (scratch, used when wh is set)
};

// Cooperative launch of the whole solve and the update of x, one CTA per SM.
template <typename T>
cudaError_t launch_lsqr(const LsqrArgs<T>& a, int num_sms, cudaStream_t s);

// Scratch the solve needs beyond u, v, w, s, tmp: partial sums and the barrier.
size_t lsqr_part_count(int num_sms);

}  // namespace slim
