// LSQR for the damped least-squares problem of one slimLS step (Eq.
// slimLSstep, Sec. 4.2), one cooperative persistent launch per step.
//
// Golub-Kahan bidiagonalisation of M (the window's rows, read from the tap
// ring) from the right-hand side c = [0; ...; r_k; ...; 0], with the QR
// factorisation of [B_i; d I] (d = lambda_k^{1/2}) updated by two plane
// rotations per iteration; s and the search direction w follow by recurrence.
// u and v are kept unnormalised (their norms beta, alpha held as scalars), so
// that an iteration needs two grid-wide sums:
//   phase A  rows:     u' = (M v_raw)/alpha - alpha u_raw/beta, tmp += M^T u'
//            elements: the previous iteration's s += (phi/rho) w,
//                      w = v_raw/alpha - (theta/rho) w
//            (the scalings by 1/alpha, 1/beta are products with reciprocals)
//            sum ||u'||^2 -> beta'
//   phase B  elements: v' = tmp/beta' - beta' v_raw/alpha, tmp = 0
//            sum ||v'||^2 -> alpha'
//   scalars  the two rotations, the stopping test.
// The last iteration's update of s and the update of x close the launch.
// Grid-wide sums are per-CTA partials summed in block order by one warp of
// every CTA (the same value everywhere, the same order every run); the
// scatter M^T u' is atomic.  Every grid barrier is bounded.
#include "slim_lsqr.cuh"

#include <algorithm>
#include <cmath>

#include "slim_device.cuh"
#include "slim_grid.cuh"

namespace slim {

namespace {

constexpr int kLsqrThreads = 256;
constexpr int kLsqrWarps = kLsqrThreads / 32;
// Sum of every thread's v over the grid, returned in every thread: CTA sums
// in part[blockIdx.x], then each CTA's warp 0 adds part[0..grid) in a fixed
// order.
__device__ bool grid_sum(double v, double* part, unsigned* bar, int* status, double* sred,
                         int* s_flag, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sred[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kLsqrWarps; ++q) t += sred[q];
    part[blockIdx.x] = t;
  }
  if (!grid_barrier(bar, status, s_flag)) return false;
  if (warp == 0) {
    double t = 0.0;
    for (int q = lane; q < (int)gridDim.x; q += 32) t += __ldcg(part + q);
    t = warp_sum(t);
    if (lane == 0) sred[kLsqrWarps] = t;
  }
  __syncthreads();
  *out = sred[kLsqrWarps];
  __syncthreads();
  return true;
}

// Plane rotation with c a + s b = r >= 0 and -s a + c b = 0.
__device__ __forceinline__ void rotation(double a, double b, double& c, double& s, double& r) {
  r = hypot(a, b);
  if (r == 0.0) {
    c = 1.0;
    s = 0.0;
  } else {
    c = a / r;
    s = b / r;
  }
}

// tmp += weight * (row q of M)
__device__ __forceinline__ void scatter_row(const int* rp, const double* rw, int taps, double weight,
                                            double* tmp) {
  for (int t = threadIdx.x & 31; t < taps; t += 32) {
    const int pix = rp[t];
    if (pix >= 0) atomicAdd(tmp + pix, rw[t] * weight);
  }
}

template <typename T>
__global__ void __launch_bounds__(kLsqrThreads) lsqr_kernel(LsqrArgs<T> a) {
  __shared__ double sred[kLsqrWarps + 1];
  __shared__ int s_flag;
  const int lane = threadIdx.x & 31;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const int gw = (int)(gt >> 5), nwarps = (int)(nthreads >> 5);
  int pb = 0;   // partial-sum buffer in use (two, alternating)
  auto reduce = [&](double v, double* out) {
    const bool ok = grid_sum(v, a.part + (size_t)pb * gridDim.x, a.bar, a.status, sred, &s_flag, out);
    pb ^= 1;
    return ok;
  };
  const double damp = sqrt(a.info->lam_k);
  auto write_stats = [&](int it, double res, double res0) {
    if (gt == 0) {
      a.stats[0] = (double)it;
      a.stats[1] = res;
      a.stats[2] = res0;
    }
  };

  // u_raw = c, tmp = M^T c, s = 0; beta_1 = ||c||
  double acc = 0.0;
  for (int q = gw; q < a.p; q += nwarps) {
    const double cq = a.c[q];
    if (lane == 0) {
      a.u[q] = cq;
      acc += cq * cq;
    }
    if (cq != 0.0 && a.ring_ids[q] >= 0)
      scatter_row(a.ring_pix + (size_t)q * a.taps, a.ring_w + (size_t)q * a.taps, a.taps, cq, a.tmp);
  }
  for (long long j = gt; j < a.n; j += nthreads) a.s[j] = 0.0;
  double beta;
  if (!reduce(acc, &beta)) return;
  beta = sqrt(beta);
  // y = 0 (c = 0, or M^T c = 0): x unchanged, or scaled by 1 - eta beta/mu (slimTik)
  auto finish_zero = [&]() {
    const double keep = 1.0 - a.eta * a.info->tik_c;
    if (keep != 1.0)
      for (long long j = gt; j < a.n; j += nthreads) a.x[j] = (T)(keep * (double)a.x[j]);
    write_stats(0, 0.0, 0.0);
  };
  if (beta == 0.0) {
    finish_zero();
    return;
  }
  // v_raw = M^T c / beta; alpha_1 = ||v_raw||  (scalings by reciprocals
  // computed once: float64 division is slow on this GPU's FP64 pipe)
  acc = 0.0;
  const double inv_beta1 = 1.0 / beta;
  const double* vg = a.wh ? a.vs : a.v;   // the vector the rows gather: wh v (or v)
  for (long long j = gt; j < a.n; j += nthreads) {
    const double whj = a.wh ? a.wh[j] : 1.0;
    const double t = whj * __ldcg(a.tmp + j) * inv_beta1;
    a.tmp[j] = 0.0;
    a.v[j] = t;
    if (a.wh) a.vs[j] = whj * t;
    acc += t * t;
  }
  double alpha;
  if (!reduce(acc, &alpha)) return;
  alpha = sqrt(alpha);
  if (alpha == 0.0) {
    finish_zero();
    return;
  }
  double rho_bar = alpha, phi_bar = beta;
  const double res0 = alpha * beta;
  double res = res0;
  double phi = 0.0, rho = 1.0, theta = 0.0;   // the last iteration's scalars
  int it = 0;
  while (it < a.max_iter) {
    ++it;
    // phase A: update of s and w owed by the previous iteration (w_1 = v_1),
    // then u' = M v - alpha u and its scatter
    const double inv_alpha = 1.0 / alpha;
    const double inv_beta = beta > 0.0 ? 1.0 / beta : 1.0;
    const double cs = phi / rho, cw = theta / rho;
    for (long long j = gt; j < a.n; j += nthreads) {
      const double vj = a.v[j] * inv_alpha;
      if (it == 1) {
        a.w[j] = vj;
      } else {
        const double wj = a.w[j];
        a.s[j] += cs * wj;
        a.w[j] = vj - cw * wj;
      }
    }
    acc = 0.0;
    for (int q = gw; q < a.p; q += nwarps) {
      const double uq = a.u[q] * inv_beta;
      double mv = 0.0;
      const bool row = a.ring_ids[q] >= 0;
      const int* rp = a.ring_pix + (size_t)q * a.taps;
      const double* rw = a.ring_w + (size_t)q * a.taps;
      if (row) {
        // four taps per lane per round: their loads are issued together
        for (int t0 = lane; t0 < a.taps; t0 += 128) {
          int pix[4];
          double wt[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int t = t0 + 32 * e;
            pix[e] = t < a.taps ? rp[t] : -1;
            wt[e] = t < a.taps ? rw[t] : 0.0;
          }
#pragma unroll
          for (int e = 0; e < 4; ++e)   // other SMs wrote v: read around L1
            if (pix[e] >= 0) mv += wt[e] * __ldcg(vg + pix[e]);
        }
        mv = warp_sum(mv) * inv_alpha;
      }
      const double un = mv - alpha * uq;
      if (lane == 0) {
        a.u[q] = un;
        acc += un * un;
      }
      if (row && un != 0.0) scatter_row(rp, rw, a.taps, un, a.tmp);
    }
    double beta_n;
    if (!reduce(acc, &beta_n)) return;
    beta_n = sqrt(beta_n);
    // phase B: v' = M^T u'/beta' - beta' v
    acc = 0.0;
    const double inv_beta_n = beta_n > 0.0 ? 1.0 / beta_n : 1.0;
    for (long long j = gt; j < a.n; j += nthreads) {
      const double whj = a.wh ? a.wh[j] : 1.0;
      const double mt = whj * __ldcg(a.tmp + j);
      a.tmp[j] = 0.0;
      const double t = mt * inv_beta_n - beta_n * (a.v[j] * inv_alpha);
      a.v[j] = t;
      if (a.wh) a.vs[j] = whj * t;
      acc += t * t;
    }
    double alpha_n;
    if (!reduce(acc, &alpha_n)) return;
    alpha_n = sqrt(alpha_n);
    // the damping row folded into the diagonal, then beta' removed
    double c1, s1, rho_hat;
    rotation(rho_bar, damp, c1, s1, rho_hat);
    const double phi_hat = c1 * phi_bar;
    double cr, sr;
    rotation(rho_hat, beta_n, cr, sr, rho);
    theta = sr * alpha_n;
    rho_bar = -cr * alpha_n;
    phi = cr * phi_hat;
    phi_bar = sr * phi_hat;
    res = fabs(phi_bar * cr) * alpha_n;
    beta = beta_n;
    if (alpha_n == 0.0) break;   // the Krylov space is exhausted: s is exact
    alpha = alpha_n;
    if (a.tol > 0.0 && res <= a.tol * res0) break;
  }
  // the last iteration's update of s, and x -= eta s (slimTik: x = (1 -
  // eta beta/mu) x - eta wh s)
  const double cs_last = phi / rho;
  const double keep = 1.0 - a.eta * a.info->tik_c;
  for (long long j = gt; j < a.n; j += nthreads) {
    const double sj = a.s[j] + cs_last * a.w[j];
    a.s[j] = sj;
    const double step = a.wh ? a.wh[j] * sj : sj;
    a.x[j] = (T)(keep * (double)a.x[j] - a.eta * step);
  }
  write_stats(it, res, res0);
}

}  // namespace

size_t lsqr_part_count(int num_sms) { return 2 * (size_t)std::max(1, num_sms) * 2; }

template <typename T>
cudaError_t launch_lsqr(const LsqrArgs<T>& a, int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lsqr_kernel<T>, kLsqrThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  // one CTA per SM: fewer arrivals at each grid barrier
  const int grid = std::max(1, num_sms) * std::min(per_sm, 1);
  if ((e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
  LsqrArgs<T> args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)lsqr_kernel<T>, dim3(grid), dim3(kLsqrThreads),
                                     params, 0, s);
}

template cudaError_t launch_lsqr<float>(const LsqrArgs<float>&, int, cudaStream_t);
template cudaError_t launch_lsqr<double>(const LsqrArgs<double>&, int, cudaStream_t);

}  // namespace slim
