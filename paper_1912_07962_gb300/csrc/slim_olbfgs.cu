// The online L-BFGS comparator, one cooperative persistent launch per step.
//
// H g is formed in the compact representation of the L-BFGS inverse (Byrd,
// Nocedal and Schnabel, Math. Programming 63, 1994).  With the m stored pairs
// in order (oldest first), S = [s_i], Y = [y_i], R the upper triangle of
// S^T Y (R_ij = s_i^T y_j for i <= j), D its diagonal and H^0 = gamma I:
//   H g = gamma g + S w - gamma Y t,   R t = S^T g,
//   R^T w = (D + gamma Y^T Y) t - gamma Y^T g.
// This is the two-loop recursion's H g up to rounding, but its 2m dot
// products S^T g, Y^T g come from one pass over the pair vectors instead of
// 2m dependent passes.  S^T Y and Y^T Y are kept between steps; each step
// adds the new pair's column.
//   P1 rows      g = A_k^T r_k (atomic); clear the block's pixel map
//   P2 elements  S^T g, Y^T g (one pass, grid sum); the small triangular
//                solves (in every CTA); d = -eta alpha_k H g, x += d, d kept
//                as the spare s; the spare y and g cleared
//   P3 rows      u = A_k s
//   P4 rows      y = A_k^T u (atomic)
//   P5 elements  s_i^T y, y_i^T y for the stored pairs and the new one (grid
//                sum); CTA 0 stores the pair if s^T y > 0
// Grid sums are per-CTA partials added in block order by every CTA (the same
// value everywhere, the same order every run).  Every grid barrier is bounded.
#include "slim_olbfgs.cuh"

#include <algorithm>

#include "slim_grid.cuh"

namespace slim {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxM = kOlbfgsMaxMem;
constexpr int kPW = 2 * kMaxM + 2;   // sums per grid reduction: 2 per stored pair + the new pair

// Sum every thread's acc[0..kPW) over the grid into out[] in every CTA.
__device__ __forceinline__ bool grid_sums(const double (&acc)[kPW], double* part, unsigned* bar,
                                          int* status, double (*s_red)[kPW], double* out,
                                          int* s_flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kPW; ++i) {
    const double v = warp_sum(acc[i]);
    if (lane == 0) s_red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < kPW) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += s_red[w][threadIdx.x];
    part[(size_t)blockIdx.x * kPW + threadIdx.x] = t;
  }
  if (!grid_barrier(bar, status, s_flag)) return false;
  for (int i = warp; i < kPW; i += kWarps) {
    double t = 0.0;
    for (int q = lane; q < (int)gridDim.x; q += 32) t += __ldcg(part + (size_t)q * kPW + i);
    t = warp_sum(t);
    if (lane == 0) out[i] = t;
  }
  __syncthreads();
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) olbfgs_kernel(OlbfgsArgs<T> a) {
  __shared__ int s_flag;
  __shared__ double s_red[kWarps][kPW];
  __shared__ double s_dot[kPW];
  __shared__ double s_cs[kMaxM], s_cy[kMaxM];
  __shared__ double s_cg;
  __shared__ int s_slot[kMaxM];
  __shared__ int s_m, s_spare;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * kWarps + warp, nwarps = gridDim.x * kWarps;
  const long long gt = (long long)blockIdx.x * kThreads + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * kThreads;
  const long long n = a.n;
  const int L = a.tau + 1;   // leading dimension of S^T Y and Y^T Y
  if (threadIdx.x == 0) {
    s_m = a.state[0];
    s_spare = a.state[1];
  }
  if (threadIdx.x < a.tau) s_slot[threadIdx.x] = a.state[2 + threadIdx.x];
  __syncthreads();
  const int m = s_m, spare = s_spare;
  const double alpha = 1.0 / a.info->lam_k;
  double* Ssp = a.S + (size_t)spare * n;
  double* Ysp = a.Y + (size_t)spare * n;

  // P1: g = A_k^T r_k
  for (int q = gwarp; q < a.ell; q += nwarps) {
    const double c = a.rhs[q];
    const int* rp = a.ring_pix + (size_t)q * a.taps;
    const double* rw = a.ring_w + (size_t)q * a.taps;
    for (int t = lane; t < a.taps; t += 32) {
      const int pix = rp[t];
      if (pix < 0) continue;
      if (c != 0.0) atomicAdd(a.g + pix, rw[t] * c);
      a.map_ray[pix] = -1;
      a.map_ray[n + pix] = -1;
    }
  }
  if (!grid_barrier(a.bar, a.status, &s_flag)) return;

  // P2: S^T g and Y^T g, then H g in compact form
  double acc[kPW];
#pragma unroll
  for (int i = 0; i < kPW; ++i) acc[i] = 0.0;
  for (long long j = gt; j < n; j += nthreads) {
    const double gj = __ldcg(a.g + j);
#pragma unroll
    for (int i = 0; i < kMaxM; ++i)
      if (i < m) {
        const size_t off = (size_t)s_slot[i] * n + j;
        acc[2 * i] += a.S[off] * gj;
        acc[2 * i + 1] += a.Y[off] * gj;
      }
  }
  if (!grid_sums(acc, a.part, a.bar, a.status, s_red, s_dot, &s_flag)) return;
  if (threadIdx.x == 0) {
    double cg = 1.0;   // H = I before the first pair
    if (m > 0) {
      double gsum = 0.0;
      for (int i = 0; i < m; ++i) {
        const int si = s_slot[i];
        gsum += a.SY[si * L + si] / a.YY[si * L + si];
      }
      cg = gsum / m;
      double t[kMaxM];
      for (int i = m - 1; i >= 0; --i) {   // R t = S^T g (back substitution)
        double v = s_dot[2 * i];
        for (int j = i + 1; j < m; ++j) v -= a.SY[s_slot[i] * L + s_slot[j]] * t[j];
        t[i] = v / a.SY[s_slot[i] * L + s_slot[i]];
      }
      for (int i = 0; i < m; ++i) {        // R^T w = (D + gamma Y^T Y) t - gamma Y^T g
        double yy = 0.0;
        for (int j = 0; j < m; ++j) yy += a.YY[s_slot[i] * L + s_slot[j]] * t[j];
        double v = a.SY[s_slot[i] * L + s_slot[i]] * t[i] + cg * yy - cg * s_dot[2 * i + 1];
        for (int j = 0; j < i; ++j) v -= a.SY[s_slot[j] * L + s_slot[i]] * s_cs[j];
        s_cs[i] = v / a.SY[s_slot[i] * L + s_slot[i]];
      }
      for (int i = 0; i < m; ++i) s_cy[i] = -cg * t[i];
    }
    s_cg = cg;
  }
  __syncthreads();
  {
    const double cg = s_cg, step = -a.eta * alpha;
    for (long long j = gt; j < n; j += nthreads) {
      const double gj = __ldcg(a.g + j);
      double h = cg * gj;
#pragma unroll
      for (int i = 0; i < kMaxM; ++i)
        if (i < m) {
          const size_t off = (size_t)s_slot[i] * n + j;
          h += s_cs[i] * a.S[off] + s_cy[i] * a.Y[off];
        }
      const double d = step * h;
      a.x[j] = (T)((double)a.x[j] + d);
      Ssp[j] = d;
      Ysp[j] = 0.0;
      a.g[j] = 0.0;
    }
  }
  if (!grid_barrier(a.bar, a.status, &s_flag)) return;

  // P3: u = A_k s
  for (int q = gwarp; q < a.ell; q += nwarps) {
    const int* rp = a.ring_pix + (size_t)q * a.taps;
    const double* rw = a.ring_w + (size_t)q * a.taps;
    double v = 0.0;
    for (int t = lane; t < a.taps; t += 32) {
      const int pix = rp[t];
      if (pix >= 0) v += rw[t] * __ldcg(Ssp + pix);
    }
    v = warp_sum(v);
    if (lane == 0) a.u[q] = v;
  }
  if (!grid_barrier(a.bar, a.status, &s_flag)) return;

  // P4: y = A_k^T u
  for (int q = gwarp; q < a.ell; q += nwarps) {
    const double c = __ldcg(a.u + q);
    if (c == 0.0) continue;
    const int* rp = a.ring_pix + (size_t)q * a.taps;
    const double* rw = a.ring_w + (size_t)q * a.taps;
    for (int t = lane; t < a.taps; t += 32) {
      const int pix = rp[t];
      if (pix >= 0) atomicAdd(Ysp + pix, rw[t] * c);
    }
  }
  if (!grid_barrier(a.bar, a.status, &s_flag)) return;

  // P5: the new pair's column of S^T Y and Y^T Y
#pragma unroll
  for (int i = 0; i < kPW; ++i) acc[i] = 0.0;
  for (long long j = gt; j < n; j += nthreads) {
    const double yj = __ldcg(Ysp + j);
#pragma unroll
    for (int i = 0; i < kMaxM; ++i)
      if (i < m) {
        const size_t off = (size_t)s_slot[i] * n + j;
        acc[2 * i] += a.S[off] * yj;
        acc[2 * i + 1] += a.Y[off] * yj;
      }
    acc[kPW - 2] += __ldcg(Ssp + j) * yj;
    acc[kPW - 1] += yj * yj;
  }
  if (!grid_sums(acc, a.part, a.bar, a.status, s_red, s_dot, &s_flag)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double sy = s_dot[kPW - 2], yy = s_dot[kPW - 1];
    if (sy > 0.0) {   // the curvature condition: store the pair
      for (int i = 0; i < m; ++i) {
        a.SY[s_slot[i] * L + spare] = s_dot[2 * i];
        a.YY[s_slot[i] * L + spare] = s_dot[2 * i + 1];
        a.YY[spare * L + s_slot[i]] = s_dot[2 * i + 1];
      }
      a.SY[spare * L + spare] = sy;
      a.YY[spare * L + spare] = yy;
      int slots[kMaxM];
      for (int i = 0; i < m; ++i) slots[i] = s_slot[i];
      int mm = m, next;
      if (mm < a.tau) {
        slots[mm++] = spare;
        // the lowest of the tau+1 slots that holds no stored pair (mm <= tau)
        next = -1;
        for (int c = 0; c <= a.tau && next < 0; ++c) {
          bool used = false;
          for (int i = 0; i < mm; ++i) used = used || slots[i] == c;
          if (!used) next = c;
        }
      } else {         // drop the oldest pair: its slot is the next spare
        next = slots[0];
        for (int i = 0; i + 1 < mm; ++i) slots[i] = slots[i + 1];
        slots[mm - 1] = spare;
      }
      a.state[0] = mm;
      a.state[1] = next;
      for (int i = 0; i < mm; ++i) a.state[2 + i] = slots[i];
    }
  }
}

}  // namespace

size_t olbfgs_scratch_count(long long n, int ell, int tau, int num_sms) {
  const size_t L = (size_t)tau + 1;
  return (size_t)n * (1 + 2 * L) + (size_t)ell + 2 * L * L +
         (size_t)std::max(1, num_sms) * kPW;
}

template <typename T>
void olbfgs_bind(OlbfgsArgs<T>* a, double* p, int num_sms) {
  const size_t L = (size_t)a->tau + 1;
  a->g = p;
  a->S = a->g + a->n;
  a->Y = a->S + L * a->n;
  a->u = a->Y + L * a->n;
  a->SY = a->u + a->ell;
  a->YY = a->SY + L * L;
  a->part = a->YY + L * L;
  (void)num_sms;
}

template <typename T>
cudaError_t launch_olbfgs(const OlbfgsArgs<T>& a, int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, olbfgs_kernel<T>, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const int grid = std::max(1, num_sms);   // one CTA per SM (the partial-sum buffer's size)
  if ((e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
  OlbfgsArgs<T> args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)olbfgs_kernel<T>, dim3(grid), dim3(kThreads),
                                     params, 0, s);
}

template void olbfgs_bind<float>(OlbfgsArgs<float>*, double*, int);
template void olbfgs_bind<double>(OlbfgsArgs<double>*, double*, int);
template cudaError_t launch_olbfgs<float>(const OlbfgsArgs<float>&, int, cudaStream_t);
template cudaError_t launch_olbfgs<double>(const OlbfgsArgs<double>&, int, cudaStream_t);

}  // namespace slim
