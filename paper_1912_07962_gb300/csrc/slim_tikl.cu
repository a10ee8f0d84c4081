// slimTik with a lower-bidiagonal L: W = (L^T L)^{-1} applied by two
// recurrences (declarations and the arithmetic in slim_tikl.cuh).
#include <algorithm>

#include "slim_device.cuh"
#include "slim_tikl.cuh"

namespace slim {

namespace {

constexpr int kRowThreads = 256;     // a CTA per row of the new block
constexpr int kVecThreads = 1024;    // the update's single vector

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// In place, by the whole CTA: y <- L^{-1} y (trans = false) or y <- L^{-T} y
// (trans = true).  In the running index k (k = i forward, k = n-1-j backward)
// the recurrence is y_k = g_k y_{k-1} + h_k with g_0 = 0, h_k = y_k / d0,
//   forward:  g_k = -d1_i / d0_i,
//   backward: g_k = -d1_{j+1} / d0_j.
// s_m: 2 * blockDim.x doubles of shared memory.
__device__ void bidiag_solve(double* y, int n, const double* d0inv, const double* d1, bool trans,
                             double* s_m) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int chunk = (n + T - 1) / T;
  const int k0 = min(n, tid * chunk), k1 = min(n, k0 + chunk);
  // affine map y_out = A y_in + B of this thread's chunk
  double A = 1.0, B = 0.0;
  for (int k = k0; k < k1; ++k) {
    const int i = trans ? n - 1 - k : k;
    const double g = k == 0 ? 0.0 : -(trans ? d1[i + 1] : d1[i]) * d0inv[i];
    const double h = y[i] * d0inv[i];
    A = g * A;
    B = fma(g, B, h);
  }
  s_m[tid] = A;
  s_m[T + tid] = B;
  __syncthreads();
  if (tid == 0) {   // chain the chunk maps: the value entering each chunk
    double yin = 0.0;
    for (int t = 0; t < T; ++t) {
      const double a = s_m[t], b = s_m[T + t];
      s_m[t] = yin;
      yin = fma(a, yin, b);
    }
  }
  __syncthreads();
  double yv = s_m[tid];
  for (int k = k0; k < k1; ++k) {
    const int i = trans ? n - 1 - k : k;
    const double g = k == 0 ? 0.0 : -(trans ? d1[i + 1] : d1[i]) * d0inv[i];
    yv = fma(g, yv, y[i] * d0inv[i]);
    y[i] = yv;
  }
  __syncthreads();
}

// CTA i: U_i = W a_i^T for row i of the new block (its taps in the ring).
template <typename T>
__global__ void __launch_bounds__(kRowThreads) tikl_rows_kernel(StepArgs<T> a, TiklArgs t) {
  __shared__ double s_m[2 * kRowThreads];
  const int i = blockIdx.x;
  const long long n = a.n;
  double* u = t.U + (size_t)i * n;
  for (long long j = threadIdx.x; j < n; j += blockDim.x) u[j] = 0.0;
  __syncthreads();
  const int q = a.info->slot * a.ell + i;
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  const double* rw = a.ring_w + (size_t)q * a.taps;
  for (int s = threadIdx.x; s < a.taps; s += blockDim.x)
    if (rp[s] >= 0) atomicAdd(&u[rp[s]], rw[s]);
  __syncthreads();
  bidiag_solve(u, (int)n, t.d0inv, t.d1, true, s_m);
  bidiag_solve(u, (int)n, t.d0inv, t.d1, false, s_m);
}

// UT[pix][i] = U[i][pix], 32 x 32 tiles through shared memory.
__global__ void tikl_transpose_kernel(const double* U, double* UT, int ell, long long n) {
  __shared__ double tile[32][33];
  const long long p0 = (long long)blockIdx.x * 32;
  const int i0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r;
    const long long pix = p0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < ell && pix < n) ? U[(size_t)i * n + pix] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const long long pix = p0 + r;
    const int i = i0 + threadIdx.x;
    if (pix < n && i < ell) UT[(size_t)pix * ell + i] = tile[threadIdx.x][r];
  }
}

// Warp per (ring row q, 32 rows of the new block): lanes over the new rows i,
// summing w_{q,t} UT[pix_{q,t}][i] over row q's taps (one coalesced read of
// UT per tap).  Writes both G[q][new_i] and G[new_i][q].
template <typename T>
__global__ void __launch_bounds__(256) tikl_gram_kernel(StepArgs<T> a, TiklArgs t) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int chunks = (a.ell + 31) / 32;
  if (w >= (long long)a.p * chunks) return;
  const int q = (int)(w / chunks), i = (int)(w % chunks) * 32 + lane;
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  const double* rw = a.ring_w + (size_t)q * a.taps;
  double acc = 0.0;
  for (int s = 0; s < a.taps; ++s) {
    const int pix = rp[s];
    if (pix >= 0 && i < a.ell) acc += rw[s] * t.UT[(size_t)pix * a.ell + i];
  }
  if (i < a.ell) {
    const int col = a.info->slot * a.ell + i;
    a.G[(size_t)q * a.P + col] = acc;
    a.G[(size_t)col * a.P + q] = acc;
  }
}

// v += z_q a_q over the ring rows (v zeroed before): v = M_k^T z.
template <typename T>
__global__ void __launch_bounds__(256) tikl_scatter_v_kernel(StepArgs<T> a, TiklArgs t) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= a.p) return;
  const double c = a.z[q];
  if (c == 0.0) return;
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  const double* rw = a.ring_w + (size_t)q * a.taps;
  for (int s = lane; s < a.taps; s += 32)
    if (rp[s] >= 0) atomicAdd(&t.v[rp[s]], c * rw[s]);
}

// v <- W v (one CTA).
__global__ void __launch_bounds__(kVecThreads) tikl_apply_kernel(TiklArgs t, int n) {
  __shared__ double s_m[2 * kVecThreads];
  bidiag_solve(t.v, n, t.d0inv, t.d1, true, s_m);
  bidiag_solve(t.v, n, t.d0inv, t.d1, false, s_m);
}

template <typename T>
__global__ void tikl_axpy_kernel(StepArgs<T> a, TiklArgs t) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < a.n;
       j += (long long)gridDim.x * blockDim.x)
    a.x[j] -= (T)(a.eta * t.v[j]);
}

}  // namespace

template <typename T>
cudaError_t launch_tikl_gram(const StepArgs<T>& a, const TiklArgs& t, cudaStream_t s) {
  tikl_rows_kernel<T><<<a.ell, kRowThreads, 0, s>>>(a, t);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tikl_transpose_kernel<<<dim3(cdiv(a.n, 32), cdiv(a.ell, 32)), dim3(32, 8), 0, s>>>(t.U, t.UT,
                                                                                    a.ell, a.n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long warps = (long long)a.p * ((a.ell + 31) / 32);
  tikl_gram_kernel<T><<<cdiv(warps, 8), 256, 0, s>>>(a, t);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tikl_update(const StepArgs<T>& a, const TiklArgs& t, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(t.v, 0, (size_t)a.n * sizeof(double), s);
  if (e != cudaSuccess) return e;
  tikl_scatter_v_kernel<T><<<cdiv(a.p, 8), 256, 0, s>>>(a, t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tikl_apply_kernel<<<1, kVecThreads, 0, s>>>(t, (int)a.n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(cdiv(a.n, 256), 152LL * 8);
  tikl_axpy_kernel<T><<<grid, 256, 0, s>>>(a, t);
  return cudaGetLastError();
}

template cudaError_t launch_tikl_gram<float>(const StepArgs<float>&, const TiklArgs&, cudaStream_t);
template cudaError_t launch_tikl_gram<double>(const StepArgs<double>&, const TiklArgs&, cudaStream_t);
template cudaError_t launch_tikl_update<float>(const StepArgs<float>&, const TiklArgs&, cudaStream_t);
template cudaError_t launch_tikl_update<double>(const StepArgs<double>&, const TiklArgs&, cudaStream_t);

}  // namespace slim
