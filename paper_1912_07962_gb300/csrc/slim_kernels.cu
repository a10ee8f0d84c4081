// Per-step kernels of the slimLS iteration (Eq. (ram) with the Woodbury form of Eq. (B_k)).
#include "slim_kernels.cuh"

namespace slim {

namespace {
constexpr int kWarpsPerCta = 8;
constexpr int kCta = 32 * kWarpsPerCta;

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Step 1: draw tau_k (Sec. 1: W_k i.i.d. uniform over the M views), set the
// ring slot of the new block, lambda_k (constant or the ramp of Sec. 4.2),
// the new block's ray ids, and clear the right-hand side.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void sample_kernel(StepArgs<T> a) {
  __shared__ long long s_k;
  __shared__ int s_view, s_slot;
  if (threadIdx.x == 0) {
    long long k = *a.done + 1;
    int view = (int)bounded32(draw64(a.seed, kStreamBlocks, (unsigned long long)(k - 1)),
                              (uint32_t)a.n_views);
    int slot = (int)((k - 1) % a.nslots);
    double lam_k = a.lam;
    if (a.ramp && k <= a.r + 1) lam_k = __ddiv_rn(__dmul_rn(a.lam, (double)(a.r + 1)), (double)k);
    a.info->k = k;
    a.info->slot = slot;
    a.info->view = view;
    a.info->lam_k = lam_k;
    *a.done = k;
    s_k = k;
    s_view = view;
    s_slot = slot;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.ell; i += blockDim.x)
    a.ring_ids[s_slot * a.ell + i] = s_view * a.D + i;
  for (int i = threadIdx.x; i < a.P; i += blockDim.x) a.rhs[i] = 0.0;
}

// ---------------------------------------------------------------------------
// Step 2 (fused): for each ray of the new block march the Joseph taps, store
// them in the ring slot (pixel, float64 weight), record the block's
// pixel -> ray map for the Gram update, and form r_k = A_k x - b_k.
// One warp per ray; lanes take the march steps; warp-shuffle reduction.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kCta) forward_residual_kernel(StepArgs<T> a) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= a.ell) return;
  const int slot = a.info->slot;
  const int q = slot * a.ell + w;
  const int ray = a.ring_ids[q];
  const int view = ray / a.D, d = ray - view * a.D;
  const ViewGeom v = a.views[view];
  const double cc = 0.5 * (double)(a.N - 1);
  const double t = (double)d - 0.5 * (double)(a.D - 1);
  int* rp = a.ring_pix + (size_t)q * a.taps;
  double* rw = a.ring_w + (size_t)q * a.taps;
  const long long n = a.n;
  T acc = T(0);
  for (int s = lane; s < a.N; s += 32) {
    Tap2 tp = joseph_step(v, t, cc, s);
    int pa = tp.wa != 0.0 ? inplane_pixel(v.row_step, a.N, s, tp.minor0) : -1;
    int pb = tp.wb != 0.0 ? inplane_pixel(v.row_step, a.N, s, tp.minor0 + 1) : -1;
    rp[2 * s] = pa;
    rp[2 * s + 1] = pb;
    rw[2 * s] = pa >= 0 ? tp.wa : 0.0;
    rw[2 * s + 1] = pb >= 0 ? tp.wb : 0.0;
    if (pa >= 0) {
      acc += (T)tp.wa * a.x[pa];
      if (atomicCAS(&a.map_ray[pa], -1, w) != -1) set_status(a.status, SLIM_EINVAL);
      a.map_w[pa] = tp.wa;
    }
    if (pb >= 0) {
      acc += (T)tp.wb * a.x[pb];
      if (atomicCAS(&a.map_ray[n + pb], -1, w) != -1) set_status(a.status, SLIM_EINVAL);
      a.map_w[n + pb] = tp.wb;
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) a.rhs[q] = (double)(acc - a.b[ray]);
}

// ---------------------------------------------------------------------------
// Step 3: incremental Gram update.  For every ring row q (each retained ray,
// the new block included) accumulate A_k a_q^T over a_q's stored taps through
// the new block's pixel map, then write row/column block `slot` of G.
// One warp per ring row; per-warp accumulator of ell doubles in shared memory.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kCta) gram_update_kernel(StepArgs<T> a) {
  extern __shared__ double acc_all[];   // kWarpsPerCta * ell
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = blockIdx.x * kWarpsPerCta;
  const int q = q0 + wib;
  double* acc = acc_all + (size_t)wib * a.ell;
  for (int i = lane; i < a.ell; i += 32) acc[i] = 0.0;
  __syncwarp();
  const long long n = a.n;
  if (q < a.p && a.ring_ids[q] >= 0) {
    const int* rp = a.ring_pix + (size_t)q * a.taps;
    const double* rw = a.ring_w + (size_t)q * a.taps;
    for (int t = lane; t < a.taps; t += 32) {
      int pix = rp[t];
      if (pix < 0) continue;
      double wq = rw[t];
      int ia = a.map_ray[pix];
      if (ia >= 0) atomicAdd(&acc[ia], wq * a.map_w[pix]);
      int ib = a.map_ray[n + pix];
      if (ib >= 0) atomicAdd(&acc[ib], wq * a.map_w[n + pix]);
    }
  }
  __syncthreads();
  const int base = a.info->slot * a.ell;
  const int nq = min(kWarpsPerCta, a.p - q0);
  // column block: G[q][base + i] (contiguous in i)
  if (q < a.p)
    for (int i = lane; i < a.ell; i += 32) a.G[(size_t)q * a.P + base + i] = acc[i];
  // row block: G[base + i][q0 .. q0+nq) (nq consecutive doubles per row)
  for (int idx = threadIdx.x; idx < a.ell * kWarpsPerCta; idx += blockDim.x) {
    int i = idx / kWarpsPerCta, wq = idx % kWarpsPerCta;
    if (wq < nq) a.G[(size_t)(base + i) * a.P + q0 + wq] = acc_all[(size_t)wq * a.ell + i];
  }
}

// ---------------------------------------------------------------------------
// Step 5: x -= eta * M_k^T z over all retained rows (atomic scatter-add), and
// clear the new block's entries of the pixel map for the next step.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kCta) scatter_kernel(StepArgs<T> a) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= a.p || a.ring_ids[q] < 0) return;
  const bool is_new = (q / a.ell) == a.info->slot;
  const T c = (T)(-a.eta * a.z[q]);
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  const double* rw = a.ring_w + (size_t)q * a.taps;
  const long long n = a.n;
  for (int t = lane; t < a.taps; t += 32) {
    int pix = rp[t];
    if (pix < 0) continue;
    if (c != T(0)) atomicAdd(&a.x[pix], c * (T)rw[t]);
    if (is_new) a.map_ray[(t & 1) * n + pix] = -1;
  }
}

template <typename TF>
__global__ void form_k_kernel(const StepInfo* info, const double* G, TF* L, int P) {
  const double lam = info->lam_k;
  const long long total = (long long)P * P;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx / P), j = (int)(idx % P);
    if (j > i) continue;
    double v = G[idx];
    if (i == j) v += lam;
    L[idx] = (TF)v;
  }
}

__global__ void refine_residual_kernel(const StepInfo* info, const double* G, const double* z,
                                       const double* rhs, double* res, int P) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= P) return;
  const double* g = G + (size_t)row * P;
  double s = 0.0;
  for (int j = lane; j < P; j += 32) s += g[j] * z[j];
  s = warp_sum(s);
  if (lane == 0) res[row] = rhs[row] - info->lam_k * z[row] - s;
}

__global__ void axpy_kernel(double* z, const double* dz, int P) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) z[i] += dz[i];
}

template <typename T>
__global__ void __launch_bounds__(kCta) project_kernel(const ViewGeom* views, int N, int D,
                                                      const int* ids, int count, const T* x,
                                                      T* y) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= count) return;
  const int ray = ids ? ids[w] : w;
  const int view = ray / D, d = ray - view * D;
  const ViewGeom v = views[view];
  const double cc = 0.5 * (double)(N - 1), t = (double)d - 0.5 * (double)(D - 1);
  T acc = T(0);
  for (int s = lane; s < N; s += 32) {
    Tap2 tp = joseph_step(v, t, cc, s);
    int pa = tp.wa != 0.0 ? inplane_pixel(v.row_step, N, s, tp.minor0) : -1;
    int pb = tp.wb != 0.0 ? inplane_pixel(v.row_step, N, s, tp.minor0 + 1) : -1;
    if (pa >= 0) acc += (T)tp.wa * x[pa];
    if (pb >= 0) acc += (T)tp.wb * x[pb];
  }
  acc = warp_sum(acc);
  if (lane == 0) y[w] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kCta) backproject_kernel(const ViewGeom* views, int N, int D,
                                                          const int* ids, int count, const T* y,
                                                          T* x) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= count) return;
  const int ray = ids ? ids[w] : w;
  const T yv = y[w];
  if (yv == T(0)) return;
  const int view = ray / D, d = ray - view * D;
  const ViewGeom v = views[view];
  const double cc = 0.5 * (double)(N - 1), t = (double)d - 0.5 * (double)(D - 1);
  for (int s = lane; s < N; s += 32) {
    Tap2 tp = joseph_step(v, t, cc, s);
    int pa = tp.wa != 0.0 ? inplane_pixel(v.row_step, N, s, tp.minor0) : -1;
    int pb = tp.wb != 0.0 ? inplane_pixel(v.row_step, N, s, tp.minor0 + 1) : -1;
    if (pa >= 0) atomicAdd(&x[pa], (T)tp.wa * yv);
    if (pb >= 0) atomicAdd(&x[pb], (T)tp.wb * yv);
  }
}

template <typename T>
__global__ void rel_err_kernel(const T* x, const double* ref, long long n, double* out) {
  double e = 0.0, r = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double d = (double)x[i] - ref[i];
    e += d * d;
    r += ref[i] * ref[i];
  }
  e = warp_sum(e);
  r = warp_sum(r);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], e);
    atomicAdd(&out[1], r);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_sample(const StepArgs<T>& a, cudaStream_t s) {
  sample_kernel<T><<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward_residual(const StepArgs<T>& a, cudaStream_t s) {
  forward_residual_kernel<T><<<cdiv(a.ell, kWarpsPerCta), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram_update(const StepArgs<T>& a, cudaStream_t s) {
  size_t smem = (size_t)kWarpsPerCta * a.ell * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gram_update_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  gram_update_kernel<T><<<cdiv(a.p, kWarpsPerCta), kCta, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter(const StepArgs<T>& a, cudaStream_t s) {
  scatter_kernel<T><<<cdiv(a.p, kWarpsPerCta), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename TF>
cudaError_t launch_form_k(const StepInfo* info, const double* G, TF* L, int P, cudaStream_t s) {
  long long total = (long long)P * P;
  int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  form_k_kernel<TF><<<grid, 256, 0, s>>>(info, G, L, P);
  return cudaGetLastError();
}

cudaError_t launch_refine_residual(const StepInfo* info, const double* G, const double* z,
                                   const double* rhs, double* res, int P, cudaStream_t s) {
  refine_residual_kernel<<<cdiv(P, kWarpsPerCta), kCta, 0, s>>>(info, G, z, rhs, res, P);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* z, const double* dz, int P, cudaStream_t s) {
  axpy_kernel<<<cdiv(P, 256), 256, 0, s>>>(z, dz, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project(const ViewGeom* views, int N, int D, const int* ids, int count,
                           const T* x, T* y, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  project_kernel<T><<<cdiv(count, kWarpsPerCta), kCta, 0, s>>>(views, N, D, ids, count, x, y);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backproject(const ViewGeom* views, int N, int D, const int* ids, int count,
                               const T* y, T* x, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  backproject_kernel<T><<<cdiv(count, kWarpsPerCta), kCta, 0, s>>>(views, N, D, ids, count, y, x);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rel_err(const T* x, const double* ref, long long n, double* out,
                           cudaStream_t s) {
  int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
  rel_err_kernel<T><<<grid, 256, 0, s>>>(x, ref, n, out);
  return cudaGetLastError();
}

#define SLIM_INSTANTIATE(T)                                                                     \
  template cudaError_t launch_sample<T>(const StepArgs<T>&, cudaStream_t);                    \
  template cudaError_t launch_forward_residual<T>(const StepArgs<T>&, cudaStream_t);          \
  template cudaError_t launch_gram_update<T>(const StepArgs<T>&, cudaStream_t);               \
  template cudaError_t launch_scatter<T>(const StepArgs<T>&, cudaStream_t);                   \
  template cudaError_t launch_form_k<T>(const StepInfo*, const double*, T*, int, cudaStream_t); \
  template cudaError_t launch_project<T>(const ViewGeom*, int, int, const int*, int, const T*, \
                                         T*, cudaStream_t);                                    \
  template cudaError_t launch_backproject<T>(const ViewGeom*, int, int, const int*, int,       \
                                             const T*, T*, cudaStream_t);                      \
  template cudaError_t launch_rel_err<T>(const T*, const double*, long long, double*, cudaStream_t);

SLIM_INSTANTIATE(float)
SLIM_INSTANTIATE(double)

}  // namespace slim
