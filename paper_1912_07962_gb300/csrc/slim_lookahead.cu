// Kernels of the pipelined view-block iteration (geometry chain ahead of the
// iterate chain; layout described in slim_lookahead.cuh).
#include <algorithm>

#include "slim_lookahead.cuh"

namespace slim {

namespace {
constexpr int kWarps = 8;
constexpr int kCta = 32 * kWarps;

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ int eslot_of(long long block, int eslots) {
  return (int)((block - 1) % eslots);
}

// ---------------------------------------------------------------------------
// Geometry chain of step j = gdone + 1
// ---------------------------------------------------------------------------

// Draw tau_j (Sec. 1: i.i.d. uniform over the views), lambda_j (constant or
// the ramp of Sec. 4.2) and the block's ray ids in its extended slot.
template <typename T>
__global__ void la_sample_kernel(LaArgs<T> a) {
  __shared__ int s_view, s_e;
  __shared__ int s_perm[kMaxCyclicViews];
  const long long j0 = *a.gdone + 1;
  const int cview = a.cyclic ? cyclic_view(a.seed, j0, a.n_views, a.perm, a.perm_epoch, s_perm) : 0;
  __syncthreads();   // every thread has read the step counter
  if (threadIdx.x == 0) {
    const long long j = j0;
    const int view = a.cyclic ? cview
                              : (int)bounded32(draw64(a.seed, kStreamBlocks,
                                                      (unsigned long long)(j - 1)),
                                               (uint32_t)a.n_views);
    double lam_j = damping_k(a.lam, j, a.r, a.ramp, a.decay_after);
    double tik_c = 0.0;
    if (a.tik_beta > 0.0) {
      // Eq. (slimTik): mu_j = lambda_j + c_j lam_tik^2 / M
      const long long cnt = a.tik_reading ? a.r : (j < a.r + 1 ? j : a.r + 1);
      lam_j = __dadd_rn(lam_j, __dmul_rn((double)cnt, a.tik_beta));
      tik_c = __ddiv_rn(a.tik_beta, lam_j);
    }
    StepInfo* inf = a.info_buf + (int)(j % a.nbuf);
    inf->k = j;
    inf->slot = (int)((j - 1) % a.nslots);
    inf->view = view;
    inf->lam_k = lam_j;
    inf->tik_c = tik_c;
    *a.gdone = j;
    s_view = view;
    s_e = eslot_of(j, a.eslots);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.ell; i += blockDim.x)
    a.ring_ids[s_e * a.ell + i] = s_view * a.D + i;
}

// March the rays of block j (one warp per ray) into its extended slot and
// record the block's pixel -> ray map (a pixel is in at most two rays of one
// view: tap a and tap b).
template <typename T>
__global__ void __launch_bounds__(kCta) la_taps_kernel(LaArgs<T> a) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= a.ell) return;
  const long long j = *a.gdone;
  const int q = eslot_of(j, a.eslots) * a.ell + w;
  const int ray = a.ring_ids[q];
  const int view = ray / a.D, d = ray - view * a.D;
  const ViewGeom v = a.views[view];
  const double cc = 0.5 * (double)(a.N - 1);
  const double t = (double)d - 0.5 * (double)(a.D - 1);
  int* rp = a.ring_pix + (size_t)q * a.taps;
  double* rw = a.ring_w + (size_t)q * a.taps;
  const long long n = a.n;
  for (int s = lane; s < a.N; s += 32) {
    Tap2 tp = joseph_step(v, t, cc, s);
    const int pa = tp.wa != 0.0 ? inplane_pixel(v.row_step, a.N, s, tp.minor0) : -1;
    const int pb = tp.wb != 0.0 ? inplane_pixel(v.row_step, a.N, s, tp.minor0 + 1) : -1;
    rp[2 * s] = pa;
    rp[2 * s + 1] = pb;
    rw[2 * s] = pa >= 0 ? tp.wa : 0.0;
    rw[2 * s + 1] = pb >= 0 ? tp.wb : 0.0;
    if (pa >= 0) {
      if (atomicCAS(&a.map_ray[pa], -1, w) != -1) set_status(a.status, SLIM_EINVAL);
      a.map_w[pa] = tp.wa;
    }
    if (pb >= 0) {
      if (atomicCAS(&a.map_ray[n + pb], -1, w) != -1) set_status(a.status, SLIM_EINVAL);
      a.map_w[n + pb] = tp.wb;
    }
  }
}

// Gram rows of block j: for every row a_q of the blocks tau_{j-r} .. tau_j
// (window position pos, block j-r+pos), A_j a_q^T through the pixel map, into
// row/column block of slot e_j of the extended Gram matrix.  One warp per
// window row, an ell-double accumulator per warp in shared memory.
template <typename T>
__global__ void __launch_bounds__(kCta) la_gram_kernel(LaArgs<T> a) {
  extern __shared__ double acc_all[];   // kWarps * ell
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long j = *a.gdone;
  const int wq0 = blockIdx.x * kWarps;
  const int wq = wq0 + wib;
  const int p = a.nslots * a.ell;
  double* acc = acc_all + (size_t)wib * a.ell;
  for (int i = lane; i < a.ell; i += 32) acc[i] = 0.0;
  __syncwarp();
  const long long n = a.n;
  const long long blk = wq < p ? j - a.r + wq / a.ell : 0;
  const int qe = blk >= 1 ? eslot_of(blk, a.eslots) * a.ell + wq % a.ell : -1;
  if (qe >= 0) {
    const int* rp = a.ring_pix + (size_t)qe * a.taps;
    const double* rw = a.ring_w + (size_t)qe * a.taps;
    for (int t = lane; t < a.taps; t += 32) {
      const int pix = rp[t];
      if (pix < 0) continue;
      const double wv = a.cinv ? rw[t] * a.cinv[pix] : rw[t];   // M C^{-1} M^T
      const int ia = a.map_ray[pix];
      if (ia >= 0) atomicAdd(&acc[ia], wv * a.map_w[pix]);
      const int ib = a.map_ray[n + pix];
      if (ib >= 0) atomicAdd(&acc[ib], wv * a.map_w[n + pix]);
    }
  }
  __syncthreads();
  const int base = eslot_of(j, a.eslots) * a.ell;
  if (qe >= 0)
    for (int i = lane; i < a.ell; i += 32) a.G[(size_t)qe * a.Pe + base + i] = acc[i];
  // row block: G[base + i][qe of each warp]
  for (int idx = threadIdx.x; idx < a.ell * kWarps; idx += blockDim.x) {
    const int i = idx / kWarps, w = idx % kWarps;
    const int wq2 = wq0 + w;
    if (wq2 >= p) continue;
    const long long b2 = j - a.r + wq2 / a.ell;
    if (b2 < 1) continue;
    const int qe2 = eslot_of(b2, a.eslots) * a.ell + wq2 % a.ell;
    a.G[(size_t)(base + i) * a.Pe + qe2] = acc_all[(size_t)w * a.ell + i];
  }
}

// Clear block j's entries of the pixel map.
template <typename T>
__global__ void __launch_bounds__(kCta) la_map_clear_kernel(LaArgs<T> a) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= a.ell) return;
  const int q = eslot_of(*a.gdone, a.eslots) * a.ell + w;
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  for (int t = lane; t < a.taps; t += 32) {
    const int pix = rp[t];
    if (pix < 0) continue;
    if (t & 1) a.map_ray[a.n + pix] = -1;
    else a.map_ray[pix] = -1;
  }
}

// Row q of the factored matrix of step k -> extended row.  The window's
// blocks are in chronological order, block k - (r - s) at position
// s = q / ell (the newest, block k, last), so that the first solve's right-hand
// side [0; ...; 0; r_k] is zero above the last block; -1 if that block index is
// < 1 or q is padding.
__global__ void la_ext_map_kernel(const StepInfo* info, int ell, int nslots, int eslots, int p,
                                  int P, int* ext) {
  const long long k = info->k;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < P; q += gridDim.x * blockDim.x) {
    int e = -1;
    if (q < p) {
      const int s = q / ell;
      const long long blk = k - (nslots - 1 - s);
      if (blk >= 1) e = eslot_of(blk, eslots) * ell + q % ell;
    }
    ext[q] = e;
  }
}

template <typename TF>
__global__ void la_form_kernel(const StepInfo* info, const int* __restrict__ ext,
                               const double* __restrict__ G, int Pe, TF* L, int P) {
  const double lam = info->lam_k;
  const long long total = (long long)P * P;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / P), j = (int)(idx % P);
    if (j > i) continue;
    const int ei = ext[i], ej = ext[j];
    double v = (ei >= 0 && ej >= 0) ? G[(size_t)ei * Pe + ej] : 0.0;
    if (i == j) v += lam;
    L[idx] = (TF)v;
  }
}

// ---------------------------------------------------------------------------
// Iterate chain of step k (the step held in `info`)
// ---------------------------------------------------------------------------

// r_k = A_k x - b_k from the stored taps of block k, into the last block of
// the right-hand side (the newest block's place in the factored matrix).
// The per-lane order of the sum is the one of the fused march-and-residual
// kernel of the plain form, so both forms give the same residual.
template <typename T>
__global__ void __launch_bounds__(kCta) la_residual_kernel(LaArgs<T> a, const StepInfo* info) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= a.ell) return;
  const long long k = info->k;
  const int q = eslot_of(k, a.eslots) * a.ell + w;
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  const double* rw = a.ring_w + (size_t)q * a.taps;
  T acc = T(0);
  for (int s = lane; s < a.N; s += 32) {
    const int pa = rp[2 * s], pb = rp[2 * s + 1];
    if (pa >= 0) acc += (T)rw[2 * s] * a.x[pa];
    if (pb >= 0) acc += (T)rw[2 * s + 1] * a.x[pb];
  }
  acc = warp_sum(acc);
  if (lane == 0) a.rhs[(a.nslots - 1) * a.ell + w] = (double)(acc - a.b[a.ring_ids[q]]);
}

// res = rhs - lambda_k z - G z over the factored rows (G gathered through the
// extended-row map).  Sixteen rows per CTA, two per warp walked together so
// that each lane keeps eight gathers of G in flight; the map and z are staged
// in shared memory once per CTA, so the rows of G are the only global stream.
constexpr int kRefineRowsPerWarp = 2;
__global__ void __launch_bounds__(kCta) la_refine_kernel(const StepInfo* info,
                                                         const int* __restrict__ ext,
                                                         const double* __restrict__ G, int Pe,
                                                         const double* z, const double* rhs,
                                                         double* res, int P) {
  extern __shared__ double s_z[];                         // P doubles, then P ints
  int* s_ext = reinterpret_cast<int*>(s_z + P);
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    s_z[j] = z[j];
    s_ext[j] = ext[j];
  }
  __syncthreads();
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = (blockIdx.x * kWarps + wib) * kRefineRowsPerWarp;
  if (row0 >= P) return;
  const double* g[kRefineRowsPerWarp];
#pragma unroll
  for (int u = 0; u < kRefineRowsPerWarp; ++u) {
    const int row = row0 + u;
    const int ei = row < P ? s_ext[row] : -1;
    g[u] = ei >= 0 ? G + (size_t)ei * Pe : nullptr;
  }
  double s[kRefineRowsPerWarp] = {};
  for (int base = 0; base < P; base += 128) {
    double gv[kRefineRowsPerWarp][4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = base + 32 * t + lane;
      const int ej = j < P ? s_ext[j] : -1;
#pragma unroll
      for (int u = 0; u < kRefineRowsPerWarp; ++u)
        gv[u][t] = (ej >= 0 && g[u]) ? __ldg(g[u] + ej) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = base + 32 * t + lane;
      if (j < P) {
#pragma unroll
        for (int u = 0; u < kRefineRowsPerWarp; ++u) s[u] += gv[u][t] * s_z[j];
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kRefineRowsPerWarp; ++u) {
    const double t = warp_sum(s[u]);
    const int row = row0 + u;
    if (lane == 0 && row < P) res[row] = rhs[row] - info->lam_k * s_z[row] - t;
  }
}

// x -= eta M_k^T z over the rows of the window (atomic scatter-add).
template <typename T>
__global__ void __launch_bounds__(kCta) la_scatter_kernel(LaArgs<T> a, const int* ext) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= a.p) return;
  const int qe = ext[q];
  if (qe < 0) return;
  const T c = (T)(-a.eta * a.z[q]);
  if (c == T(0)) return;
  const int* rp = a.ring_pix + (size_t)qe * a.taps;
  const double* rw = a.ring_w + (size_t)qe * a.taps;
  for (int t = lane; t < a.taps; t += 32) {
    const int pix = rp[t];
    if (pix >= 0) atomicAdd(&a.x[pix], c * (T)(a.cinv ? rw[t] * a.cinv[pix] : rw[t]));
  }
}

// slimTik (Eq. slimTik, C_k = diag(c)): rhs c - (beta/mu_k) M_k x_{k-1} over
// the factored rows (one warp per row), then x *= 1 - eta beta/mu_k before
// the scatter adds -eta C^{-1} M_k^T z.
template <typename T>
__global__ void __launch_bounds__(kCta) la_tik_rhs_kernel(LaArgs<T> a, const int* ext,
                                                          const StepInfo* info) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= a.p) return;
  const int qe = ext[q];
  if (qe < 0) return;
  const int* rp = a.ring_pix + (size_t)qe * a.taps;
  const double* rw = a.ring_w + (size_t)qe * a.taps;
  double acc = 0.0;
  for (int t = lane; t < a.taps; t += 32) {
    const int pix = rp[t];
    if (pix >= 0) acc += rw[t] * (double)a.x[pix];
  }
  acc = warp_sum(acc);
  if (lane == 0) a.rhs[q] -= info->tik_c * acc;
}

template <typename T>
__global__ void la_tik_scale_kernel(LaArgs<T> a, const StepInfo* info) {
  const T f = (T)(1.0 - a.eta * info->tik_c);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x)
    a.x[i] *= f;
}

}  // namespace

template <typename T>
cudaError_t la_launch_sample(const LaArgs<T>& a, cudaStream_t s) {
  la_sample_kernel<T><<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t la_launch_taps(const LaArgs<T>& a, cudaStream_t s) {
  la_taps_kernel<T><<<cdiv(a.ell, kWarps), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t la_launch_gram(const LaArgs<T>& a, cudaStream_t s) {
  const size_t smem = (size_t)kWarps * a.ell * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(la_gram_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  la_gram_kernel<T><<<cdiv((long long)a.nslots * a.ell, kWarps), kCta, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t la_launch_map_clear(const LaArgs<T>& a, cudaStream_t s) {
  la_map_clear_kernel<T><<<cdiv(a.ell, kWarps), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t la_launch_ext_map(const StepInfo* info, int ell, int nslots, int eslots, int p, int P,
                              int* ext, cudaStream_t s) {
  la_ext_map_kernel<<<cdiv(P, 256), 256, 0, s>>>(info, ell, nslots, eslots, p, P, ext);
  return cudaGetLastError();
}

template <typename TF>
cudaError_t la_launch_form(const StepInfo* info, const int* ext, const double* G, int Pe, TF* L,
                           int P, cudaStream_t s) {
  const long long total = (long long)P * P;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  la_form_kernel<TF><<<grid, 256, 0, s>>>(info, ext, G, Pe, L, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t la_launch_residual(const LaArgs<T>& a, const StepInfo* info, cudaStream_t s) {
  la_residual_kernel<T><<<cdiv(a.ell, kWarps), kCta, 0, s>>>(a, info);
  return cudaGetLastError();
}

cudaError_t la_launch_refine(const StepInfo* info, const int* ext, const double* G, int Pe,
                             const double* z, const double* rhs, double* res, int P,
                             cudaStream_t s) {
  const size_t smem = (size_t)P * (sizeof(double) + sizeof(int));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(la_refine_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  la_refine_kernel<<<cdiv(P, kWarps * kRefineRowsPerWarp), kCta, smem, s>>>(info, ext, G, Pe, z,
                                                                            rhs, res, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t la_launch_scatter(const LaArgs<T>& a, const int* ext, cudaStream_t s) {
  la_scatter_kernel<T><<<cdiv(a.p, kWarps), kCta, 0, s>>>(a, ext);
  return cudaGetLastError();
}

template <typename T>
cudaError_t la_launch_tik_rhs(const LaArgs<T>& a, const int* ext, const StepInfo* info,
                              cudaStream_t s) {
  la_tik_rhs_kernel<T><<<cdiv(a.p, kWarps), kCta, 0, s>>>(a, ext, info);
  return cudaGetLastError();
}

template <typename T>
cudaError_t la_launch_tik_scale(const LaArgs<T>& a, const StepInfo* info, cudaStream_t s) {
  const int grid = (int)std::min<long long>((a.n + 255) / 256, 152LL * 8);
  la_tik_scale_kernel<T><<<grid, 256, 0, s>>>(a, info);
  return cudaGetLastError();
}

#define SLIM_LA_INST(T)                                                                      \
  template cudaError_t la_launch_sample<T>(const LaArgs<T>&, cudaStream_t);                  \
  template cudaError_t la_launch_taps<T>(const LaArgs<T>&, cudaStream_t);                    \
  template cudaError_t la_launch_gram<T>(const LaArgs<T>&, cudaStream_t);                    \
  template cudaError_t la_launch_map_clear<T>(const LaArgs<T>&, cudaStream_t);               \
  template cudaError_t la_launch_residual<T>(const LaArgs<T>&, const StepInfo*, cudaStream_t); \
  template cudaError_t la_launch_scatter<T>(const LaArgs<T>&, const int*, cudaStream_t);      \
  template cudaError_t la_launch_tik_rhs<T>(const LaArgs<T>&, const int*, const StepInfo*,     \
                                            cudaStream_t);                                     \
  template cudaError_t la_launch_tik_scale<T>(const LaArgs<T>&, const StepInfo*, cudaStream_t);
SLIM_LA_INST(float)
SLIM_LA_INST(double)
template cudaError_t la_launch_form<float>(const StepInfo*, const int*, const double*, int, float*,
                                           int, cudaStream_t);
template cudaError_t la_launch_form<double>(const StepInfo*, const int*, const double*, int,
                                            double*, int, cudaStream_t);

}  // namespace slim
