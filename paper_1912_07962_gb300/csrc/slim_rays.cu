// Random-ray blocks: sampling, the fused ray march + residual, the Gram matrix
// from pairwise ray overlaps, and (3D) the per-slice damped solves.
#include "slim_rays.cuh"

namespace slim {

namespace {
constexpr int kWarpsPerCta = 8;
constexpr int kCta = 32 * kWarpsPerCta;
inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Ray id = (view * Dv + v) * Du + u; t = u - (Du-1)/2; the ray lies in z-slice v.
struct RayDesc {
  int view, slice;
  double t;
};
__device__ __forceinline__ RayDesc decode_ray(int ray, int Du, int Dv) {
  const int rpv = Du * Dv;
  RayDesc d;
  d.view = ray / rpv;
  const int rem = ray - d.view * rpv;
  d.slice = rem / Du;
  d.t = (double)(rem - d.slice * Du) - 0.5 * (double)(Du - 1);
  return d;
}

// Steps [lo, hi] of ray i (its major axis) outside which its taps cannot meet
// those of ray j.  Joseph taps lie within one pixel of the ray's line, so
// overlapping pixels lie within distance 1 of both lines, i.e. within
// 2/|sin(theta_i - theta_j)| of the intersection along ray i; parallel rays
// (same view) can only overlap for adjacent bins and are marched in full.
__device__ __forceinline__ bool overlap_window(const ViewGeom& gi, const RayDesc& ri,
                                               const ViewGeom& gj, const RayDesc& rj, int N,
                                               int& lo, int& hi) {
  lo = 0;
  hi = N - 1;
  if (ri.view == rj.view) return fabs(ri.t - rj.t) <= 1.0;
  const double det = gi.co * gj.si - gi.si * gj.co;   // sin(theta_j - theta_i)
  if (fabs(det) < 1e-9) return true;
  const double cc = 0.5 * (double)(N - 1);
  const double px = (ri.t * gj.si - gi.si * rj.t) / det;
  const double py = (gi.co * rj.t - ri.t * gj.co) / det;
  const double sc = (gi.row_step ? py : px) + cc;
  const double half = 3.0 / fabs(det) + 2.0;
  const double l = floor(sc - half), h = ceil(sc + half);
  if (h < 0.0 || l > (double)(N - 1)) return false;
  lo = l < 0.0 ? 0 : (int)l;
  hi = h > (double)(N - 1) ? N - 1 : (int)h;
  return lo <= hi;
}

// sum_pixels a_i(pix) a_j(pix) for two rays in the same slice, read from the
// stored taps: tap 2s / 2s+1 of a ray are its two taps at step s, so ray j's
// taps at a pixel are at the step of ray j that covers the pixel.
__device__ double pair_overlap(const RayArgs& a, int qi, int qj) {
  const int rayi = a.ring_ids[qi], rayj = a.ring_ids[qj];
  if (rayi < 0 || rayj < 0) return 0.0;
  const RayDesc ri = decode_ray(rayi, a.Du, a.Dv), rj = decode_ray(rayj, a.Du, a.Dv);
  if (ri.slice != rj.slice) return 0.0;
  const ViewGeom gi = a.views[ri.view], gj = a.views[rj.view];
  int lo, hi;
  if (!overlap_window(gi, ri, gj, rj, a.N, lo, hi)) return 0.0;
  const int* pi = a.ring_pix + (size_t)qi * a.taps;
  const double* wi = a.ring_w + (size_t)qi * a.taps;
  const int* pj = a.ring_pix + (size_t)qj * a.taps;
  const double* wj = a.ring_w + (size_t)qj * a.taps;
  const long long plane = (long long)a.N * a.N;
  double acc = 0.0;
  for (int s = lo; s <= hi; ++s) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int pix = pi[2 * s + e];
      if (pix < 0) continue;
      const int in = (int)(pix % plane);
      const int sj = gj.row_step ? in / a.N : in % a.N;   // step of ray j covering the pixel
      const double w = wi[2 * s + e];
      if (pj[2 * sj] == pix) acc += w * wj[2 * sj];
      if (pj[2 * sj + 1] == pix) acc += w * wj[2 * sj + 1];
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Sampling: ray ids of step k, i.i.d. over all rays (kind 1) or over the rays
// of the views that have arrived (kind 2: view v from step steps_per_view*v+1).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void sample_rays_kernel(RayArgs a) {
  __shared__ long long s_k;
  __shared__ int s_slot;
  __shared__ unsigned int s_avail;
  if (threadIdx.x == 0) {
    const long long k = *a.done + 1;
    const int slot = (int)((k - 1) % a.nslots);
    double lam_k = a.lam;
    if (a.ramp && k <= a.r + 1) lam_k = __ddiv_rn(__dmul_rn(a.lam, (double)(a.r + 1)), (double)k);
    long long avail = a.m;
    if (a.kind == 2) {
      long long arrived = (k - 1) / a.steps_per_view + 1;
      if (arrived > a.n_views) arrived = a.n_views;
      avail = arrived * (long long)a.Du * a.Dv;
    }
    a.info->k = k;
    a.info->slot = slot;
    a.info->view = -1;
    a.info->lam_k = lam_k;
    *a.done = k;
    s_k = k;
    s_slot = slot;
    s_avail = (unsigned int)avail;
  }
  __syncthreads();
  const unsigned long long base = (unsigned long long)(s_k - 1) * (unsigned long long)a.ell;
  for (int i = threadIdx.x; i < a.ell; i += blockDim.x)
    a.ring_ids[s_slot * a.ell + i] =
        (int)bounded32(draw64(a.seed, kStreamRays, base + (unsigned long long)i), s_avail);
  const int nr = a.dim == 3 ? a.p : a.P;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    a.rhs[i] = 0.0;
    if (a.dim == 3) a.z[i] = 0.0;
  }
}

// March the new block's rays (one warp per ray, lanes over steps), store the
// taps in the ring (voxel index and float64 weight, tap 2s/2s+1 at step s), and
// form r_k = A_k x - b_k.
template <typename T>
__global__ void __launch_bounds__(kCta) forward_rays_kernel(RayArgs a, const T* __restrict__ x,
                                                            const T* __restrict__ b) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= a.ell) return;
  const int q = a.info->slot * a.ell + w;
  const int ray = a.ring_ids[q];
  const RayDesc rd = decode_ray(ray, a.Du, a.Dv);
  const ViewGeom v = a.views[rd.view];
  const double cc = 0.5 * (double)(a.N - 1);
  const long long off = (long long)rd.slice * a.N * a.N;
  int* rp = a.ring_pix + (size_t)q * a.taps;
  double* rw = a.ring_w + (size_t)q * a.taps;
  T acc = T(0);
  for (int s = lane; s < a.N; s += 32) {
    const Tap2 tp = joseph_step(v, rd.t, cc, s);
    const int pa = tp.wa != 0.0 ? inplane_pixel(v.row_step, a.N, s, tp.minor0) : -1;
    const int pb = tp.wb != 0.0 ? inplane_pixel(v.row_step, a.N, s, tp.minor0 + 1) : -1;
    rp[2 * s] = pa >= 0 ? (int)(off + pa) : -1;
    rp[2 * s + 1] = pb >= 0 ? (int)(off + pb) : -1;
    rw[2 * s] = pa >= 0 ? tp.wa : 0.0;
    rw[2 * s + 1] = pb >= 0 ? tp.wb : 0.0;
    if (pa >= 0) acc += (T)tp.wa * x[off + pa];
    if (pb >= 0) acc += (T)tp.wb * x[off + pb];
  }
  acc = warp_sum(acc);
  if (lane == 0) a.rhs[q] = (double)(acc - b[ray]);
}

// 2D: one thread per (new ray i, ring row q): G[new_i][q] = G[q][new_i].
// The ray with the smaller ring index is the one marched, so both threads of
// a pair inside the new block compute the same value.
__global__ void gram_pairs_kernel(RayArgs a) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)a.ell * a.p) return;
  const int i = (int)(idx / a.p), q = (int)(idx % a.p);
  const int qi = a.info->slot * a.ell + i;
  const double v = pair_overlap(a, min(qi, q), max(qi, q));
  a.G[(size_t)qi * a.P + q] = v;
  a.G[(size_t)q * a.P + qi] = v;
}

// 3D: one warp per slice lists the ring rows whose ray lies in it (ring order).
__global__ void slice_collect_kernel(RayArgs a) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= a.S) return;
  int cnt = 0;
  for (int q0 = 0; q0 < a.p; q0 += 32) {
    const int q = q0 + lane;
    bool hit = false;
    if (q < a.p) {
      const int ray = a.ring_ids[q];
      hit = ray >= 0 && decode_ray(ray, a.Du, a.Dv).slice == s;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    const int pos = cnt + __popc(mask & ((1u << lane) - 1u));
    if (hit && pos < a.cap) a.slice_rows[(size_t)s * a.cap + pos] = q;
    cnt += __popc(mask);
  }
  if (lane == 0) {
    a.slice_cnt[s] = cnt;
    if (cnt > a.cap) set_status(a.status, SLIM_ENOTSUP);
  }
}

// 3D: per slice, G entries between the new block's rays and the slice's rays.
__global__ void slice_gram_kernel(RayArgs a) {
  const int s = blockIdx.x;
  const int n = min(a.slice_cnt[s], a.cap);
  const int* rows = a.slice_rows + (size_t)s * a.cap;
  const int slot = a.info->slot;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int u = idx / n, v = idx % n;
    const int qu = rows[u], qv = rows[v];
    // pairs with row u new; a pair of two new rows only once (v >= u)
    if (qu / a.ell != slot || (qv / a.ell == slot && v < u)) continue;
    const double g = pair_overlap(a, min(qu, qv), max(qu, qv));
    a.G[(size_t)qu * a.p + qv] = g;
    a.G[(size_t)qv * a.p + qu] = g;
  }
}

// 3D: per slice, K_s = lambda_k I + G_s from the stored Gram, float64
// Cholesky in shared memory, then the solves with the right-hand side
// restricted to the slice (residuals of the new block's rows, 0 elsewhere).
__global__ void slice_solve_kernel(RayArgs a) {
  extern __shared__ double smem[];
  const int s = blockIdx.x, tid = threadIdx.x;
  const int n = min(a.slice_cnt[s], a.cap);
  if (n == 0) return;
  const int ld = a.cap + 1;
  double* K = smem;                 // cap x ld
  double* y = K + (size_t)a.cap * ld;
  __shared__ double s_inv;
  const int* rows = a.slice_rows + (size_t)s * a.cap;
  const double lam = a.info->lam_k;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int u = idx / n, v = idx % n;
    K[u * ld + v] = a.G[(size_t)rows[u] * a.p + rows[v]] + (u == v ? lam : 0.0);
  }
  for (int u = tid; u < n; u += blockDim.x) y[u] = a.rhs[rows[u]];
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (tid == 0) {
      double d = K[c * ld + c];
      if (!(d > 0.0)) {
        set_status(a.status, SLIM_ENOTPD);
        d = 1.0;
      }
      const double sd = sqrt(d);
      K[c * ld + c] = sd;
      s_inv = 1.0 / sd;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = c + 1 + tid; i < n; i += blockDim.x) K[i * ld + c] *= inv;
    __syncthreads();
    const int w = n - c - 1;
    for (int idx = tid; idx < w * w; idx += blockDim.x) {
      const int i = c + 1 + idx / w, j = c + 1 + idx % w;
      if (j <= i) K[i * ld + j] -= K[i * ld + c] * K[j * ld + c];
    }
    __syncthreads();
  }
  // L y = e, then L^T z = y, by one warp
  if (tid < 32) {
    for (int i = 0; i < n; ++i) {
      double t = 0.0;
      for (int j = tid; j < i; j += 32) t += K[i * ld + j] * y[j];
      t = warp_sum(t);
      if (tid == 0) y[i] = (y[i] - t) / K[i * ld + i];
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = 0.0;
      for (int j = i + 1 + tid; j < n; j += 32) t += K[j * ld + i] * y[j];
      t = warp_sum(t);
      if (tid == 0) y[i] = (y[i] - t) / K[i * ld + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int u = tid; u < n; u += blockDim.x) a.z[rows[u]] = y[u];
}

template <typename T>
__global__ void __launch_bounds__(kCta) project_rays_kernel(const ViewGeom* views, int N, int Du,
                                                            int Dv, const int* ids, long long count,
                                                            const T* x, T* y) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= count) return;
  const int ray = ids ? ids[w] : (int)w;
  const RayDesc rd = decode_ray(ray, Du, Dv);
  const ViewGeom v = views[rd.view];
  const double cc = 0.5 * (double)(N - 1);
  const long long off = (long long)rd.slice * N * N;
  T acc = T(0);
  for (int s = lane; s < N; s += 32) {
    const Tap2 tp = joseph_step(v, rd.t, cc, s);
    const int pa = tp.wa != 0.0 ? inplane_pixel(v.row_step, N, s, tp.minor0) : -1;
    const int pb = tp.wb != 0.0 ? inplane_pixel(v.row_step, N, s, tp.minor0 + 1) : -1;
    if (pa >= 0) acc += (T)tp.wa * x[off + pa];
    if (pb >= 0) acc += (T)tp.wb * x[off + pb];
  }
  acc = warp_sum(acc);
  if (lane == 0) y[w] = acc;
}

}  // namespace

template <typename T>
cudaError_t launch_sample_rays(const RayArgs& a, cudaStream_t s) {
  sample_rays_kernel<T><<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward_rays(const RayArgs& a, T* x, const T* b, cudaStream_t s) {
  forward_rays_kernel<T><<<cdiv(a.ell, kWarpsPerCta), kCta, 0, s>>>(a, x, b);
  return cudaGetLastError();
}

cudaError_t launch_gram_pairs(const RayArgs& a, cudaStream_t s) {
  const long long total = (long long)a.ell * a.p;
  gram_pairs_kernel<<<cdiv(total, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_slice_collect(const RayArgs& a, cudaStream_t s) {
  slice_collect_kernel<<<cdiv(a.S, kWarpsPerCta), kCta, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  slice_gram_kernel<<<a.S, 256, 0, s>>>(a);
  return cudaGetLastError();
}

size_t slice_solve_smem(int cap) { return ((size_t)cap * (cap + 1) + cap) * sizeof(double); }

cudaError_t prepare_slice_solve(int cap) {
  return cudaFuncSetAttribute(slice_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)slice_solve_smem(cap));
}

cudaError_t launch_slice_solve(const RayArgs& a, cudaStream_t s) {
  slice_solve_kernel<<<a.S, 256, slice_solve_smem(a.cap), s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project_rays(const ViewGeom* views, int N, int Du, int Dv, const int* ids,
                                long long count, const T* x, T* y, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  project_rays_kernel<T><<<cdiv(count, kWarpsPerCta), kCta, 0, s>>>(views, N, Du, Dv, ids, count,
                                                                    x, y);
  return cudaGetLastError();
}

#define SLIM_RAYS_INSTANTIATE(T)                                                                 \
  template cudaError_t launch_sample_rays<T>(const RayArgs&, cudaStream_t);                      \
  template cudaError_t launch_forward_rays<T>(const RayArgs&, T*, const T*, cudaStream_t);       \
  template cudaError_t launch_project_rays<T>(const ViewGeom*, int, int, int, const int*,        \
                                              long long, const T*, T*, cudaStream_t);

SLIM_RAYS_INSTANTIATE(float)
SLIM_RAYS_INSTANTIATE(double)

}  // namespace slim
