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
  // bounds only: float32 suffices given the margin of 2 steps
  const float ci = (float)gi.co, si = (float)gi.si, cj = (float)gj.co, sj = (float)gj.si;
  const float ti = (float)ri.t, tj = (float)rj.t;
  const float det = ci * sj - si * cj;   // sin(theta_j - theta_i)
  if (fabsf(det) < 1e-5f) return true;
  const float rdet = 1.0f / det;
  const float cc = 0.5f * (float)(N - 1);
  const float sc = (gi.row_step ? (ci * tj - ti * cj) : (ti * sj - si * tj)) * rdet + cc;
  const float half = 3.0f * fabsf(rdet) + 2.0f;
  const float l = floorf(sc - half), h = ceilf(sc + half);
  if (h < 0.0f || l > (float)(N - 1)) return false;
  lo = l < 0.0f ? 0 : (int)l;
  hi = h > (float)(N - 1) ? N - 1 : (int)h;
  return lo <= hi;
}

// Overlap of ray i's two taps at step s with ray j (same slice, plane offset
// `off`), read from the stored taps: tap 2s / 2s+1 of a ray are its taps at
// step s, so ray j's taps at a pixel are at the step of ray j that covers the
// pixel.  A ray stepping along rows has the pixel's row as its step, one
// stepping along columns the column; ray i's taps at step s lie in row s or
// column s.  A row from a pixel index is an exact division by N, done as a
// multiply-high by magic_n = ceil(2^32 / N) (exact for multiples of N below
// 2^32 when N < 2^16).
__device__ __forceinline__ double taps_at_step(const int* __restrict__ pi,
                                               const double* __restrict__ wi,
                                               const int* __restrict__ pj,
                                               const double* __restrict__ wj, int s, int i_rows,
                                               int j_rows, int N, unsigned magic_n, int off) {
  const int2 pp = *reinterpret_cast<const int2*>(pi + 2 * s);
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int pix = e ? pp.y : pp.x;
    if (pix < 0) continue;
    int sj = s;                                        // same stepping axis
    if (i_rows != j_rows)
      sj = i_rows ? pix - off - s * N                  // the pixel's column
                  : (int)__umulhi((unsigned)(pix - off - s), magic_n);   // its row
    const int2 pq = *reinterpret_cast<const int2*>(pj + 2 * sj);
    if (pq.x == pix) acc += wi[2 * s + e] * wj[2 * sj];
    if (pq.y == pix) acc += wi[2 * s + e] * wj[2 * sj + 1];
  }
  return acc;
}

// The rays of ring rows qi, qj and the steps [lo, hi] of ray qi that can meet
// ray qj (hi < lo: no overlap).
struct PairWindow {
  int lo = 0, hi = -1, i_rows = 0, j_rows = 0, off = 0;
};
__device__ __forceinline__ PairWindow pair_window(const RayArgs& a, int qi, int qj) {
  PairWindow w;
  const int rayi = a.ring_ids[qi], rayj = a.ring_ids[qj];
  if (rayi < 0 || rayj < 0) return w;
  const RayDesc ri = decode_ray(rayi, a.Du, a.Dv), rj = decode_ray(rayj, a.Du, a.Dv);
  if (ri.slice != rj.slice) return w;
  const ViewGeom gi = a.views[ri.view], gj = a.views[rj.view];
  int lo, hi;
  if (!overlap_window(gi, ri, gj, rj, a.N, lo, hi)) return w;
  w.lo = lo;
  w.hi = hi;
  w.i_rows = gi.row_step;
  w.j_rows = gj.row_step;
  w.off = ri.slice * a.N * a.N;
  return w;
}

// sum_pixels a_i(pix) a_j(pix) for two rays of the ring, ray qi marched over
// its window; the steps are split over `lanes` threads starting at `lane`
// (the caller reduces the partial sums).
__device__ double pair_overlap(const RayArgs& a, int qi, int qj, int lane = 0, int lanes = 1) {
  const PairWindow w = pair_window(a, qi, qj);
  const int* pi = a.ring_pix + (size_t)qi * a.taps;
  const double* wi = a.ring_w + (size_t)qi * a.taps;
  const int* pj = a.ring_pix + (size_t)qj * a.taps;
  const double* wj = a.ring_w + (size_t)qj * a.taps;
  double acc = 0.0;
  for (int s = w.lo + lane; s <= w.hi; s += lanes)
    acc += taps_at_step(pi, wi, pj, wj, s, w.i_rows, w.j_rows, a.N, a.magic_n, w.off);
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
    const double lam_k = damping_k(a.lam, k, a.r, a.ramp, a.decay_after);
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
  if (a.distinct) {
    __shared__ int s_t[kMaxDistinctRays], s_tab[kDistinctTable];
    floyd_rays(a.seed, s_k, a.ell, s_avail, a.ring_ids + s_slot * a.ell, s_t, s_tab);
  } else {
    const unsigned long long base = (unsigned long long)(s_k - 1) * (unsigned long long)a.ell;
    for (int i = threadIdx.x; i < a.ell; i += blockDim.x)
      a.ring_ids[s_slot * a.ell + i] =
          (int)bounded32(draw64(a.seed, kStreamRays, base + (unsigned long long)i), s_avail);
  }
  const int nr = a.dense ? a.P : a.p;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    a.rhs[i] = 0.0;
    if (!a.dense) a.z[i] = 0.0;
  }
}

// March the new block's rays (one warp per ray, lanes over steps), store the
// taps in the ring (voxel index and float64 weight, tap 2s/2s+1 at step s), and
// form r_k = A_k x - b_k.
template <typename T>
__global__ void __launch_bounds__(kCta) forward_rays_kernel(RayArgs a, const T* __restrict__ x,
                                                            const T* __restrict__ b) {
  // a group of a.lanes threads per ray (a warp holds 32 / a.lanes rays); every
  // lane of the warp takes part in the group reductions
  const int L = a.lanes;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = gt / L, lane = gt % L;
  const bool active = w < a.ell;
  const int q = active ? a.info->slot * a.ell + w : 0;
  T acc = T(0);
  if (active) {
    const int ray = a.ring_ids[q];
    const RayDesc rd = decode_ray(ray, a.Du, a.Dv);
    const ViewGeom v = a.views[rd.view];
    const double cc = 0.5 * (double)(a.N - 1);
    const long long off = (long long)rd.slice * a.N * a.N;
    int* rp = a.ring_pix + (size_t)q * a.taps;
    double* rw = a.ring_w + (size_t)q * a.taps;
    for (int s = lane; s < a.N; s += L) {
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
  }
  for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, L);
  if (active && lane == 0) a.rhs[q] = (double)(acc - b[a.ring_ids[q]]);
}

// 2D: G[new_i][q] = G[q][new_i] for every ring row q, a thread per pair
// (i, q) marching the new ray i over its overlap window with ray q.  Windows
// longer than a.short_window steps (near-parallel rays, and the diagonal) go
// to the whole warp afterwards, one at a time, with the steps split over the
// lanes.  A pair of two new rows is computed once, by the thread of the
// smaller ring index, which writes both entries.
__global__ void __launch_bounds__(kCta) gram_pairs_kernel(RayArgs a) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int base = a.info->slot * a.ell;
  int qi = 0, q = 0;
  bool mine = false;
  PairWindow w;
  if (idx < (long long)a.ell * a.p) {
    qi = base + (int)(idx / a.p);
    q = (int)(idx % a.p);
    mine = q < base || q >= base + a.ell || q >= qi;
    if (mine) w = pair_window(a, qi, q);
  }
  const bool longw = w.hi - w.lo + 1 > a.short_window;
  double acc = 0.0;
  if (!longw) {
    const int* pi = a.ring_pix + (size_t)qi * a.taps;
    const double* wi = a.ring_w + (size_t)qi * a.taps;
    const int* pj = a.ring_pix + (size_t)q * a.taps;
    const double* wj = a.ring_w + (size_t)q * a.taps;
    for (int s = w.lo; s <= w.hi; ++s)
      acc += taps_at_step(pi, wi, pj, wj, s, w.i_rows, w.j_rows, a.N, a.magic_n, w.off);
  }
  unsigned pending = __ballot_sync(0xffffffffu, longw);
  while (pending) {
    const int src = __ffs(pending) - 1;
    pending &= pending - 1;
    const int sqi = __shfl_sync(0xffffffffu, qi, src), sq = __shfl_sync(0xffffffffu, q, src);
    const int lo = __shfl_sync(0xffffffffu, w.lo, src), hi = __shfl_sync(0xffffffffu, w.hi, src);
    const int ir = __shfl_sync(0xffffffffu, w.i_rows, src);
    const int jr = __shfl_sync(0xffffffffu, w.j_rows, src);
    const int off = __shfl_sync(0xffffffffu, w.off, src);
    const int* pi = a.ring_pix + (size_t)sqi * a.taps;
    const double* wi = a.ring_w + (size_t)sqi * a.taps;
    const int* pj = a.ring_pix + (size_t)sq * a.taps;
    const double* wj = a.ring_w + (size_t)sq * a.taps;
    double v = 0.0;
    for (int s = lo + lane; s <= hi; s += 32)
      v += taps_at_step(pi, wi, pj, wj, s, ir, jr, a.N, a.magic_n, off);
    v = warp_sum(v);
    if (lane == src) acc = v;
  }
  if (mine) {
    a.G[(size_t)qi * a.P + q] = acc;
    a.G[(size_t)q * a.P + qi] = acc;
  }
}

// 3D: bucket the ring rows by z-slice (one thread per row; the order inside
// a bucket is fixed afterwards by slice_gram_kernel, which sorts it).
__global__ void slice_fill_kernel(RayArgs a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.p) return;
  const int ray = a.ring_ids[q];
  if (ray < 0) return;
  const int s = decode_ray(ray, a.Du, a.Dv).slice;
  const int pos = atomicAdd(&a.slice_cnt[s], 1);
  if (pos < a.cap) a.slice_rows[(size_t)s * a.cap + pos] = q;
}

// 3D: per slice, G entries between the new block's rays and the slice's rays;
// one warp per pair, lanes splitting the overlap window.  The slice's rows and
// the positions of its new rows are staged in shared memory first, so warps
// walk only the (new, member) pairs.
constexpr int kSliceCapMax = 128;
__global__ void __launch_bounds__(kCta) slice_gram_kernel(RayArgs a) {
  __shared__ int srows[kSliceCapMax], snew[kSliceCapMax];
  __shared__ int s_nnew;
  __shared__ int sraw[kSliceCapMax];
  const int s = blockIdx.x;
  const int cnt = a.slice_cnt[s];
  const int n = min(cnt, a.cap);
  const int slot = a.info->slot;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0 && cnt > a.cap) set_status(a.status, SLIM_ENOTSUP);
  for (int u = threadIdx.x; u < n; u += blockDim.x) sraw[u] = a.slice_rows[(size_t)s * a.cap + u];
  __syncthreads();
  // ring order inside the slice (ring rows are distinct): rank sort
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    const int key = sraw[u];
    int rank = 0;
    for (int v = 0; v < n; ++v) rank += sraw[v] < key;
    srows[rank] = key;
  }
  __syncthreads();
  for (int u = threadIdx.x; u < n; u += blockDim.x) a.slice_rows[(size_t)s * a.cap + u] = srows[u];
  if (wib == 0) {
    int cnt = 0;
    for (int u0 = 0; u0 < n; u0 += 32) {
      const int u = u0 + lane;
      const bool isnew = u < n && srows[u] / a.ell == slot;
      const unsigned mask = __ballot_sync(0xffffffffu, isnew);
      if (isnew) snew[cnt + __popc(mask & ((1u << lane) - 1u))] = u;
      cnt += __popc(mask);
    }
    if (lane == 0) s_nnew = cnt;
  }
  __syncthreads();
  const int total = s_nnew * n;
  for (int t = wib; t < total; t += kWarpsPerCta) {
    const int u = snew[t / n], v = t % n;
    const int qu = srows[u], qv = srows[v];
    if (qv / a.ell == slot && v < u) continue;    // a pair of two new rows only once
    double g = pair_overlap(a, min(qu, qv), max(qu, qv), lane, 32);
    g = warp_sum(g);
    if (lane == 0) {
      a.G[(size_t)qu * a.p + qv] = g;
      a.G[(size_t)qv * a.p + qu] = g;
    }
  }
}


// 3D: one CTA of 4 warps per slice: K_s = lambda_k I + G_s from the stored
// Gram, float64 Cholesky in shared memory (one pivot reciprocal per column,
// rows of the trailing update split over 4 threads each), then L y = e and
// L^T z = y with e the residuals of the slice's new rows.
constexpr int kSolveThreads = 128;
__global__ void __launch_bounds__(kSolveThreads) slice_solve_kernel(RayArgs a) {
  extern __shared__ double smem[];
  const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  const int n = min(a.slice_cnt[s], a.cap);
  if (n == 0) return;
  const int ld = a.cap + 1;
  double* K = smem;                 // cap x ld
  double* y = K + (size_t)a.cap * ld;
  double* rdiag = y + a.cap;        // 1/L[c][c]
  const int* rows = a.slice_rows + (size_t)s * a.cap;
  const double lam = a.info->lam_k;
  for (int idx = tid; idx < n * n; idx += kSolveThreads) {
    const int u = idx / n, v = idx % n;
    if (v <= u) K[u * ld + v] = a.G[(size_t)rows[u] * a.p + rows[v]] + (u == v ? lam : 0.0);
  }
  for (int u = tid; u < n; u += kSolveThreads) y[u] = a.rhs[rows[u]];
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (tid == 0) {
      const double d = K[c * ld + c];
      const double inv = rsqrt_pivot(d, a.status);
      K[c * ld + c] = d > 0.0 ? d * inv : 1.0;   // sqrt(d) = d / sqrt(d)
      rdiag[c] = inv;
    }
    __syncthreads();
    const double inv = rdiag[c];
    for (int i = c + 1 + tid; i < n; i += kSolveThreads) K[i * ld + c] *= inv;
    __syncthreads();
    for (int i = c + 1 + (tid >> 2); i < n; i += kSolveThreads / 4) {
      const double lic = K[i * ld + c];
      for (int j = c + 1 + (tid & 3); j <= i; j += 4) K[i * ld + j] -= lic * K[j * ld + c];
    }
    __syncthreads();
  }
  if (tid < 32) {
    for (int i = 0; i < n; ++i) {
      double t = 0.0;
      for (int j = lane; j < i; j += 32) t += K[i * ld + j] * y[j];
      t = warp_sum(t);
      if (lane == 0) y[i] = (y[i] - t) * rdiag[i];
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = 0.0;
      for (int j = i + 1 + lane; j < n; j += 32) t += K[j * ld + i] * y[j];
      t = warp_sum(t);
      if (lane == 0) y[i] = (y[i] - t) * rdiag[i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int u = tid; u < n; u += kSolveThreads) a.z[rows[u]] = y[u];
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

// Full-view forward projection in the per-slice geometry (views rotating
// about z, det_v = N): ray (a, v, u) lies in slice v and its in-plane taps do
// not depend on v.  A CTA takes kFvRays consecutive bins of one view, marches
// their taps once (the float64 Joseph steps every kernel uses, so the same
// weights) into shared memory, and applies them to all N slices: one march
// serves N x kFvRays rays.  The taps are laid out so that lanes run along the
// image's contiguous axis: across the bins for row-stepping views (adjacent
// bins meet adjacent pixels of one row), along the steps for column-stepping
// views (adjacent steps are adjacent pixels of one row).
constexpr int kFvRays = 16;

__host__ __device__ inline size_t fullview_smem(int N, int elem) {
  return (size_t)N * kFvRays * (2 * sizeof(int) + 2 * (size_t)elem);
}

template <typename T>
__global__ void __launch_bounds__(256) project_fullview_kernel(const ViewGeom* views, int N,
                                                               int Du, const T* x, T* y) {
  extern __shared__ __align__(16) unsigned char fv_smem[];
  int2* s_pix = reinterpret_cast<int2*>(fv_smem);                       // [N * kFvRays]
  T* s_w = reinterpret_cast<T*>(s_pix + (size_t)N * kFvRays);           // [N * kFvRays * 2]
  const int tiles = (Du + kFvRays - 1) / kFvRays;
  const int a = blockIdx.x / tiles, u0 = (blockIdx.x % tiles) * kFvRays;
  const ViewGeom v = views[a];
  const bool rows = v.row_step != 0;
  // tap slot of (step s, ray r)
  auto slot = [&](int s, int r) { return rows ? s * kFvRays + r : r * N + s; };
  const double cc = 0.5 * (double)(N - 1);
  for (int e = threadIdx.x; e < N * kFvRays; e += blockDim.x) {
    const int s = e / kFvRays, r = e % kFvRays, u = u0 + r;
    int2 px = make_int2(-1, -1);
    T wa = T(0), wb = T(0);
    if (u < Du) {
      const double t = (double)u - 0.5 * (double)(Du - 1);
      const Tap2 tp = joseph_step(v, t, cc, s);
      px.x = tp.wa != 0.0 ? inplane_pixel(v.row_step, N, s, tp.minor0) : -1;
      px.y = tp.wb != 0.0 ? inplane_pixel(v.row_step, N, s, tp.minor0 + 1) : -1;
      wa = (T)tp.wa;
      wb = (T)tp.wb;
    }
    const int q = slot(s, r);
    s_pix[q] = px;
    s_w[2 * q] = wa;
    s_w[2 * q + 1] = wb;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long long NN = (long long)N * N;
  if (rows) {
    // half-warps over the 16 bins, the two halves over even and odd steps
    const int r = lane & 15, ph = lane >> 4, u = u0 + r;
    for (int sl = warp; sl < N; sl += nw) {
      const T* xs = x + sl * NN;
      T acc = T(0);
      for (int s = ph; s < N; s += 2) {
        const int q = s * kFvRays + r;
        const int2 px = s_pix[q];
        if (px.x >= 0) acc += s_w[2 * q] * xs[px.x];
        if (px.y >= 0) acc += s_w[2 * q + 1] * xs[px.y];
      }
      acc += __shfl_down_sync(0xffffffffu, acc, 16);
      if (ph == 0 && u < Du) y[((long long)a * N + sl) * Du + u] = acc;
    }
  } else {
    // a warp per (slice, bin), lanes over the steps
    for (int w = warp; w < N * kFvRays; w += nw) {
      const int sl = w / kFvRays, r = w % kFvRays, u = u0 + r;
      if (u >= Du) continue;
      const T* xs = x + sl * NN;
      T acc = T(0);
      for (int s = lane; s < N; s += 32) {
        const int q = r * N + s;
        const int2 px = s_pix[q];
        if (px.x >= 0) acc += s_w[2 * q] * xs[px.x];
        if (px.y >= 0) acc += s_w[2 * q + 1] * xs[px.y];
      }
      acc = warp_sum(acc);
      if (lane == 0) y[((long long)a * N + sl) * Du + u] = acc;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_sample_rays(const RayArgs& a, cudaStream_t s) {
  sample_rays_kernel<T><<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward_rays(const RayArgs& a, T* x, const T* b, cudaStream_t s) {
  forward_rays_kernel<T><<<cdiv((long long)a.ell * a.lanes, kCta), kCta, 0, s>>>(a, x, b);
  return cudaGetLastError();
}

cudaError_t launch_gram_pairs(const RayArgs& a, cudaStream_t s) {
  const long long total = (long long)a.ell * a.p;
  gram_pairs_kernel<<<cdiv(total, kCta), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_slice_collect(const RayArgs& a, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.slice_cnt, 0, (size_t)a.S * sizeof(int), s);
  if (e != cudaSuccess) return e;
  slice_fill_kernel<<<cdiv(a.p, 256), 256, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  slice_gram_kernel<<<a.S, kCta, 0, s>>>(a);
  return cudaGetLastError();
}

size_t slice_solve_smem(int cap) { return ((size_t)cap * (cap + 1) + 2 * (size_t)cap) * sizeof(double); }

cudaError_t prepare_slice_solve(int cap) {
  return cudaFuncSetAttribute(slice_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)slice_solve_smem(cap));
}

cudaError_t launch_slice_solve(const RayArgs& a, cudaStream_t s) {
  slice_solve_kernel<<<a.S, kSolveThreads, slice_solve_smem(a.cap), s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project_rays(const ViewGeom* views, int N, int Du, int Dv, const int* ids,
                                long long count, const T* x, T* y, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t fv = fullview_smem(N, sizeof(T));
  if (!ids && Dv == N && fv <= 200 * 1024 && count % ((long long)Du * Dv) == 0) {
    // every ray of every view in order: the taps of a bin serve all N slices
    cudaError_t e = cudaFuncSetAttribute(project_fullview_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fv);
    if (e != cudaSuccess) return e;
    const long long views_n = count / ((long long)Du * Dv);
    const long long grid = views_n * ((Du + kFvRays - 1) / kFvRays);
    project_fullview_kernel<T><<<(unsigned)grid, 256, fv, s>>>(views, N, Du, x, y);
    return cudaGetLastError();
  }
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
