// Per-step kernels of the slimLS iteration (Eq. (ram) with the Woodbury form of Eq. (B_k)).
#include <algorithm>
#include <cuda_bf16.h>

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
  __shared__ int s_perm[kMaxCyclicViews];
  const long long k0 = *a.done + 1;
  const int cview = a.cyclic ? cyclic_view(a.seed, k0, a.n_views, a.perm, a.perm_epoch, s_perm) : 0;
  __syncthreads();   // every thread has read the step counter
  if (threadIdx.x == 0) {
    long long k = k0;
    int view = a.cyclic ? cview
                        : (int)bounded32(draw64(a.seed, kStreamBlocks, (unsigned long long)(k - 1)),
                                         (uint32_t)a.n_views);
    int slot = (int)((k - 1) % a.nslots);
    double lam_k = damping_k(a.lam, k, a.r, a.ramp, a.decay_after);
    double tik_c = 0.0;
    if (a.tik_beta > 0.0) {
      // Eq. (slimTik): mu_k = lambda_k + c_k lam_tik^2 / M
      const long long cnt = a.tik_reading ? a.r : (k < a.r + 1 ? k : a.r + 1);
      lam_k = __dadd_rn(lam_k, __dmul_rn((double)cnt, a.tik_beta));
      tik_c = __ddiv_rn(a.tik_beta, lam_k);
    }
    a.info->k = k;
    a.info->slot = slot;
    a.info->view = view;
    a.info->lam_k = lam_k;
    a.info->tik_c = tik_c;
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

__device__ __forceinline__ float csr_value(const void* val, int bf16, long long e) {
  return bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(val)[e])
              : reinterpret_cast<const float*>(val)[e];
}

// Step 2 with stored rows: the new block's rows come from the CSR instead of
// the projector.  Ring taps take the stored values (as float64); map slots are
// claimed in order (a pixel is in at most two rows of one view).
template <typename T>
__global__ void __launch_bounds__(kCta) csr_forward_residual_kernel(StepArgs<T> a) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= a.ell) return;
  const int q = a.info->slot * a.ell + w;
  const int ray = a.ring_ids[q];
  const int e0 = a.csr_ptr[ray], len = a.csr_ptr[ray + 1] - e0;
  int* rp = a.ring_pix + (size_t)q * a.taps;
  double* rw = a.ring_w + (size_t)q * a.taps;
  const long long n = a.n;
  T acc = T(0);
  for (int t = lane; t < a.taps; t += 32) {
    if (t >= len) {
      rp[t] = -1;
      rw[t] = 0.0;
      continue;
    }
    const int pix = a.csr_col[e0 + t];
    const double wv = (double)csr_value(a.csr_val, a.csr_bf16, e0 + t);
    rp[t] = pix;
    rw[t] = wv;
    acc += (T)wv * a.x[pix];
    if (atomicCAS(&a.map_ray[pix], -1, w) == -1) {
      a.map_w[pix] = wv;
    } else if (atomicCAS(&a.map_ray[n + pix], -1, w) == -1) {
      a.map_w[n + pix] = wv;
    } else {
      set_status(a.status, SLIM_EINVAL);
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) a.rhs[q] = (double)(acc - a.b[ray]);
}

// ---------------------------------------------------------------------------
// Building the stored matrix
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCta) csr_count_kernel(const ViewGeom* views, int N, int D,
                                                         long long m, int* counts) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const int ray = (int)w, view = ray / D, d = ray - view * D;
  const ViewGeom v = views[view];
  const double cc = 0.5 * (double)(N - 1), t = (double)d - 0.5 * (double)(D - 1);
  int cnt = 0;
  for (int s = lane; s < N; s += 32) {
    Tap2 tp = joseph_step(v, t, cc, s);
    cnt += (tp.wa != 0.0 && inplane_pixel(v.row_step, N, s, tp.minor0) >= 0);
    cnt += (tp.wb != 0.0 && inplane_pixel(v.row_step, N, s, tp.minor0 + 1) >= 0);
  }
  cnt = warp_sum(cnt);
  if (lane == 0) counts[ray] = cnt;
}

// Exclusive scan of n counts into ptr[0..n] by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) scan_kernel(const int* counts, int* ptr, long long n,
                                                    long long* total) {
  __shared__ long long part[1024];
  const int tid = threadIdx.x;
  const long long chunk = (n + 1023) / 1024;
  const long long lo = tid * chunk, hi = min(n, lo + chunk);
  long long sum = 0;
  for (long long i = lo; i < hi; ++i) sum += counts[i];
  part[tid] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    long long v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  long long run = part[tid] - sum;   // exclusive prefix of this chunk
  for (long long i = lo; i < hi; ++i) {
    ptr[i] = (int)run;
    run += counts[i];
  }
  if (tid == 1023) {
    ptr[n] = (int)part[1023];
    *total = part[1023];
  }
}

// Fill the CSR rows in march order (tap a then tap b per step), as the oracle does.
__global__ void __launch_bounds__(kCta) csr_fill_kernel(const ViewGeom* views, int N, int D,
                                                        long long m, const int* row_ptr, int* col,
                                                        void* val, int bf16) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const int ray = (int)w, view = ray / D, d = ray - view * D;
  const ViewGeom v = views[view];
  const double cc = 0.5 * (double)(N - 1), t = (double)d - 0.5 * (double)(D - 1);
  int pos = row_ptr[ray];
  for (int s0 = 0; s0 < N; s0 += 32) {
    const int s = s0 + lane;
    int pa = -1, pb = -1;
    double wa = 0.0, wb = 0.0;
    if (s < N) {
      Tap2 tp = joseph_step(v, t, cc, s);
      if (tp.wa != 0.0) pa = inplane_pixel(v.row_step, N, s, tp.minor0);
      if (tp.wb != 0.0) pb = inplane_pixel(v.row_step, N, s, tp.minor0 + 1);
      wa = tp.wa;
      wb = tp.wb;
    }
    const int c = (pa >= 0) + (pb >= 0);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int e = pos + incl - c;
    if (pa >= 0) {
      col[e] = pa;
      if (bf16) reinterpret_cast<__nv_bfloat16*>(val)[e] = __float2bfloat16_rn((float)wa);
      else reinterpret_cast<float*>(val)[e] = (float)wa;
      ++e;
    }
    if (pb >= 0) {
      col[e] = pb;
      if (bf16) reinterpret_cast<__nv_bfloat16*>(val)[e] = __float2bfloat16_rn((float)wb);
      else reinterpret_cast<float*>(val)[e] = (float)wb;
    }
    pos += __shfl_sync(0xffffffffu, incl, 31);
  }
}

__global__ void csc_count_kernel(const int* col, long long nnz, int* ccount) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
       e += (long long)gridDim.x * blockDim.x)
    atomicAdd(&ccount[col[e]], 1);
}

__global__ void __launch_bounds__(kCta) csc_fill_kernel(long long m, const int* row_ptr,
                                                        const int* col, const void* val, int bf16,
                                                        int* cursor, int* crow, void* cval) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  for (int e = row_ptr[w] + lane; e < row_ptr[w + 1]; e += 32) {
    const int j = col[e];
    const int pos = atomicAdd(&cursor[j], 1);
    crow[pos] = (int)w;
    if (bf16) reinterpret_cast<__nv_bfloat16*>(cval)[pos] = reinterpret_cast<const __nv_bfloat16*>(val)[e];
    else reinterpret_cast<float*>(cval)[pos] = reinterpret_cast<const float*>(val)[e];
  }
}

// ---------------------------------------------------------------------------
// Full passes over the stored matrix (HBM streams of the index and value
// arrays; x or y gathers stay in L2).  One warp per output row (column for
// the transpose); lanes read consecutive entries; streaming loads bypass L1.
// ---------------------------------------------------------------------------
template <typename T, bool BF16>
__global__ void __launch_bounds__(kCta) spmv_kernel(const int* __restrict__ ptr,
                                                    const int* __restrict__ idx,
                                                    const void* __restrict__ val,
                                                    const int* __restrict__ rows, long long count,
                                                    const T* __restrict__ x, T* __restrict__ y,
                                                    int accumulate) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // the CTA's consecutive rows take their pointers from one coalesced load
  __shared__ int sptr[kWarpsPerCta + 1];
  if (!rows) {
    const long long row0 = (long long)blockIdx.x * kWarpsPerCta;
    if (threadIdx.x <= kWarpsPerCta && row0 + threadIdx.x <= count)
      sptr[threadIdx.x] = __ldg(ptr + row0 + threadIdx.x);
    __syncthreads();
  }
  if (w >= count) return;
  const int r = rows ? rows[w] : (int)w;
  const int e0 = rows ? __ldg(ptr + r) : sptr[wib];
  const int e1 = rows ? __ldg(ptr + r + 1) : sptr[wib + 1];
  // each lane takes 4 consecutive entries per chunk from a 4-aligned base, so
  // index and value loads are 16-byte (8-byte for bfloat16) vectors; entries
  // outside [e0, e1) are masked.  The loads of up to kBatch chunks are issued
  // before any dependent gather of x, to keep enough bytes in flight.
  constexpr int kBatch = 4;
  T acc = T(0);
  for (int base0 = (e0 & ~3) + 4 * lane; base0 - 4 * lane < e1; base0 += 128 * kBatch) {
    int4 j4[kBatch];
    float v[kBatch][4];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int base = base0 + 128 * b;
      if (base < e1) {
        j4[b] = __ldcs(reinterpret_cast<const int4*>(idx + base));
        if constexpr (BF16) {
          const uint2 raw = __ldcs(reinterpret_cast<const uint2*>(
              reinterpret_cast<const unsigned short*>(val) + base));
          v[b][0] = __uint_as_float(raw.x << 16);
          v[b][1] = __uint_as_float(raw.x & 0xffff0000u);
          v[b][2] = __uint_as_float(raw.y << 16);
          v[b][3] = __uint_as_float(raw.y & 0xffff0000u);
        } else {
          const float4 f =
              __ldcs(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(val) + base));
          v[b][0] = f.x; v[b][1] = f.y; v[b][2] = f.z; v[b][3] = f.w;
        }
      } else {
        j4[b] = make_int4(0, 0, 0, 0);
        v[b][0] = v[b][1] = v[b][2] = v[b][3] = 0.f;
      }
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int base = base0 + 128 * b;
      const int jj[4] = {j4[b].x, j4[b].y, j4[b].z, j4[b].w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = base + t;
        if (e >= e0 && e < e1) acc += (T)v[b][t] * __ldg(x + jj[t]);
      }
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) y[w] = accumulate ? y[w] + acc : acc;
}

// Sort each CSC column by row id (one warp per column, rank sort in shared
// memory; a ray taps a pixel at most once, so row ids in a column are distinct).
constexpr int kSortCap = 1024;   // longest column handled (2 x views)
__global__ void __launch_bounds__(128) csc_sort_kernel(const int* col_ptr, int* row, void* cval,
                                                       int bf16, long long n) {
  __shared__ int srow[4][kSortCap];
  __shared__ unsigned int sval[4][kSortCap];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long j = (long long)blockIdx.x * 4 + wib;
  if (j >= n) return;
  const int e0 = col_ptr[j], len = col_ptr[j + 1] - e0;
  if (len > kSortCap) return;
  for (int i = lane; i < len; i += 32) {
    srow[wib][i] = row[e0 + i];
    sval[wib][i] = bf16 ? (unsigned int)reinterpret_cast<const unsigned short*>(cval)[e0 + i]
                        : __float_as_uint(reinterpret_cast<const float*>(cval)[e0 + i]);
  }
  __syncwarp();
  for (int i = lane; i < len; i += 32) {
    const int key = srow[wib][i];
    int rank = 0;
    for (int k = 0; k < len; ++k) rank += srow[wib][k] < key;
    row[e0 + rank] = key;
    if (bf16) reinterpret_cast<unsigned short*>(cval)[e0 + rank] = (unsigned short)sval[wib][i];
    else reinterpret_cast<float*>(cval)[e0 + rank] = __uint_as_float(sval[wib][i]);
  }
}

// Slice lengths (longest line of each 32-line slice) and the SELL fill.
__global__ void sell_len_kernel(const int* ptr, long long lines, int* slen) {
  const long long sidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long slices = (lines + 31) / 32;
  if (sidx >= slices) return;
  int mx = 0;
  for (int l = 0; l < 32; ++l) {
    const long long r = sidx * 32 + l;
    if (r < lines) mx = max(mx, ptr[r + 1] - ptr[r]);
  }
  slen[sidx] = 32 * mx;
}

__global__ void __launch_bounds__(kCta) sell_fill_kernel(const int* ptr, const int* idx,
                                                         const void* val, int bf16, long long lines,
                                                         const int* slice_ptr, int* sidx,
                                                         void* sval) {
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long slices = (lines + 31) / 32;
  if (s >= slices) return;
  const long long r = s * 32 + lane;
  const int e0 = r < lines ? ptr[r] : 0, len = r < lines ? ptr[r + 1] - e0 : 0;
  const int depth = (slice_ptr[s + 1] - slice_ptr[s]) / 32;
  for (int k = 0; k < depth; ++k) {
    const long long o = slice_ptr[s] + 32LL * k + lane;
    const bool ok = k < len;
    sidx[o] = ok ? idx[e0 + k] : 0;
    if (bf16) reinterpret_cast<unsigned short*>(sval)[o] =
        ok ? reinterpret_cast<const unsigned short*>(val)[e0 + k] : (unsigned short)0;
    else reinterpret_cast<float*>(sval)[o] = ok ? reinterpret_cast<const float*>(val)[e0 + k] : 0.f;
  }
}

// Full pass over a SELL-32 copy: one slice per CTA of 4 warps; lane l owns
// line l of the slice and warp w takes entries k = w, w+4, ...; loads are
// 128-byte coalesced and the gathers of 32 adjacent rays (pixels) at the same
// step hit neighbouring addresses.
template <typename T, bool BF16>
__global__ void __launch_bounds__(128) sell_spmv_kernel(const int* __restrict__ slice_ptr,
                                                        const int* __restrict__ idx,
                                                        const void* __restrict__ val,
                                                        long long lines, const T* __restrict__ x,
                                                        T* __restrict__ y, int accumulate) {
  __shared__ T part[4][32];
  const long long s = blockIdx.x;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o0 = __ldg(slice_ptr + s), depth = (__ldg(slice_ptr + s + 1) - o0) / 32;
  T acc = T(0);
  int k = wib;
#pragma unroll 1
  for (; k + 12 < depth; k += 16) {
    int j[4];
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long o = o0 + 32LL * (k + 4 * u) + lane;
      j[u] = __ldcs(idx + o);
      if constexpr (BF16) v[u] = __uint_as_float(((unsigned)__ldcs(reinterpret_cast<const unsigned short*>(val) + o)) << 16);
      else v[u] = __ldcs(reinterpret_cast<const float*>(val) + o);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc += (T)v[u] * __ldg(x + j[u]);
  }
  for (; k < depth; k += 4) {
    const long long o = o0 + 32LL * k + lane;
    const int jj = __ldcs(idx + o);
    float vv;
    if constexpr (BF16) vv = __uint_as_float(((unsigned)__ldcs(reinterpret_cast<const unsigned short*>(val) + o)) << 16);
    else vv = __ldcs(reinterpret_cast<const float*>(val) + o);
    acc += (T)vv * __ldg(x + jj);
  }
  part[wib][lane] = acc;
  __syncthreads();
  if (wib == 0) {
    const long long r = s * 32 + lane;
    const T t = part[0][lane] + part[1][lane] + part[2][lane] + part[3][lane];
    if (r < lines) y[r] = accumulate ? y[r] + t : t;
  }
}

// x += A_rows^T y through the stored rows (atomics), for a ray subset.
template <typename T, bool BF16>
__global__ void __launch_bounds__(kCta) csr_scatter_kernel(const int* ptr, const int* idx,
                                                           const void* val, const int* rows,
                                                           int count, const T* y, T* x) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= count) return;
  const int r = rows[w];
  const T yv = y[w];
  for (int e = ptr[r] + lane; e < ptr[r + 1]; e += 32) {
    float v;
    if constexpr (BF16) {
      v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(val)[e]);
    } else {
      v = reinterpret_cast<const float*>(val)[e];
    }
    atomicAdd(&x[idx[e]], (T)v * yv);
  }
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
      if (a.cinv) wq *= a.cinv[pix];   // M C^{-1} M^T (slimTik, diagonal C)
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
  // a group of a.lanes threads per ring row (no group reductions: early exit is safe)
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = gt / a.lanes, lane = gt % a.lanes;
  if (q >= a.p || a.ring_ids[q] < 0) return;
  const bool is_new = (q / a.ell) == a.info->slot;
  // sg: x -= eta alpha_k A_k^T r_k, alpha_k = 1/lambda_k
  const double zq = a.sg ? a.rhs[q] * (1.0 / a.info->lam_k) : a.z[q];
  const T c = (T)(-a.eta * zq);
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  const double* rw = a.ring_w + (size_t)q * a.taps;
  const long long n = a.n;
  for (int t = lane; t < a.taps; t += a.lanes) {
    int pix = rp[t];
    if (pix < 0) continue;
    if (c != T(0)) atomicAdd(&a.x[pix], c * (T)(a.cinv ? rw[t] * a.cinv[pix] : rw[t]));
    if (is_new && a.map_ray) {
      a.map_ray[pix] = -1;
      a.map_ray[n + pix] = -1;
    }
  }
}

// ---------------------------------------------------------------------------
// slimTik (Eq. slimTik, C_k = diag(c)).  With W = C^{-1} and beta = lam_tik^2/M
// the step is s = (beta/mu) x + W M^T z, (mu I + M W M^T) z = c - (beta/mu) M x,
// c = [0; ...; r_k]: the right-hand side takes the window's projection of
// x_{k-1}, and x_k = (1 - eta beta/mu) x_{k-1} - eta W M^T z.
// One warp per ring row.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kCta) tik_rhs_kernel(StepArgs<T> a) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= a.p || a.ring_ids[q] < 0) return;
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  const double* rw = a.ring_w + (size_t)q * a.taps;
  double acc = 0.0;
  for (int t = lane; t < a.taps; t += 32) {
    const int pix = rp[t];
    if (pix >= 0) acc += rw[t] * (double)a.x[pix];
  }
  acc = warp_sum(acc);
  if (lane == 0) a.rhs[q] -= a.info->tik_c * acc;
}

template <typename T>
__global__ void tik_scale_kernel(StepArgs<T> a) {
  const T f = (T)(1.0 - a.eta * a.info->tik_c);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x)
    a.x[i] *= f;
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
  if (a.csr_ptr)
    csr_forward_residual_kernel<T><<<cdiv(a.ell, kWarpsPerCta), kCta, 0, s>>>(a);
  else
    forward_residual_kernel<T><<<cdiv(a.ell, kWarpsPerCta), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

// SELL-32 copy of a CSR-like (ptr, idx, val) matrix with `lines` lines;
// `scratch` holds at least (lines+31)/32 + 1 ints.
cudaError_t build_sell(const int* ptr, const int* idx, const void* val, int bf16, long long lines,
                       int* scratch, long long* d_total, Sell* out, cudaStream_t s) {
  const size_t vs = bf16 ? 2 : 4;
  const long long slices = (lines + 31) / 32;
  cudaError_t e;
  out->lines = lines;
  if ((e = cudaMalloc(&out->slice_ptr, (size_t)(slices + 1) * sizeof(int))) != cudaSuccess) return e;
  sell_len_kernel<<<cdiv(slices, 256), 256, 0, s>>>(ptr, lines, scratch);
  scan_kernel<<<1, 1024, 0, s>>>(scratch, out->slice_ptr, slices, d_total);
  long long stored = 0;
  if ((e = cudaMemcpyAsync(&stored, d_total, sizeof(stored), cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if (stored >= (1LL << 31)) return cudaErrorInvalidValue;
  out->stored = stored;
  if ((e = cudaMalloc(&out->idx, (size_t)stored * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&out->val, (size_t)stored * vs)) != cudaSuccess) return e;
  sell_fill_kernel<<<cdiv(slices, kWarpsPerCta), kCta, 0, s>>>(ptr, idx, val, bf16, lines,
                                                               out->slice_ptr, out->idx, out->val);
  return cudaGetLastError();
}

void free_sell(Sell* a) {
  if (a->slice_ptr) cudaFree(a->slice_ptr);
  if (a->idx) cudaFree(a->idx);
  if (a->val) cudaFree(a->val);
  *a = Sell{};
}

cudaError_t build_csr(const ViewGeom* views, int N, int D, long long m, long long n, int bf16,
                      CsrStore* st, cudaStream_t s) {
  *st = CsrStore{};
  st->bf16 = bf16;
  const size_t vs = bf16 ? 2 : 4;
  int* counts = nullptr;
  long long* d_total = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc(&counts, (size_t)(std::max(m, n) + 1) * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&d_total, sizeof(long long))) != cudaSuccess) { cudaFree(counts); return e; }
  auto done = [&](cudaError_t err) { cudaFree(counts); cudaFree(d_total); return err; };
  if ((e = cudaMalloc(&st->row_ptr, (size_t)(m + 1) * sizeof(int))) != cudaSuccess) return done(e);
  csr_count_kernel<<<cdiv(m, kWarpsPerCta), kCta, 0, s>>>(views, N, D, m, counts);
  scan_kernel<<<1, 1024, 0, s>>>(counts, st->row_ptr, m, d_total);
  if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
  long long nnz = 0;
  if ((e = cudaMemcpyAsync(&nnz, d_total, sizeof(nnz), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return done(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return done(e);
  if (nnz >= (1LL << 31)) return done(cudaErrorInvalidValue);
  st->nnz = nnz;
  // a row of at most 2N - 3 entries lies in one aligned window of 2N entries
  st->max_row = 2 * N;
  // arrays padded by 4 entries: vector loads start at a 4-aligned index <= the
  // last entry and read up to 3 entries past it (masked out)
  const size_t pad = 4;
  if ((e = cudaMalloc(&st->col, ((size_t)nnz + pad) * sizeof(int))) != cudaSuccess) return done(e);
  if ((e = cudaMalloc(&st->val, ((size_t)nnz + pad) * vs)) != cudaSuccess) return done(e);
  csr_fill_kernel<<<cdiv(m, kWarpsPerCta), kCta, 0, s>>>(views, N, D, m, st->row_ptr, st->col,
                                                         st->val, bf16);
  // CSC copy: counts per pixel, scan, fill by atomic cursors
  if ((e = cudaMalloc(&st->col_ptr, (size_t)(n + 1) * sizeof(int))) != cudaSuccess) return done(e);
  if ((e = cudaMalloc(&st->row, ((size_t)nnz + pad) * sizeof(int))) != cudaSuccess) return done(e);
  if ((e = cudaMalloc(&st->cval, ((size_t)nnz + pad) * vs)) != cudaSuccess) return done(e);
  // the padding is read (then masked), so give it defined contents
  if ((e = cudaMemsetAsync(st->col + nnz, 0, pad * sizeof(int), s)) != cudaSuccess) return done(e);
  if ((e = cudaMemsetAsync(st->row + nnz, 0, pad * sizeof(int), s)) != cudaSuccess) return done(e);
  if ((e = cudaMemsetAsync((char*)st->val + nnz * vs, 0, pad * vs, s)) != cudaSuccess) return done(e);
  if ((e = cudaMemsetAsync((char*)st->cval + nnz * vs, 0, pad * vs, s)) != cudaSuccess) return done(e);
  if ((e = cudaMemsetAsync(counts, 0, (size_t)(n + 1) * sizeof(int), s)) != cudaSuccess) return done(e);
  csc_count_kernel<<<152 * 8, 256, 0, s>>>(st->col, nnz, counts);
  // a pixel is tapped at most twice per view, so a column has at most 2 A_v entries
  st->max_col = 2 * (int)(m / D);
  scan_kernel<<<1, 1024, 0, s>>>(counts, st->col_ptr, n, d_total);
  if ((e = cudaMemcpyAsync(counts, st->col_ptr, (size_t)n * sizeof(int), cudaMemcpyDeviceToDevice,
                           s)) != cudaSuccess)
    return done(e);
  csc_fill_kernel<<<cdiv(m, kWarpsPerCta), kCta, 0, s>>>(m, st->row_ptr, st->col, st->val, bf16,
                                                         counts, st->row, st->cval);
  if (st->max_col > kSortCap) return done(cudaErrorInvalidValue);
  csc_sort_kernel<<<cdiv(n, 4), 128, 0, s>>>(st->col_ptr, st->row, st->cval, bf16, n);
  if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
  if ((e = build_sell(st->col_ptr, st->row, st->cval, bf16, n, counts, d_total, &st->cols32, s)) !=
      cudaSuccess)
    return done(e);
  return done(cudaStreamSynchronize(s));
}

void free_csr(CsrStore* st) {
  free_sell(&st->cols32);
  void* ptrs[] = {st->row_ptr, st->col, st->val, st->col_ptr, st->row, st->cval};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  *st = CsrStore{};
}

template <typename T, bool BF16>
void launch_spmv(const int* ptr, const int* idx, const void* val, const int* rows,
                 long long count, const T* x, T* y, int accumulate, int /*max_len*/,
                 cudaStream_t s) {
  spmv_kernel<T, BF16><<<cdiv(count, kWarpsPerCta), kCta, 0, s>>>(ptr, idx, val, rows, count, x, y,
                                                                  accumulate);
}

template <typename T>
cudaError_t launch_csr_project(const CsrStore& a, const int* ids, int count, const T* x, T* y,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (!ids) {
    // rays entering the image at different rows misalign a sliced layout, so
    // the forward pass streams the CSR one warp per ray
    if (a.bf16) launch_spmv<T, true>(a.row_ptr, a.col, a.val, nullptr, count, x, y, 0, a.max_row, s);
    else launch_spmv<T, false>(a.row_ptr, a.col, a.val, nullptr, count, x, y, 0, a.max_row, s);
    return cudaGetLastError();
  }
  if (a.bf16)
    spmv_kernel<T, true><<<cdiv(count, kWarpsPerCta), kCta, 0, s>>>(a.row_ptr, a.col, a.val, ids,
                                                                      count, x, y, 0);
  else
    spmv_kernel<T, false><<<cdiv(count, kWarpsPerCta), kCta, 0, s>>>(a.row_ptr, a.col, a.val, ids,
                                                                       count, x, y, 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_csr_backproject(const CsrStore& a, long long n, const int* ids, int count,
                                   const T* y, T* x, cudaStream_t s) {
  if (!ids) {
    // x += A^T y: lines of A^T are pixels (the SELL copy of the CSC)
    const Sell& q = a.cols32;
    const long long slices = (q.lines + 31) / 32;
    if (a.bf16)
      sell_spmv_kernel<T, true><<<(int)slices, 128, 0, s>>>(q.slice_ptr, q.idx, q.val, q.lines, y, x, 1);
    else
      sell_spmv_kernel<T, false><<<(int)slices, 128, 0, s>>>(q.slice_ptr, q.idx, q.val, q.lines, y, x, 1);
    return cudaGetLastError();
  }
  if (count <= 0) return cudaSuccess;
  if (a.bf16)
    csr_scatter_kernel<T, true><<<cdiv(count, kWarpsPerCta), kCta, 0, s>>>(a.row_ptr, a.col, a.val,
                                                                            ids, count, y, x);
  else
    csr_scatter_kernel<T, false><<<cdiv(count, kWarpsPerCta), kCta, 0, s>>>(a.row_ptr, a.col,
                                                                             a.val, ids, count, y, x);
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
  scatter_kernel<T><<<cdiv((long long)a.p * a.lanes, kCta), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tik_rhs(const StepArgs<T>& a, cudaStream_t s) {
  tik_rhs_kernel<T><<<cdiv(a.p, kWarpsPerCta), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tik_scale(const StepArgs<T>& a, cudaStream_t s) {
  const int grid = (int)std::min<long long>((a.n + 255) / 256, 152LL * 8);
  tik_scale_kernel<T><<<grid, 256, 0, s>>>(a);
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
  template cudaError_t launch_csr_project<T>(const CsrStore&, const int*, int, const T*, T*,     \
                                             cudaStream_t);                                     \
  template cudaError_t launch_csr_backproject<T>(const CsrStore&, long long, const int*, int,    \
                                                 const T*, T*, cudaStream_t);                   \
  template cudaError_t launch_sample<T>(const StepArgs<T>&, cudaStream_t);                    \
  template cudaError_t launch_forward_residual<T>(const StepArgs<T>&, cudaStream_t);          \
  template cudaError_t launch_gram_update<T>(const StepArgs<T>&, cudaStream_t);               \
  template cudaError_t launch_scatter<T>(const StepArgs<T>&, cudaStream_t);                   \
  template cudaError_t launch_tik_rhs<T>(const StepArgs<T>&, cudaStream_t);                   \
  template cudaError_t launch_tik_scale<T>(const StepArgs<T>&, cudaStream_t);                 \
  template cudaError_t launch_form_k<T>(const StepInfo*, const double*, T*, int, cudaStream_t); \
  template cudaError_t launch_project<T>(const ViewGeom*, int, int, const int*, int, const T*, \
                                         T*, cudaStream_t);                                    \
  template cudaError_t launch_backproject<T>(const ViewGeom*, int, int, const int*, int,       \
                                             const T*, T*, cudaStream_t);                      \
  template cudaError_t launch_rel_err<T>(const T*, const double*, long long, double*, cudaStream_t);

SLIM_INSTANTIATE(float)
SLIM_INSTANTIATE(double)

}  // namespace slim
