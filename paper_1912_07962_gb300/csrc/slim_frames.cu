// Kernels of the random-direction 3D geometry: the Joseph march, the fused
// march + residual of a block of random rays with its voxel lists, the Gram
// entries of the window, and A x / A^T y.
#include "slim_frames.cuh"

#include <algorithm>
#include <cmath>

namespace slim {

FrameGeom make_frame_geom(const double* r) {
  FrameGeom f;
  for (int c = 0; c < 3; ++c) {
    f.d[c] = r[c];
    f.u[c] = r[3 + c];
    f.v[c] = r[6 + c];
  }
  f.k = 0;
  for (int c = 1; c < 3; ++c)
    if (std::fabs(f.d[c]) > std::fabs(f.d[f.k])) f.k = c;
  f.i = f.k == 0 ? 1 : 0;
  f.j = f.k == 2 ? 1 : 2;
  f.inv = 1.0 / f.d[f.k];
  f.ia = std::fabs(f.inv);
  f.pad_ = 0;
  return f;
}

namespace {

constexpr int kWarps = 8;
constexpr int kCta = 32 * kWarps;

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

struct RayPoint {
  int view;
  double p0[3];   // the ray's point on the detector plane through the centre
};

__device__ __forceinline__ RayPoint frame_ray(const FrameGeom* frames, int ray, int Du, int Dv) {
  RayPoint rp;
  const int per_view = Du * Dv;
  rp.view = ray / per_view;
  const int rem = ray - rp.view * per_view;
  const int iv = rem / Du, iu = rem - iv * Du;
  const FrameGeom& f = frames[rp.view];
  const double tu = (double)iu - 0.5 * (double)(Du - 1);
  const double tv = (double)iv - 0.5 * (double)(Dv - 1);
  for (int c = 0; c < 3; ++c) rp.p0[c] = __dadd_rn(__dmul_rn(tu, f.u[c]), __dmul_rn(tv, f.v[c]));
  return rp;
}

// The four taps at slice s of the march axis: voxel index (-1 when dropped)
// and weight (0 when dropped).
__device__ __forceinline__ void frame_taps(const FrameGeom& f, const double (&p0)[3], double cc,
                                           int N, int s, int (&vox)[4], double (&w)[4]) {
  const double tau = __dmul_rn(__dsub_rn(__dsub_rn((double)s, cc), p0[f.k]), f.inv);
  const double fi = __dadd_rn(__dadd_rn(p0[f.i], __dmul_rn(tau, f.d[f.i])), cc);
  const double fj = __dadd_rn(__dadd_rn(p0[f.j], __dmul_rn(tau, f.d[f.j])), cc);
  const double i0f = floor(fi), j0f = floor(fj);
  const double wi = __dsub_rn(fi, i0f), wj = __dsub_rn(fj, j0f);
  const double ui = __dsub_rn(1.0, wi), uj = __dsub_rn(1.0, wj);
  w[0] = __dmul_rn(__dmul_rn(ui, uj), f.ia);
  w[1] = __dmul_rn(__dmul_rn(wi, uj), f.ia);
  w[2] = __dmul_rn(__dmul_rn(ui, wj), f.ia);
  w[3] = __dmul_rn(__dmul_rn(wi, wj), f.ia);
  // |f_i|, |f_j| are bounded by the detector's extent: the conversions are exact
  const int i0 = (int)i0f, j0 = (int)j0f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int ci = i0 + (e & 1), cj = j0 + (e >> 1);
    const bool in = ci >= 0 && ci < N && cj >= 0 && cj < N && w[e] != 0.0;
    const int cx = f.k == 0 ? s : (f.i == 0 ? ci : cj);
    const int cy = f.k == 1 ? s : (f.i == 1 ? ci : cj);
    const int cz = f.k == 2 ? s : (f.i == 2 ? ci : cj);
    vox[e] = in ? (cz * N + cy) * N + cx : -1;
    if (!in) w[e] = 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kCta) forward_frames_kernel(RayArgs a, FrameArgs f,
                                                              const T* __restrict__ x,
                                                              const T* __restrict__ b) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= a.ell) return;
  const int q = a.info->slot * a.ell + w;
  const int ray = a.ring_ids[q];
  const RayPoint rp = frame_ray(f.frames, ray, a.Du, a.Dv);
  const FrameGeom fg = f.frames[rp.view];
  const double cc = 0.5 * (double)(a.N - 1);
  int* pix = a.ring_pix + (size_t)q * a.taps;
  double* wt = a.ring_w + (size_t)q * a.taps;
  const int ebase = w * a.taps;   // entry ids of this ray in the block's lists
  T acc = T(0);
  for (int s = lane; s < a.N; s += 32) {
    int vox[4];
    double tw[4];
    frame_taps(fg, rp.p0, cc, a.N, s, vox, tw);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int t = 4 * s + e;
      pix[t] = vox[e];
      wt[t] = tw[e];
      if (vox[e] >= 0) {
        acc += (T)tw[e] * x[vox[e]];
        f.vnext[ebase + t] = atomicExch(&f.vhead[vox[e]], ebase + t);
      }
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) a.rhs[q] = (double)(acc - b[ray]);
}

// One warp per ring row q: walk q's taps through the new block's voxel lists
// and add each product into G[q][slot block] (float64 atomics in L2).  Without a per-warp accumulator in shared memory
// the kernel runs at full occupancy, which its chains of dependent loads
// (tap, list head, list entries) need.  A list longer than any block can make
// (4 ell entries at one voxel) is cut and reported (SLIM_EINVAL).
__global__ void __launch_bounds__(kCta) gram_frames_kernel(RayArgs a, FrameArgs f) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= a.p || a.ring_ids[q] < 0) return;
  const int base = a.info->slot * a.ell;
  const double* nw = a.ring_w + (size_t)base * a.taps;   // weight of entry e of the new block
  double* grow = a.G + (size_t)q * a.P + base;
  // this warp is the only writer of its row's block: clear it, then add
  for (int i = lane; i < a.ell; i += 32) grow[i] = 0.0;
  __syncwarp();
  const int max_hops = 4 * a.ell;
  const int* rp = a.ring_pix + (size_t)q * a.taps;
  const double* rw = a.ring_w + (size_t)q * a.taps;
  for (int t = lane; t < a.taps; t += 32) {
    const int vox = rp[t];
    if (vox < 0) continue;
    const double wq = rw[t];
    int hops = 0;
    for (int e = f.vhead[vox]; e >= 0; e = f.vnext[e]) {
      if (++hops > max_hops) {
        set_status(a.status, SLIM_EINVAL);
        break;
      }
      atomicAdd(grow + e / a.taps, wq * nw[e]);
    }
  }
}

// G[slot block][q] = G[q][slot block] for the ring rows q outside the new
// block (whose rows hold both halves already): 32 x 32 tiles through shared
// memory, reads and writes coalesced.
__global__ void __launch_bounds__(kCta) gram_frames_mirror_kernel(RayArgs a) {
  __shared__ double tile[32][33];
  const int base = a.info->slot * a.ell;
  const int i0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    const int q = q0 + r, i = i0 + tx;
    tile[r][tx] = (q < a.p && i < a.ell) ? a.G[(size_t)q * a.P + base + i] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, q = q0 + tx;
    if (i < a.ell && q < a.p && (q < base || q >= base + a.ell))
      a.G[(size_t)(base + i) * a.P + q] = tile[tx][r];
  }
}

template <typename T>
__global__ void __launch_bounds__(kCta) project_frames_kernel(const FrameGeom* frames, int N,
                                                              int Du, int Dv, const int* ids,
                                                              long long count,
                                                              const T* __restrict__ x, T* y) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= count) return;
  const int ray = ids ? ids[w] : (int)w;
  const RayPoint rp = frame_ray(frames, ray, Du, Dv);
  const FrameGeom fg = frames[rp.view];
  const double cc = 0.5 * (double)(N - 1);
  T acc = T(0);
  for (int s = lane; s < N; s += 32) {
    int vox[4];
    double tw[4];
    frame_taps(fg, rp.p0, cc, N, s, vox, tw);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (vox[e] >= 0) acc += (T)tw[e] * x[vox[e]];
  }
  acc = warp_sum(acc);
  if (lane == 0) y[w] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kCta) backproject_frames_kernel(const FrameGeom* frames, int N,
                                                                  int Du, int Dv, const int* ids,
                                                                  long long count,
                                                                  const T* __restrict__ y, T* x) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= count) return;
  const int ray = ids ? ids[w] : (int)w;
  const T c = y[w];
  if (c == T(0)) return;
  const RayPoint rp = frame_ray(frames, ray, Du, Dv);
  const FrameGeom fg = frames[rp.view];
  const double cc = 0.5 * (double)(N - 1);
  for (int s = lane; s < N; s += 32) {
    int vox[4];
    double tw[4];
    frame_taps(fg, rp.p0, cc, N, s, vox, tw);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (vox[e] >= 0) atomicAdd(&x[vox[e]], (T)tw[e] * c);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_forward_frames(const RayArgs& a, const FrameArgs& f, const T* x, const T* b,
                                  cudaStream_t s) {
  forward_frames_kernel<T><<<cdiv(a.ell, kWarps), kCta, 0, s>>>(a, f, x, b);
  return cudaGetLastError();
}

cudaError_t launch_gram_frames(const RayArgs& a, const FrameArgs& f, cudaStream_t s) {
  gram_frames_kernel<<<cdiv(a.p, kWarps), kCta, 0, s>>>(a, f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_frames_mirror_kernel<<<dim3(cdiv(a.ell, 32), cdiv(a.p, 32)), kCta, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project_frames(const FrameGeom* frames, int N, int Du, int Dv, const int* ids,
                                  long long count, const T* x, T* y, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  project_frames_kernel<T><<<cdiv(count, kWarps), kCta, 0, s>>>(frames, N, Du, Dv, ids, count, x,
                                                                  y);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backproject_frames(const FrameGeom* frames, int N, int Du, int Dv,
                                      const int* ids, long long count, const T* y, T* x,
                                      cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  backproject_frames_kernel<T><<<cdiv(count, kWarps), kCta, 0, s>>>(frames, N, Du, Dv, ids,
                                                                      count, y, x);
  return cudaGetLastError();
}

#define SLIM_FRAMES_INST(T)                                                                     \
  template cudaError_t launch_forward_frames<T>(const RayArgs&, const FrameArgs&, const T*,     \
                                                const T*, cudaStream_t);                        \
  template cudaError_t launch_project_frames<T>(const FrameGeom*, int, int, int, const int*,    \
                                                long long, const T*, T*, cudaStream_t);         \
  template cudaError_t launch_backproject_frames<T>(const FrameGeom*, int, int, int, const int*, \
                                                    long long, const T*, T*, cudaStream_t);
SLIM_FRAMES_INST(float)
SLIM_FRAMES_INST(double)

}  // namespace slim
