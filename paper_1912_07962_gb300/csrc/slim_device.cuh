// Device-side building blocks shared by the slimLS kernels: the counter-based
// generator, the Joseph ray geometry, warp reductions and the status word.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/slim.h"

namespace slim {

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a counter-based
// generator: output i of the sequence seeded with `seed` is
// mix(seed + (i+1) * 0x9E3779B97F4A7C15).  Draw (seed, stream, counter)
// is output stream * 2^40 + counter.  Bounded integers use Lemire's
// multiply-shift on the top 32 bits.
// ---------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kStreamShift = 40;
constexpr int kStreamBlocks = 2;
constexpr int kStreamRays = 3;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t draw64(uint64_t seed, uint64_t stream, uint64_t counter) {
  uint64_t index = (stream << kStreamShift) + counter;
  return mix64(seed + (index + 1ull) * kGamma);
}
__host__ __device__ inline uint32_t bounded32(uint64_t u, uint32_t k) {
  return (uint32_t)(((u >> 32) * (uint64_t)k) >> 32);
}

// ---------------------------------------------------------------------------
// Sampling without replacement.
//
// Random cyclic order of view blocks (the walnut experiment of Sec. 4.3 visits
// its blocks in a random cyclic order): epoch e = (k-1) / V of the steps visits
// every view once, in the order of the Fisher-Yates (Durstenfeld) shuffle of
// 0..V-1 in which swap i, for i = V-1 down to 1, exchanges entries i and
// bounded(draw(seed, 7, e*V + V-1-i), i+1).  Step k takes entry (k-1) mod V.
// ---------------------------------------------------------------------------
constexpr int kStreamCyclic = 7;
constexpr int kMaxCyclicViews = 4096;

// View of step k in the random cyclic order.  Every thread of the block calls
// it with the same arguments (its branches are uniform).  The permutation of
// the current epoch is cached in perm[V] with its epoch in *perm_epoch (-1:
// none), and recomputed in s_perm (kMaxCyclicViews shared ints) when the
// epoch changes.  A block-wide barrier follows any recomputation.
__device__ inline int cyclic_view(uint64_t seed, long long k, int V, int* perm,
                                  long long* perm_epoch, int* s_perm) {
  const long long e = (k - 1) / V;
  const int pos = (int)((k - 1) % V);
  if (*perm_epoch == e) return perm[pos];
  for (int i = threadIdx.x; i < V; i += blockDim.x) s_perm[i] = i;
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t base = (uint64_t)e * (uint64_t)V;
    for (int i = V - 1; i >= 1; --i) {
      const int j = (int)bounded32(draw64(seed, kStreamCyclic, base + (uint64_t)(V - 1 - i)),
                                   (uint32_t)(i + 1));
      const int t = s_perm[i];
      s_perm[i] = s_perm[j];
      s_perm[j] = t;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < V; i += blockDim.x) perm[i] = s_perm[i];
  const int view = s_perm[pos];
  __syncthreads();   // every thread has read *perm_epoch and s_perm
  if (threadIdx.x == 0) *perm_epoch = e;
  return view;
}

// Distinct rays in a random-ray block: Floyd's algorithm (Bentley and Floyd,
// "A sample of brilliance", CACM 1987) for ell distinct ids of [0, n): for
// i = 0 .. ell-1, with j = n - ell + i and t = bounded(draw(seed, 3,
// (k-1)*ell + i), j+1), insert t unless it is already in the sample, else
// insert j.  The ids are kept in insertion order.
constexpr int kMaxDistinctRays = 2048;
constexpr int kDistinctTable = 2 * kMaxDistinctRays;   // open-addressing set, power of two

// Fills ids[0..ell) for step k.  Every thread of the block calls it; s_t
// (kMaxDistinctRays ints) and s_tab (kDistinctTable ints) are shared memory.
// ell <= kMaxDistinctRays and ell <= n are the caller's to check.
__device__ inline void floyd_rays(uint64_t seed, long long k, int ell, uint32_t n, int* ids,
                                  int* s_t, int* s_tab) {
  const uint64_t base = (uint64_t)(k - 1) * (uint64_t)ell;
  for (int i = threadIdx.x; i < ell; i += blockDim.x) {
    const uint32_t j = n - (uint32_t)ell + (uint32_t)i;
    s_t[i] = (int)bounded32(draw64(seed, kStreamRays, base + (uint64_t)i), j + 1u);
  }
  for (int i = threadIdx.x; i < kDistinctTable; i += blockDim.x) s_tab[i] = -1;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < ell; ++i) {
      const int j = (int)(n - (uint32_t)ell + (uint32_t)i);
      int v = s_t[i];
      // look v up; j itself can never be in the set yet (every earlier entry is < j)
      uint32_t h = ((uint32_t)v * 0x9E3779B1u) & (kDistinctTable - 1);
      bool found = false;
      while (s_tab[h] != -1) {
        if (s_tab[h] == v) { found = true; break; }
        h = (h + 1) & (kDistinctTable - 1);
      }
      if (found) {
        v = j;
        h = ((uint32_t)v * 0x9E3779B1u) & (kDistinctTable - 1);
        while (s_tab[h] != -1) h = (h + 1) & (kDistinctTable - 1);
      }
      s_tab[h] = v;
      s_t[i] = v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ell; i += blockDim.x) ids[i] = s_t[i];
}

// ---------------------------------------------------------------------------
// Joseph geometry.  Per view: co = cos(theta), si = sin(theta) from the host
// table; row-stepping iff |co| >= |si|; rc = 1/co (row) or 1/si (column);
// ia = |rc| is the path length per step.  For step s (row iy or column ix):
//   pos = s - cc;  u = t - pos*(row ? si : co);  f = u*rc + cc
//   j0 = floor(f);  w1 = f - j0;  wa = (1 - w1)*ia;  wb = w1*ia
// Every operation is an explicitly rounded intrinsic so the compiler cannot
// contract it into a fused multiply-add: the taps are bit-identical to a
// plain IEEE float64 evaluation of the same formula.
// ---------------------------------------------------------------------------
struct ViewGeom {
  double co, si, rc, ia;
  int row_step;
  int pad_;
};

struct Tap2 {
  int minor0;      // interpolated index of tap a (tap b is minor0 + 1)
  double wa, wb;
};

__device__ __forceinline__ Tap2 joseph_step(const ViewGeom& v, double t, double cc, int s) {
  double pos = (double)s - cc;
  double u = __dsub_rn(t, __dmul_rn(pos, v.row_step ? v.si : v.co));
  double f = __dadd_rn(__dmul_rn(u, v.rc), cc);
  double j0f = floor(f);
  double w1 = __dsub_rn(f, j0f);
  Tap2 r;
  r.minor0 = (int)j0f;
  r.wa = __dmul_rn(__dsub_rn(1.0, w1), v.ia);
  r.wb = __dmul_rn(w1, v.ia);
  return r;
}

// Pixel index of in-plane tap (step s, interpolated index j) in an N x N slice,
// or -1 when the tap falls outside the image.
__device__ __forceinline__ int inplane_pixel(int row_step, int N, int s, int j) {
  if (j < 0 || j >= N) return -1;
  return row_step ? (s * N + j) : (j * N + s);
}

// ---------------------------------------------------------------------------
// Reductions and status
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

// 1/sqrt(d) in float64 from a float seed refined by two Newton-Raphson steps
// r <- r (3/2 - d r^2 / 2) (each roughly doubles the correct bits, about
// 22 -> 44 -> the float64 precision);
// a handful of float64 operations where the library square root and division
// are long sequences on the float64 pipe.  d <= 0 is reported as SLIM_ENOTPD
// and replaced by 1; magnitudes outside the float range take the slow path.
__device__ __forceinline__ double rsqrt_pivot(double d, int* status) {
  if (!(d > 0.0)) {
    set_status(status, SLIM_ENOTPD);
    d = 1.0;
  }
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double r = (double)rsqrtf((float)d);
  const double h = 0.5 * d;
  r = r * fma(-h * r, r, 1.5);
  r = r * fma(-h * r, r, 1.5);
  return r;
}

// Per-step values computed on the device by the sampler.
// lambda_k: the damping ramp of Sec. 4.2 (lambda (r+1)/k for k <= r+1), the
// 1/k decay after step decay_after (lambda k / decay_after; 0: none), else
// lambda.  Each operation rounded once.
__device__ __forceinline__ double damping_k(double lam, long long k, int r, int ramp,
                                            int decay_after) {
  if (ramp && k <= r + 1) return __ddiv_rn(__dmul_rn(lam, (double)(r + 1)), (double)k);
  if (decay_after > 0 && k > decay_after)
    return __ddiv_rn(__dmul_rn(lam, (double)k), (double)decay_after);
  return lam;
}

struct StepInfo {
  long long k;      // 1-based index of the step being taken
  int slot;         // ring slot of the new block
  int view;         // sampled view (view blocks)
  double lam_k;     // shift of the Gram system: lambda_k, or mu_k = lambda_k + c_k beta (slimTik)
  double tik_c;     // slimTik: beta / mu_k; 0 otherwise
};

}  // namespace slim
