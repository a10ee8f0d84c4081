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
