// U-Net for the learned initial guess x_0 = f(A^T b): forward, backward and
// Adam, all in hand-written kernels.  The paper starts from x_0 = 0 (Sec. 4);
// the network is an extension of this library.
//
// Layout: activations are channel-major over the batch, C x (n*H*W) float32
// ("CNHW"), so every layer is one GEMM:
//   conv3x3    Y = W col(X) + b        col = im2col of X (K = 9 C_in rows),
//              dW += dY col(X)^T,  dX = Wf col(dY)   (Wf: the adjoint conv's weights)
//              implicit GEMMs: col is gathered into shared memory, never stored
//   tconv2x2   Y4 = W^T X (rows (o,u,v)), scattered to the 2x upsampled grid
//              dW += X dY4^T,  dX = W dY4   (dY4 gathered from dY); the
//              scatter is the GEMM's epilogue and the gather its loaders
//   conv1x1    Y = W X + b
// The decoder's concatenation [upsampled; skip] is one buffer whose lower
// channel rows are written by the encoder directly.  Weights used by the
// forward pass are the float32 master values rounded to bfloat16 (nearest
// even); biases are used unrounded.  Accumulation is float32 throughout.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/slim.h"
#include "slim_tcgen05.cuh"
#include "slim_unet.cuh"

namespace {

constexpr int kT = 256;

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }
inline int grid_for(long long n) { return (int)std::min<long long>(std::max<long long>(cdiv(n, kT), 1), 152LL * 32); }

// ---------------------------------------------------------------------------
// GEMM: C[m][n] (+)= sum_k op(A)[m][k] op(B)[k][n] (+ bias[m]) (ReLU)
//   op(A)[m][k] = TA ? A[k*lda + m] : A[m*lda + k]
//   op(B)[k][n] = TB ? B[n*ldb + k] : B[k*ldb + n]
// BM x BN tile per CTA of 256 threads (4 x 4 outputs each), k in chunks of
// 16 staged k-major in shared memory.  With gridDim.z > 1 the k range is
// split and partial sums are added atomically into C (which holds the
// accumulated value on entry).
// ---------------------------------------------------------------------------
constexpr int kBK = 16;

template <bool TA, bool TB, int BM, int BN>
__global__ void __launch_bounds__(kT) sgemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                   int lda, const float* __restrict__ B, int ldb,
                                                   float* C, int ldc, const float* __restrict__ bias,
                                                   int relu, int accumulate, int kchunk) {
  static_assert((BM / 4) * (BN / 4) == kT, "tile shape");
  __shared__ __align__(16) float As[kBK][BM + 4];
  __shared__ __align__(16) float Bs[kBK][BN + 4];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  const int tm = tid / (BN / 4), tn = tid % (BN / 4);
  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += kBK) {
    for (int idx = tid; idx < BM * kBK; idx += kT) {
      int mm, kk;
      if (TA) { mm = idx % BM; kk = idx / BM; } else { kk = idx % kBK; mm = idx / kBK; }
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < kend) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      As[kk][mm] = v;
    }
    for (int idx = tid; idx < BN * kBK; idx += kT) {
      int nn, kk;
      if (TB) { kk = idx % kBK; nn = idx / kBK; } else { nn = idx % BN; kk = idx / BN; }
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.f;
      if (n < N && k < kend) v = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][tm * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tn * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
  const bool split = gridDim.z > 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + tm * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tn * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      float* c = C + (size_t)m * ldc + n;
      if (split) {
        atomicAdd(c, v);
      } else {
        if (bias) v += bias[m];
        if (accumulate) v += *c;
        if (relu) v = fmaxf(v, 0.f);
        *c = v;
      }
    }
  }
}

template <bool TA, bool TB>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                 int ldc, const float* bias, bool relu, bool accumulate, int splits, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  splits = std::max(1, std::min(splits, cdiv(K, kBK)));
  const int kchunk = cdiv(cdiv(K, splits), kBK) * kBK;
  splits = cdiv(K, kchunk);
  if (M <= 32) {
    dim3 grid(cdiv(N, 128), cdiv(M, 32), splits);
    sgemm_kernel<TA, TB, 32, 128><<<grid, kT, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias,
                                                       relu, accumulate, kchunk);
  } else {
    dim3 grid(cdiv(N, 64), cdiv(M, 64), splits);
    sgemm_kernel<TA, TB, 64, 64><<<grid, kT, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu,
                                                     accumulate, kchunk);
  }
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Tensor-core GEMM with operand loaders, so that the 3x3 convolutions run as
// implicit GEMMs: the im2col matrix is gathered tile by tile from the
// activations into shared memory and never written out.
//
//   C[m][n] (+)= sum_k A(m, k) B(n, k)  (+ bias[m]) (ReLU)
//
// Float32 values reach the bfloat16 tensor cores as a sum of T bfloat16
// terms, x = x_0 + x_1 + ... with x_j = bf16(x - x_0 - ... - x_{j-1})
// (nearest even).  T = 3 carries 24 significant bits, i.e. the float32 value
// itself (up to the last bit); T = 2 carries 16.  The weights used by the
// network are bfloat16 values already (T = 1).  The products x_i y_j with
// i + j < max(TA, TB) are accumulated, which drops only terms below the
// float32 rounding of the sum (T = 3 x 1) or below 2^-16 relative (2 x 2).
// A loader gives 8 consecutive k of one row at a time; with gridDim.z > 1
// the k range is split and the partial sums are added atomically into C.
// The kernel itself (tcgen05, tensor memory) is t5_gemm_kernel below.
// ---------------------------------------------------------------------------

// C[m][n] = acc (+ bias[m]) (+ C[m][n]) (ReLU); atomically added when split.
struct OutPlain {
  float* C;
  long long ldc;
  int M, N;
  const float* bias;
  int relu, accumulate;
  __device__ void store(int m, int n, float v, bool split) const {
    float* c = C + (size_t)m * ldc + n;
    if (split) {
      atomicAdd(c, v);
      return;
    }
    if (bias) v += bias[m];
    if (accumulate) v += *c;
    if (relu) v = fmaxf(v, 0.f);
    *c = v;
  }
};

// 2x2 stride-2 transposed conv: row m = o*4 + u*2 + v, column n = input pixel
// (global image row R = n / W, column x); the value lands at output
// Y[o][2R+u][2x+v] (images stacked along R) plus bias[o].  Never split.
struct OutUp {
  float* Y;
  long long Pout;
  int M, N, W;
  const float* bias;
  __device__ void store(int m, int n, float v, bool) const {
    const int o = m >> 2, u = (m >> 1) & 1, vv = m & 1;
    const int R = n / W, x = n - R * W;
    Y[(size_t)o * Pout + (size_t)(2 * R + u) * (2 * W) + 2 * x + vv] = v + (bias ? bias[o] : 0.f);
  }
};

// A(row, k) = p[row * ld + k]
struct LoadRowK {
  const float* p;
  long long ld;
  int rows;
  struct Row { const float* ptr; };
  __device__ Row row(int r) const { return {r < rows ? p + (size_t)r * ld : nullptr}; }
  __device__ void load8(const Row& c, int k, int kend, float (&v)[8]) const {
    if (c.ptr && k + 8 <= kend && (reinterpret_cast<uintptr_t>(c.ptr + k) & 15) == 0) {
      const float4 a = *reinterpret_cast<const float4*>(c.ptr + k);
      const float4 b = *reinterpret_cast<const float4*>(c.ptr + k + 4);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = (c.ptr && k + i < kend) ? c.ptr[k + i] : 0.f;
  }
};

// A(row, k) = p[k * ld + row]
struct LoadKRow {
  const float* p;
  long long ld;
  int rows;
  struct Row { const float* ptr; };
  __device__ Row row(int r) const { return {r < rows ? p + r : nullptr}; }
  __device__ void load8(const Row& c, int k, int kend, float (&v)[8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = (c.ptr && k + i < kend) ? c.ptr[(size_t)(k + i) * ld] : 0.f;
  }
};

// Rows are pixels p of X (C x P, n images of H x W), k = t*C + c with tap
// t = u*3 + v: A(p, k) = X[c][img, y+u-1, x+v-1], zero outside the image.
// Tap-major k: when C is a multiple of 8 a group of 8 k shares one tap, so
// one bounds test and one offset serve its 8 loads (stride P).
struct LoadPixTap {
  const float* X;
  long long P;
  int H, W, C;
  struct Row { long long p; int y, x; };
  __device__ Row row(int r) const {
    if (r >= P) return {-1, 0, 0};
    const int rem = (int)(r % ((long long)H * W));
    return {r, rem / W, rem % W};
  }
  __device__ void load8(const Row& c, int k, int kend, float (&v)[8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.f;
    if (c.p < 0) return;
    int t = k / C, ch = k - t * C;
    if ((C & 7) == 0 && k + 8 <= kend) {
      const int du = t / 3 - 1, dv = t % 3 - 1;
      const int yy = c.y + du, xx = c.x + dv;
      if (yy < 0 || yy >= H || xx < 0 || xx >= W) return;
      const float* src = X + (size_t)ch * P + c.p + (long long)du * W + dv;
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = src[(size_t)i * P];
      return;
    }
    for (int i = 0; i < 8 && k + i < kend; ++i) {
      const int du = t / 3 - 1, dv = t % 3 - 1;
      const int yy = c.y + du, xx = c.x + dv;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W)
        v[i] = X[(size_t)ch * P + c.p + (long long)du * W + dv];
      if (++ch == C) { ch = 0; ++t; }
    }
  }
};

// Conv weights W [O][C][3][3] as A(o, k = t*C + c) = W[o][c][t] (tap-major k,
// matching LoadPixTap).
struct LoadWTap {
  const float* Wt;
  int C, rows;
  struct Row { const float* ptr; };
  __device__ Row row(int r) const { return {r < rows ? Wt + (size_t)r * C * 9 : nullptr}; }
  __device__ void load8(const Row& c, int k, int kend, float (&v)[8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.f;
    if (!c.ptr) return;
    int t = k / C, ch = k - t * C;
    if ((C & 7) == 0 && k + 8 <= kend) {
      const float* src = c.ptr + ch * 9 + t;
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = src[i * 9];
      return;
    }
    for (int i = 0; i < 8 && k + i < kend; ++i) {
      v[i] = c.ptr[ch * 9 + t];
      if (++ch == C) { ch = 0; ++t; }
    }
  }
};

// Rows are taps r = c*9 + u*3 + v, k = pixel p of X:
// A(r, p) = X[c][img, y+u-1, x+v-1], zero outside the image.
struct LoadTapPix {
  const float* X;
  long long P;
  int H, W, rows;
  struct Row { long long base; int du, dv; };
  __device__ Row row(int r) const {
    if (r >= rows) return {-1, 0, 0};
    const int ch = r / 9, t = r % 9;
    return {(long long)ch * P, t / 3 - 1, t % 3 - 1};
  }
  __device__ void load8(const Row& c, int k, int kend, float (&v)[8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.f;
    if (c.base < 0) return;
    const int HW = H * W;
    int rem = (int)(k % HW);
    int y = rem / W, x = rem % W;
    const int yy = y + c.du;
    if ((W & 7) == 0 && k + 8 <= kend) {
      // the 8 pixels share image row y (k is a multiple of 8); only the
      // first or last can fall off the row
      if (yy < 0 || yy >= H) return;
      const float* src = X + c.base + k + (long long)c.du * W + c.dv;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int xx = x + i + c.dv;
        if (xx >= 0 && xx < W) v[i] = src[i];
      }
      return;
    }
    for (int i = 0; i < 8 && k + i < kend; ++i) {
      const int yy2 = y + c.du, xx = x + c.dv;
      if (yy2 >= 0 && yy2 < H && xx >= 0 && xx < W)
        v[i] = X[c.base + k + i + (long long)c.du * W + c.dv];
      if (++x == W) { x = 0; if (++y == H) y = 0; }
    }
  }
};

// Weights of the adjoint 3x3 conv read in place from W [O][C][3][3]:
// A(c, k = t*O + o) = W[o][c][8 - t] (tap-major k, matching LoadPixTap on dY).
struct LoadFlipW {
  const float* Wt;
  int C, O;
  struct Row { int c; };
  __device__ Row row(int r) const { return {r < C ? r : -1}; }
  __device__ void load8(const Row& c, int k, int kend, float (&v)[8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.f;
    if (c.c < 0) return;
    int t = k / O, o = k - t * O;
    if ((O & 7) == 0 && k + 8 <= kend) {
      const float* src = Wt + ((size_t)o * C + c.c) * 9 + 8 - t;
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = src[(size_t)i * C * 9];
      return;
    }
    for (int i = 0; i < 8 && k + i < kend; ++i) {
      v[i] = Wt[((size_t)o * C + c.c) * 9 + 8 - t];
      if (++o == O) { o = 0; ++t; }
    }
  }
};

// Rows are input pixels p of a 2x2 stride-2 transposed conv (global image
// row R = p / W, column x), k = o*4 + u*2 + v: A(p, k) = dY[o][2R+u][2x+v].
struct LoadUpPix {
  const float* dY;
  long long Pout;
  int W, rows;
  struct Row { long long base; };
  __device__ Row row(int r) const {
    if (r >= rows) return {-1};
    const int R = r / W, x = r - R * W;
    return {(long long)(2 * R) * (2 * W) + 2 * x};
  }
  __device__ void load8(const Row& c, int k, int kend, float (&v)[8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int kk = k + i;
      v[i] = (c.base >= 0 && kk < kend)
                 ? dY[(size_t)(kk >> 2) * Pout + c.base + ((kk >> 1) & 1) * (2 * W) + (kk & 1)]
                 : 0.f;
    }
  }
};

// Rows are taps r = o*4 + u*2 + v, k = input pixel p (R = p / W, x):
// A(r, p) = dY[o][2R+u][2x+v].
struct LoadUpTapPix {
  const float* dY;
  long long Pout;
  int W, rows;
  struct Row { long long base; int u, v; };
  __device__ Row row(int r) const {
    if (r >= rows) return {-1, 0, 0};
    return {(long long)(r >> 2) * Pout, (r >> 1) & 1, r & 1};
  }
  __device__ void load8(const Row& c, int k, int kend, float (&v)[8]) const {
    int R = k / W, x = k - R * W;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      v[i] = (c.base >= 0 && k + i < kend)
                 ? dY[c.base + (long long)(2 * R + c.u) * (2 * W) + 2 * x + c.v]
                 : 0.f;
      if (++x == W) { x = 0; ++R; }
    }
  }
};

// ---------------------------------------------------------------------------
// The same GEMM on the tcgen05 tensor cores.  The MMA's M is the GEMM's n
// (pixels, 128 per CTA) and its N the GEMM's m (channels, BN = 32..256 per
// CTA), so one tile covers all output channels of up to 128 pixels and the
// float32 accumulator lives in BN columns of tensor memory.  K runs in
// slices of 64 (128-byte rows of bfloat16): the 256 threads gather a slice
// of both operands through the loaders, split it into bfloat16 terms and
// store each term tile in the 128-byte-swizzled K-major layout; one thread
// issues the term products a_i b_j (i + j < max(TA, TB)) of its four K = 16
// steps and commits them to the slice's mbarrier, while the threads gather
// the next slice into the other stage.  The epilogue reads the accumulator
// (warp w: lanes 32 (w % 4) .. +31, half w / 4 of the columns) and writes
// through the output policy; consecutive lanes are consecutive pixels.
// Every mbarrier wait is bounded: one that runs out records 1 in
// g_t5_timeout and the CTA skips to the end.
// ---------------------------------------------------------------------------
constexpr int kT5N = 128;            // pixels per CTA (the MMA's M)
constexpr int kT5K = 64;             // K per slice
constexpr unsigned kT5Spin = 1u << 24;
__device__ int g_t5_timeout = 0;

// Split 8 float32 values into T bfloat16 terms at chunk kg of row r of a
// 128-byte-swizzled K-major tile (term j at tile0 + j * tile_bytes).
template <int T>
__device__ __forceinline__ void stage_terms128(unsigned char* tile0, int tile_bytes, int r, int kg,
                                               float (&v)[8]) {
  const uint32_t off = slim::t5::sw128_off(r, kg);
#pragma unroll
  for (int j = 0; j < T; ++j) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
      w[q] = *reinterpret_cast<const uint32_t*>(&h);
      if (j + 1 < T) {
        const float2 f = __bfloat1622float2(h);
        v[2 * q] -= f.x;
        v[2 * q + 1] -= f.y;
      }
    }
    *reinterpret_cast<uint4*>(tile0 + j * tile_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int BN, int TA, int TB>
struct T5Shape {
  static constexpr int kTermN = kT5N * 128;            // bytes of one pixel-side term tile
  static constexpr int kTermM = BN * 128;              // of one channel-side term tile
  static constexpr int kStage = TB * kTermN + TA * kTermM;
  static constexpr int kSmem = 2 * kStage + 1024;      // two stages, 1024-byte alignment slack
  static constexpr int kCallsN = kT5N * 8 / kT;        // 8-value gathers per thread and slice
  static constexpr int kCallsM = (BN * 8 + kT - 1) / kT;
};

template <class LA, class LB, class OUT, int BN, int TA, int TB>
__global__ void __launch_bounds__(kT, 1) t5_gemm_kernel(OUT out, LA la, LB lb, int K, int kchunk) {
  using S = T5Shape<BN, TA, TB>;
  namespace t5 = slim::t5;
  extern __shared__ unsigned char t5_raw[];
  __shared__ uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(t5_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  const int nslice = kend > kbeg ? (kend - kbeg + kT5K - 1) / kT5K : 0;
  const int ntiles = (out.N + kT5N - 1) / kT5N;
  constexpr int TMAX = TA > TB ? TA : TB;
  constexpr uint32_t kIdesc = t5::idesc_bf16(kT5N, BN);

  if (tid == 0) {
    t5::mbar_init(t5::smem_u32(&s_bar[0]), 1);
    t5::mbar_init(t5::smem_u32(&s_bar[1]), 1);
    s_fail = 0;
    t5::fence_barrier_init();
  }
  if (warp == 0) t5::tmem_alloc(t5::smem_u32(&s_tmem), BN);
  t5::fence_before();
  __syncthreads();
  t5::fence_after();
  const uint32_t tmem = s_tmem;

  // this thread's rows: pixel row tid % 128 (chunks tid / 128 + 2 i), and
  // channel rows idx % BN for idx = tid + 256 i (chunk idx / BN)
  const int rn = tid % kT5N;
  typename LA::Row rowM[S::kCallsM];
#pragma unroll
  for (int i = 0; i < S::kCallsM; ++i) {
    const int idx = tid + i * kT;
    rowM[i] = la.row(idx < BN * 8 ? m0 + idx % BN : m0 + BN);   // past the tile: unused
  }

  // pixel tiles blockIdx.x, + gridDim.x, ...; slices are numbered across the
  // tiles (cg) for the stages' mbarrier phases
  int cg = 0;
  for (int tile = blockIdx.x; tile < ntiles && !s_fail; tile += gridDim.x) {
    const int n0 = tile * kT5N;
    const typename LB::Row rowN = lb.row(n0 + rn);
    bool started = false;   // thread 0: an MMA has written this tile's accumulator
    for (int c = 0; c < nslice; ++c, ++cg) {
      const int st = cg & 1;
      unsigned char* sn = smem + st * S::kStage;
      unsigned char* sm = sn + TB * S::kTermN;
      if (cg >= 2 &&
          !t5::mbar_wait(t5::smem_u32(&s_bar[st]), (uint32_t)(((cg >> 1) - 1) & 1), kT5Spin))
        s_fail = 1;
      const int k0 = kbeg + c * kT5K;
      {
        float vn[S::kCallsN][8], vm[S::kCallsM][8];
#pragma unroll
        for (int i = 0; i < S::kCallsN; ++i) lb.load8(rowN, k0 + (tid / kT5N + 2 * i) * 8, kend, vn[i]);
#pragma unroll
        for (int i = 0; i < S::kCallsM; ++i) {
          const int idx = tid + i * kT;
          if (idx < BN * 8) la.load8(rowM[i], k0 + (idx / BN) * 8, kend, vm[i]);
        }
#pragma unroll
        for (int i = 0; i < S::kCallsN; ++i)
          stage_terms128<TB>(sn, S::kTermN, rn, tid / kT5N + 2 * i, vn[i]);
#pragma unroll
        for (int i = 0; i < S::kCallsM; ++i) {
          const int idx = tid + i * kT;
          if (idx < BN * 8) stage_terms128<TA>(sm, S::kTermM, idx % BN, idx / BN, vm[i]);
        }
      }
      t5::fence_proxy_async();
      __syncthreads();
      if (s_fail) break;   // uniform after the barrier
      if (tid == 0) {
        t5::fence_after();
        const uint32_t an = t5::smem_u32(sn), bm = t5::smem_u32(sm);
#pragma unroll
        for (int kk = 0; kk < kT5K / 16; ++kk) {
#pragma unroll
          for (int i = TB - 1; i >= 0; --i)       // smallest terms first
#pragma unroll
            for (int j = TA - 1; j >= 0; --j) {
              if (i + j >= TMAX) continue;
              const uint64_t ad = t5::desc_sw128(an + i * S::kTermN) + (uint64_t)(kk * 2);
              const uint64_t bd = t5::desc_sw128(bm + j * S::kTermM) + (uint64_t)(kk * 2);
              t5::mma_bf16(tmem, ad, bd, kIdesc, started ? 1u : 0u);   // the first one overwrites
              started = true;
            }
        }
        t5::mma_commit(t5::smem_u32(&s_bar[st]));
      }
    }
    if (s_fail) break;
    if (nslice > 0) {   // this tile's last slice (commits complete in order)
      const int cl = cg - 1;
      if (!t5::mbar_wait(t5::smem_u32(&s_bar[cl & 1]), (uint32_t)((cl >> 1) & 1), kT5Spin))
        s_fail = 1;
    }
    t5::fence_after();
    __syncthreads();
    if (s_fail) break;
    const int q = warp & 3, h = warp >> 2;
    const int n = n0 + 32 * q + lane;
    const bool split = gridDim.z > 1;
#pragma unroll 1
    for (int g = 0; g < BN / 16; ++g) {
      const int col = h * (BN / 2) + 8 * g;
      float v[8];
      if (nslice > 0) {
        t5::tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col, v);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
      }
      if (n < out.N) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int m = m0 + col + e;
          if (m < out.M) out.store(m, n, v[e], split);
        }
      }
    }
    // the next tile's MMAs overwrite the accumulator after every warp has read it
    t5::fence_before();
    __syncthreads();
  }
  if (s_fail && tid == 0) atomicExch(&g_t5_timeout, 1);
  t5::fence_before();
  __syncthreads();
  if (warp == 0) t5::tmem_dealloc(tmem, BN);
}

template <int BN, int TA, int TB, class OUT, class LA, class LB>
cudaError_t t5_launch_bn(const OUT& o, int K, LA la, LB lb, int splits, cudaStream_t s) {
  using S = T5Shape<BN, TA, TB>;
  auto kern = t5_gemm_kernel<LA, LB, OUT, BN, TA, TB>;
  static unsigned long long attr_set = 0;   // per device: shared-memory opt-in done
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !(attr_set >> dev & 1)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmem);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set |= 1ULL << dev;
  }
  splits = std::max(1, std::min(splits, cdiv(K, kT5K)));
  const int kchunk = cdiv(cdiv(K, splits), kT5K) * kT5K;
  splits = cdiv(K, kchunk);
  // one pixel tile per CTA (measured faster than fewer CTAs looping over
  // tiles, with one or two CTAs per SM); the kernel loops when the grid is
  // capped
  const int ntiles = cdiv(o.N, kT5N);
  dim3 grid((unsigned)std::min(ntiles, 65535), cdiv(o.M, BN), splits);
  kern<<<grid, kT, S::kSmem, s>>>(o, la, lb, K, kchunk);
  return cudaGetLastError();
}

// Channel tile: all of M up to 256 (the smallest of 32, 64, 128, 256 that holds it).
inline int t5_bn(int M) { return M <= 32 ? 32 : M <= 64 ? 64 : M <= 128 ? 128 : 256; }

template <int TA, int TB, class OUT, class LA, class LB>
cudaError_t tc_launch(const OUT& o, int K, LA la, LB lb, int splits, cudaStream_t s) {
  if (o.M <= 0 || o.N <= 0) return cudaSuccess;
  switch (t5_bn(o.M)) {
    case 32: return t5_launch_bn<32, TA, TB>(o, K, la, lb, splits, s);
    case 64: return t5_launch_bn<64, TA, TB>(o, K, la, lb, splits, s);
    case 128: return t5_launch_bn<128, TA, TB>(o, K, la, lb, splits, s);
    default: return t5_launch_bn<256, TA, TB>(o, K, la, lb, splits, s);
  }
}

// Split-K factor for the weight gradients (reductions over all pixels).
int wgrad_splits(int M, int N, int K) {
  const long long tiles = (long long)cdiv(M, t5_bn(M)) * cdiv(N, kT5N);
  const long long want = std::max<long long>(1, 152 * 2 / std::max<long long>(tiles, 1));
  return (int)std::min<long long>(want, std::max(1, K / 1024));
}


// ---------------------------------------------------------------------------
// Convolutions from activations split in advance.  A 3x3 convolution reads
// every activation nine times (once per tap) from the tiles of every output
// channel block; splitting it into bfloat16 terms inside each CTA repeats
// that work and keeps the gathers in registers.  Instead the activation
// X [C][P] is split once into three planes, term j at planes + j P C, each
// pixel's C terms contiguous ([P][C], C a multiple of 8): the 64 k of a
// slice (one tap, 64 channels, or two taps of 32) of one pixel are then
// 16-byte runs that cp.async copies straight into the 128-byte-swizzled
// K-major tile, zero-filled outside the image.  The weight operand A(m, k)
// (one bfloat16 term) is laid out once per call as rows of K bfloat16
// (arrange_rows_kernel), so its 16-byte runs are copied the same way.  The
// copies of the next kStages - 1 slices are in flight while the tensor cores
// work on this one.  The split is the same rounding as stage_terms128<3>
// (and <1> for the weights), so the products are those of t5_gemm_kernel.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) split_planes_kernel(const float* __restrict__ X, int C,
                                                           long long P,
                                                           __nv_bfloat16* __restrict__ planes) {
  __shared__ float tile[32][33];
  const long long p0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = c0 + ty + 8 * i;
    const long long p = p0 + tx;
    tile[ty + 8 * i][tx] = (c < C && p < P) ? X[(size_t)c * P + p] : 0.f;
  }
  __syncthreads();
  const size_t plane = (size_t)P * C;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long p = p0 + ty + 8 * i;
    const int c = c0 + tx;
    if (p >= P || c >= C) continue;
    float v = tile[tx][ty + 8 * i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const __nv_bfloat16 t = __float2bfloat16_rn(v);
      planes[j * plane + (size_t)p * C + c] = t;
      v -= __bfloat162float(t);
    }
  }
}

cudaError_t split_planes(const float* X, int C, long long P, __nv_bfloat16* planes,
                         cudaStream_t s) {
  split_planes_kernel<<<dim3((unsigned)cdiv(P, 32), (unsigned)cdiv(C, 32)), 256, 0, s>>>(X, C, P,
                                                                                        planes);
  return cudaGetLastError();
}

// A(m, k) of a loader as bfloat16 rows of K (K a multiple of 8), one thread
// per 8 consecutive k.
template <class LA>
__global__ void __launch_bounds__(256) arrange_rows_kernel(LA la, int M, int K,
                                                           __nv_bfloat16* __restrict__ out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int kc = K / 8;
  if (q >= (long long)M * kc) return;
  const int m = (int)(q / kc), k = (int)(q - (long long)m * kc) * 8;
  float v[8];
  la.load8(la.row(m), k, K, v);
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
  *reinterpret_cast<uint4*>(out + (size_t)m * K + k) = make_uint4(w[0], w[1], w[2], w[3]);
}

template <class LA>
cudaError_t arrange_rows(LA la, int M, int K, __nv_bfloat16* out, cudaStream_t s) {
  const long long n = (long long)M * (K / 8);
  arrange_rows_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(la, M, K, out);
  return cudaGetLastError();
}

constexpr int kConvChunksN = kT5N * 8 / kT;   // 16-byte chunks of the 128-row side per thread

// Operand source of t5_conv_kernel.  A source places one 64-wide K slice
// of both operands as 16-byte copies: the GEMM's N side (the MMA's 128 rows,
// kTB bfloat16 terms) and its M side (BN rows, kTA terms).  off_n / off_m
// give the element offset of term 0 of a chunk of 8 consecutive k, or -1
// where the chunk is zero; term j lies stride_n (stride_m) elements further.
// (Weight gradients through row-shifted two-term planes of X were measured
// too: the same bytes move either way, and the training step did not gain.)

// 3x3 convolution: N rows are pixels p, k = t C + c with tap t = 3u + v,
// B(p, k) = X[c][img, y+u-1, x+v-1] from planes [3][P][C] (C a multiple of
// 8); A(m, k) the weights as bfloat16 rows of K.
struct ConvSrc {
  static constexpr int kTA = 1, kTB = 3;
  const __nv_bfloat16* wa;
  const __nv_bfloat16* planes;
  long long P;
  int H, W, C, M, K;
  struct State {
    long long pix[kConvChunksN];
    int py[kConvChunksN], px[kConvChunksN];
  };
  __device__ void tile(State& st, int n0, int tid) const {
    const int HW = H * W;
#pragma unroll
    for (int i = 0; i < kConvChunksN; ++i) {
      const long long p = n0 + ((tid + i * kT) >> 3);
      st.pix[i] = p < P ? p : -1;
      const int rem = p < P ? (int)(p % HW) : 0;
      st.py[i] = rem / W;
      st.px[i] = rem - st.py[i] * W;
    }
  }
  __device__ long long off_n(const State& st, int i, int k, int kend) const {
    if (st.pix[i] < 0 || k >= kend) return -1;
    const int t = k / C, ch = k - t * C;
    const int du = t / 3 - 1, dv = t % 3 - 1;
    const int yy = st.py[i] + du, xx = st.px[i] + dv;
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) return -1;
    return (st.pix[i] + (long long)du * W + dv) * C + ch;
  }
  __device__ long long off_m(int m, int k, int kend) const {
    return m < M && k < kend ? (long long)m * K + k : -1;
  }
  __device__ const __nv_bfloat16* base_n() const { return planes; }
  __device__ const __nv_bfloat16* base_m() const { return wa; }
  __device__ size_t stride_n() const { return (size_t)P * C; }
  __device__ size_t stride_m() const { return 0; }
};

template <int BN, int TA, int TB>
struct T5ConvShape {
  static constexpr int kTermN = kT5N * 128;                 // one 128-row term tile
  static constexpr int kTermM = BN * 128;                   // one BN-row term tile
  static constexpr int kStage = TB * kTermN + TA * kTermM;
  static constexpr int kFit = (227 * 1024 - 1024 - 256) / kStage;
  static constexpr int kStages = kFit > 4 ? 4 : kFit;
  static constexpr int kSmem = kStages * kStage + 1024;
  static constexpr int kChunksM = (BN * 8 + kT - 1) / kT;    // 16-byte M-side chunks per thread
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <class OUT, class SRC, int BN>
__global__ void __launch_bounds__(kT, 1) t5_conv_kernel(OUT out, SRC src, int K, int kchunk) {
  constexpr int TA = SRC::kTA, TB = SRC::kTB, TMAX = TA > TB ? TA : TB;
  using S = T5ConvShape<BN, TA, TB>;
  constexpr int NS = S::kStages;
  namespace t5 = slim::t5;
  extern __shared__ unsigned char t5_raw[];
  __shared__ uint64_t s_bar[NS];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(t5_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  const int nslice = kend > kbeg ? (kend - kbeg + kT5K - 1) / kT5K : 0;
  const int ntiles = (out.N + kT5N - 1) / kT5N;
  constexpr uint32_t kIdesc = t5::idesc_bf16(kT5N, BN);

  if (tid == 0) {
    for (int i = 0; i < NS; ++i) t5::mbar_init(t5::smem_u32(&s_bar[i]), 1);
    s_fail = 0;
    t5::fence_barrier_init();
  }
  if (warp == 0) t5::tmem_alloc(t5::smem_u32(&s_tmem), BN);
  t5::fence_before();
  __syncthreads();
  t5::fence_after();
  const uint32_t tmem = s_tmem;

  int cg = 0;   // slices across the CTA's tiles: stage cg % NS, phase cg / NS
  for (int tile = blockIdx.x; tile < ntiles && !s_fail; tile += gridDim.x) {
    const int n0 = tile * kT5N;
    typename SRC::State st;
    src.tile(st, n0, tid);
    // this thread's copies of slice c into stage sg: chunk q = tid + 256 i is
    // row q / 8, k-chunk q % 8 (a warp covers four rows' 128-byte runs)
    auto issue = [&](int c, int sg) {
      const uint32_t sn = t5::smem_u32(smem + sg * S::kStage), sm = sn + TB * S::kTermN;
#pragma unroll
      for (int i = 0; i < S::kChunksM; ++i) {
        const int q = tid + i * kT, row = q >> 3, g = q & 7;
        if (row >= BN) break;
        const long long o = src.off_m(m0 + row, kbeg + c * kT5K + 8 * g, kend);
        const __nv_bfloat16* b = src.base_m() + (o >= 0 ? o : 0);
#pragma unroll
        for (int j = 0; j < TA; ++j)
          cp_async16(sm + j * S::kTermM + t5::sw128_off(row, g), o >= 0 ? b + j * src.stride_m() : b,
                     o >= 0 ? 16u : 0u);
      }
#pragma unroll
      for (int i = 0; i < kConvChunksN; ++i) {
        const int q = tid + i * kT, row = q >> 3, g = q & 7;
        const long long o = src.off_n(st, i, kbeg + c * kT5K + 8 * g, kend);
        const __nv_bfloat16* b = src.base_n() + (o >= 0 ? o : 0);
#pragma unroll
        for (int j = 0; j < TB; ++j)
          cp_async16(sn + j * S::kTermN + t5::sw128_off(row, g), o >= 0 ? b + j * src.stride_n() : b,
                     o >= 0 ? 16u : 0u);
      }
    };
#pragma unroll 1
    for (int c = 0; c < NS - 1; ++c) {
      if (c < nslice) issue(c, (cg + c) % NS);
      cp_async_commit();
    }
    bool started = false;
    for (int c = 0; c < nslice; ++c, ++cg) {
      const int sg = cg % NS;
      // the prefetch of slice c + NS - 1 reuses the stage of slice cg - 1:
      // its products must be done
      if (c + NS - 1 < nslice) {
        if (cg >= 1 && !t5::mbar_wait(t5::smem_u32(&s_bar[(cg - 1) % NS]),
                                      (uint32_t)(((cg - 1) / NS) & 1), kT5Spin))
          s_fail = 1;
        if (!s_fail) issue(c + NS - 1, (cg + NS - 1) % NS);
      }
      cp_async_commit();
      cp_async_wait<NS - 1>();   // this thread's copies of slice c have landed
      t5::fence_proxy_async();
      __syncthreads();
      if (s_fail) break;   // uniform after the barrier
      if (tid == 0) {
        t5::fence_after();
        const uint32_t an = t5::smem_u32(smem + sg * S::kStage), bm = an + TB * S::kTermN;
#pragma unroll
        for (int kk = 0; kk < kT5K / 16; ++kk) {
#pragma unroll
          for (int i = TB - 1; i >= 0; --i)   // smallest terms first, as t5_gemm_kernel
#pragma unroll
            for (int j = TA - 1; j >= 0; --j) {
              if (i + j >= TMAX) continue;
              const uint64_t ad = t5::desc_sw128(an + i * S::kTermN) + (uint64_t)(kk * 2);
              const uint64_t bd = t5::desc_sw128(bm + j * S::kTermM) + (uint64_t)(kk * 2);
              t5::mma_bf16(tmem, ad, bd, kIdesc, started ? 1u : 0u);
              started = true;
            }
        }
        t5::mma_commit(t5::smem_u32(&s_bar[sg]));
      }
    }
    if (s_fail) break;
    if (nslice > 0) {
      const int cl = cg - 1;
      if (!t5::mbar_wait(t5::smem_u32(&s_bar[cl % NS]), (uint32_t)((cl / NS) & 1), kT5Spin))
        s_fail = 1;
    }
    t5::fence_after();
    __syncthreads();
    if (s_fail) break;
    const int q = warp & 3, h = warp >> 2;
    const int n = n0 + 32 * q + lane;
    const bool split = gridDim.z > 1;
#pragma unroll 1
    for (int g = 0; g < BN / 16; ++g) {
      const int col = h * (BN / 2) + 8 * g;
      float v[8];
      if (nslice > 0) {
        t5::tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col, v);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
      }
      if (n < out.N) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int m = m0 + col + e;
          if (m < out.M) out.store(m, n, v[e], split);
        }
      }
    }
    t5::fence_before();
    __syncthreads();
  }
  cp_async_wait_all();   // no copy is left in flight into the CTA's shared memory
  if (s_fail && tid == 0) atomicExch(&g_t5_timeout, 1);
  t5::fence_before();
  __syncthreads();
  if (warp == 0) t5::tmem_dealloc(tmem, BN);
}

template <int BN, class OUT, class SRC>
cudaError_t t5_conv_launch_bn(const OUT& o, int K, const SRC& src, int splits, cudaStream_t s) {
  using S = T5ConvShape<BN, SRC::kTA, SRC::kTB>;
  auto kern = t5_conv_kernel<OUT, SRC, BN>;
  static unsigned long long attr_set = 0;   // per device: shared-memory opt-in done
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !(attr_set >> dev & 1)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmem);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set |= 1ULL << dev;
  }
  splits = std::max(1, std::min(splits, cdiv(K, kT5K)));
  const int kchunk = cdiv(cdiv(K, splits), kT5K) * kT5K;
  splits = cdiv(K, kchunk);
  const int ntiles = cdiv(o.N, kT5N);
  dim3 grid((unsigned)std::min(ntiles, 65535), cdiv(o.M, BN), splits);
  kern<<<grid, kT, S::kSmem, s>>>(o, src, K, kchunk);
  return cudaGetLastError();
}

template <class OUT, class SRC>
cudaError_t conv_launch(const OUT& o, int K, const SRC& src, int splits, cudaStream_t s) {
  if (o.M <= 0 || o.N <= 0) return cudaSuccess;
  switch (t5_bn(o.M)) {
    case 32: return t5_conv_launch_bn<32>(o, K, src, splits, s);
    case 64: return t5_conv_launch_bn<64>(o, K, src, splits, s);
    case 128: return t5_conv_launch_bn<128>(o, K, src, splits, s);
    default: return t5_conv_launch_bn<256>(o, K, src, splits, s);
  }
}

// ---------------------------------------------------------------------------
// Layout kernels
// ---------------------------------------------------------------------------
// 2x2 max-pool: first maximum in row-major window order (arg in 0..3).
__global__ void maxpool_kernel(const float* __restrict__ X, int C, int n, int H, int W, float* Y,
                               unsigned char* arg) {
  const int H2 = H / 2, W2 = W / 2;
  const long long Q = (long long)n * H2 * W2, total = (long long)C * Q;
  const long long P = (long long)n * H * W;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / Q);
    const long long q = idx % Q;
    const int img = (int)(q / ((long long)H2 * W2));
    const int rem = (int)(q % ((long long)H2 * W2));
    const int y = 2 * (rem / W2), x = 2 * (rem % W2);
    const float* base = X + (size_t)c * P + ((size_t)img * H + y) * W + x;
    const float v[4] = {base[0], base[1], base[W], base[W + 1]};
    int a = 0;
    for (int t = 1; t < 4; ++t)
      if (v[t] > v[a]) a = t;
    Y[idx] = v[a];
    arg[idx] = (unsigned char)a;
  }
}

// dX (holding the skip gradient) += the pooled gradient routed to its argmax.
__global__ void maxpool_bwd_kernel(const float* __restrict__ dY, const unsigned char* arg, int C,
                                   int n, int H, int W, float* dX) {
  const int H2 = H / 2, W2 = W / 2;
  const long long Q = (long long)n * H2 * W2, total = (long long)C * Q;
  const long long P = (long long)n * H * W;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / Q);
    const long long q = idx % Q;
    const int img = (int)(q / ((long long)H2 * W2));
    const int rem = (int)(q % ((long long)H2 * W2));
    const int a = arg[idx];
    const int y = 2 * (rem / W2) + a / 2, x = 2 * (rem % W2) + a % 2;
    dX[(size_t)c * P + ((size_t)img * H + y) * W + x] += dY[idx];
  }
}

// db[c] += sum_p dY[c][p]: blockIdx.x = channel, blockIdx.y strides over
// chunks of pixels; one atomic add per CTA.
__global__ void rowsum_kernel(const float* __restrict__ dY, long long P, float* db) {
  const int c = blockIdx.x;
  float s = 0.f;
  for (long long p = blockIdx.y * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.y * blockDim.x)
    s += dY[(size_t)c * P + p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float red[kT / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kT / 32; ++w) t += red[w];
    atomicAdd(db + c, t);
  }
}

// Row sums of dY [C][P] added into db, with about 4 CTAs per SM in total.
cudaError_t rowsum(const float* dY, int C, long long P, float* db, cudaStream_t s) {
  const long long per = std::max<long long>(1, std::min<long long>(cdiv(P, kT), cdiv(4 * 152, C)));
  rowsum_kernel<<<dim3(C, (unsigned)per), kT, 0, s>>>(dY, P, db);
  return cudaGetLastError();
}

__global__ void relu_mask_kernel(float* d, const float* __restrict__ y, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    if (!(y[i] > 0.f)) d[i] = 0.f;
}

// ---------------------------------------------------------------------------
// Layers (CNHW: channel c of image i at row c, column i*H*W + y*W + x)
// ---------------------------------------------------------------------------
// y[m][p] = max?(y[m][p] + b[m], 0) after a split-K accumulation.
__global__ void bias_act_kernel(float* Y, const float* __restrict__ b, int relu, int M, long long P) {
  const long long total = (long long)M * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    float v = Y[i];
    if (b) v += b[i / P];
    if (relu) v = fmaxf(v, 0.f);
    Y[i] = v;
  }
}

// k-splits for an output GEMM whose tile grid alone would leave SMs idle
// (the deep levels): enough CTAs for two per SM, at least 8 k-slabs each.
int out_splits(int M, int N, int K) {
  const long long tiles = (long long)cdiv(M, t5_bn(M)) * cdiv(N, kT5N);
  if (tiles >= 152) return 1;
  const long long want = cdiv(152, tiles);
  return (int)std::max<long long>(1, std::min<long long>(want, K / (4 * kT5K)));
}

// C [M][N] (contiguous) = op + bias, ReLU: one pass when the grid fills the
// GPU, else zero, split-K atomics and a bias / ReLU pass.
template <int TA, int TB, class LA, class LB>
cudaError_t gemm_out(float* C, int M, int N, int K, LA la, LB lb, const float* bias, bool relu,
                     cudaStream_t s) {
  const int splits = out_splits(M, N, K);
  if (splits == 1)
    return tc_launch<TA, TB>(OutPlain{C, N, M, N, bias, relu ? 1 : 0, 0}, K, la, lb, 1, s);
  cudaError_t e = cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), s);
  if (e != cudaSuccess) return e;
  e = tc_launch<TA, TB>(OutPlain{C, N, M, N, nullptr, 0, 1}, K, la, lb, splits, s);
  if (e != cudaSuccess || (!bias && !relu)) return e;
  bias_act_kernel<<<grid_for((long long)M * N), kT, 0, s>>>(C, bias, relu ? 1 : 0, M, N);
  return cudaGetLastError();
}

// gemm_out with both operands copied asynchronously (t5_conv_kernel): the
// weight operand laid out at wa (M x K bfloat16), the pixel operand from the
// planes of the gathered tensor (C_g channels, [3][P][C_g]).
template <class LA>
cudaError_t conv_out(float* C, int M, int N, int K, LA la, __nv_bfloat16* wa,
                     const __nv_bfloat16* planes, long long P, int H, int W, int Cg,
                     const float* bias, bool relu, cudaStream_t s) {
  cudaError_t e = arrange_rows(la, M, K, wa, s);
  if (e != cudaSuccess) return e;
  const ConvSrc src{wa, planes, P, H, W, Cg, M, K};
  const int splits = out_splits(M, N, K);
  if (splits == 1)
    return conv_launch(OutPlain{C, N, M, N, bias, relu ? 1 : 0, 0}, K, src, 1, s);
  e = cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), s);
  if (e != cudaSuccess) return e;
  e = conv_launch(OutPlain{C, N, M, N, nullptr, 0, 1}, K, src, splits, s);
  if (e != cudaSuccess || (!bias && !relu)) return e;
  bias_act_kernel<<<grid_for((long long)M * N), kT, 0, s>>>(C, bias, relu ? 1 : 0, M, N);
  return cudaGetLastError();
}

// Bytes of the planes of a C x P activation; 0 when C is not a multiple of 8
// (those convolutions gather and split in the CTA).
size_t planes_bytes(int C, long long P) { return C % 8 ? 0 : 3 * (size_t)C * P * sizeof(__nv_bfloat16); }
// Bytes of the laid-out weight operand of a 3x3 convolution (either direction).
size_t conv_weight_bytes(int Ci, int Co) { return 9 * (size_t)Ci * Co * sizeof(__nv_bfloat16); }

// Y = W * col(X) + b (ReLU): M = C_out, N = pixels, K = 9 C_in (tap-major).
// With scratch for the planes (planes_bytes(C_in, P)) and the weights
// (conv_weight_bytes) both operands are laid out once and copied
// asynchronously.
cudaError_t conv3x3_fwd(const float* X, int n, int Ci, int H, int W, const float* Wt,
                        const float* b, int Co, bool relu, float* Y, cudaStream_t s,
                        __nv_bfloat16* planes = nullptr, __nv_bfloat16* wa = nullptr) {
  const long long P = (long long)n * H * W;
  if (planes && wa && Ci % 8 == 0) {
    cudaError_t e = split_planes(X, Ci, P, planes, s);
    if (e != cudaSuccess) return e;
    return conv_out(Y, Co, (int)P, 9 * Ci, LoadWTap{Wt, Ci, Co}, wa, planes, P, H, W, Ci, b, relu,
                    s);
  }
  return gemm_out<1, 3>(Y, Co, (int)P, 9 * Ci, LoadWTap{Wt, Ci, Co}, LoadPixTap{X, P, H, W, Ci}, b,
                        relu, s);
}

// dY is the gradient at the conv's output (before any ReLU).
//   dW += dY col(X)^T      M = C_out, N = 9 C_in, K = pixels (split-K)
//   db += row sums of dY
//   dX  = Wf col(dY)       the adjoint conv, Wf[c][t*C_out + o] = W[o][c][8-t]:
//                          M = C_in, N = pixels, K = 9 C_out
cudaError_t conv3x3_bwd(const float* X, const float* dY, int n, int Ci, int H, int W,
                        const float* Wt, int Co, float* dW, float* db, float* dX, cudaStream_t s,
                        __nv_bfloat16* planes = nullptr, __nv_bfloat16* wa = nullptr) {
  const long long P = (long long)n * H * W;
  const int K9 = 9 * Ci;
  cudaError_t e = tc_launch<2, 2>(OutPlain{dW, K9, Co, K9, nullptr, 0, 1}, (int)P,
                                  LoadRowK{dY, P, Co}, LoadTapPix{X, P, H, W, K9},
                                  wgrad_splits(Co, K9, (int)P), s);
  if (e != cudaSuccess) return e;
  if (db && (e = rowsum(dY, Co, P, db, s)) != cudaSuccess) return e;
  if (!dX) return cudaSuccess;
  if (planes && wa && Co % 8 == 0) {
    if ((e = split_planes(dY, Co, P, planes, s)) != cudaSuccess) return e;
    return conv_out(dX, Ci, (int)P, 9 * Co, LoadFlipW{Wt, Ci, Co}, wa, planes, P, H, W, Co, nullptr,
                    false, s);
  }
  return gemm_out<1, 3>(dX, Ci, (int)P, 9 * Co, LoadFlipW{Wt, Ci, Co}, LoadPixTap{dY, P, H, W, Co},
                        nullptr, false, s);
}

// 2x2 stride-2 transposed conv, W [C_in][C_out][2][2]: Y4 = W^T X with
// M = 4 C_out, N = input pixels, K = C_in, each value written to its place
// on the 2x grid (plus bias) by the epilogue.
cudaError_t tconv2x2_fwd(const float* X, int n, int Ci, int H, int W, const float* Wt,
                         const float* b, int Co, float* Y, cudaStream_t s) {
  const long long Pin = (long long)n * H * W;
  return tc_launch<1, 3>(OutUp{Y, 4 * Pin, 4 * Co, (int)Pin, W, b}, Ci,
                         LoadKRow{Wt, 4LL * Co, 4 * Co}, LoadKRow{X, Pin, (int)Pin}, 1, s);
}

//   dW += X dY4^T    M = C_in, N = 4 C_out, K = input pixels (split-K)
//   db += row sums of dY
//   dX  = W dY4      M = C_in, N = input pixels, K = 4 C_out
// with dY4[o*4+u*2+v][p] = dY[o][2R+u][2x+v] gathered by the loaders.
cudaError_t tconv2x2_bwd(const float* X, const float* dY, int n, int Ci, int H, int W,
                         const float* Wt, int Co, float* dW, float* db, float* dX, cudaStream_t s) {
  const long long Pin = (long long)n * H * W;
  cudaError_t e = tc_launch<2, 2>(OutPlain{dW, 4LL * Co, Ci, 4 * Co, nullptr, 0, 1}, (int)Pin,
                                  LoadRowK{X, Pin, Ci}, LoadUpTapPix{dY, 4 * Pin, W, 4 * Co},
                                  wgrad_splits(Ci, 4 * Co, (int)Pin), s);
  if (e != cudaSuccess) return e;
  if (db && (e = rowsum(dY, Co, 4 * Pin, db, s)) != cudaSuccess) return e;
  if (!dX) return cudaSuccess;
  return tc_launch<1, 3>(OutPlain{dX, Pin, Ci, (int)Pin, nullptr, 0, 0}, 4 * Co,
                         LoadRowK{Wt, 4LL * Co, Ci}, LoadUpPix{dY, 4 * Pin, W, (int)Pin}, 1, s);
}

// grad = 2 (y - t) / count;  loss += sum (y - t)^2
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, long long count,
                           float* grad, double* loss) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    grad[i] = 2.f * d / (float)count;
    s += (double)d * d;
  }
  __shared__ double red[kT];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// Adam (Kingma and Ba, 2015) on the float32 master copy; refreshes the
// forward copy (bfloat16-rounded weights, unrounded biases).
__global__ void adam_kernel(float* master, float* eff, const float* __restrict__ g, float* m,
                            float* v, const unsigned char* __restrict__ is_w, long long count,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float p = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    master[i] = p;
    eff[i] = is_w[i] ? __bfloat162float(__float2bfloat16_rn(p)) : p;
  }
}

__global__ void refresh_eff_kernel(const float* __restrict__ master, float* eff,
                                   const unsigned char* __restrict__ is_w, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    eff[i] = is_w[i] ? __bfloat162float(__float2bfloat16_rn(master[i])) : master[i];
}

__global__ void scale_copy_kernel(const float* __restrict__ in, float* out, long long count,
                                  float s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = s * in[i];
}

// ---------------------------------------------------------------------------
// The network
// ---------------------------------------------------------------------------
enum Kind { kConv = 0, kTconv = 1, kConv1 = 2 };
struct LayerSpec {
  const char* name;
  int o, i, kind;   // conv: o x i x 3 x 3; tconv: i x o x 2 x 2 (in, out); conv1: o x i
};
// in the order of the oracle's parameter list
const LayerSpec kLayers[] = {
    {"enc1a", 32, 1, kConv},    {"enc1b", 32, 32, kConv},   {"enc2a", 64, 32, kConv},
    {"enc2b", 64, 64, kConv},   {"enc3a", 128, 64, kConv},  {"enc3b", 128, 128, kConv},
    {"bota", 256, 128, kConv},  {"botb", 256, 256, kConv},  {"up3", 128, 256, kTconv},
    {"dec3a", 128, 256, kConv}, {"dec3b", 128, 128, kConv}, {"up2", 64, 128, kTconv},
    {"dec2a", 64, 128, kConv},  {"dec2b", 64, 64, kConv},   {"up1", 32, 64, kTconv},
    {"dec1a", 32, 64, kConv},   {"dec1b", 32, 32, kConv},   {"out", 1, 32, kConv1},
};
constexpr int kNumLayers = sizeof(kLayers) / sizeof(kLayers[0]);
enum {
  L_ENC1A, L_ENC1B, L_ENC2A, L_ENC2B, L_ENC3A, L_ENC3B, L_BOTA, L_BOTB, L_UP3, L_DEC3A, L_DEC3B,
  L_UP2, L_DEC2A, L_DEC2B, L_UP1, L_DEC1A, L_DEC1B, L_OUT
};

long long weight_count(const LayerSpec& l) {
  return l.kind == kConv ? 9LL * l.o * l.i : l.kind == kTconv ? 4LL * l.o * l.i : (long long)l.o * l.i;
}

}  // namespace

struct slim_unet {
  int H = 0, W = 0, max_n = 0;
  long long nparams = 0;
  long long woff[kNumLayers] = {}, boff[kNumLayers] = {};
  float *master = nullptr, *eff = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  unsigned char* is_w = nullptr;
  long long t = 0;
  // activations (channel-major over the batch) and their gradients
  float *x = nullptr, *a1 = nullptr, *c1 = nullptr, *p1 = nullptr, *a2 = nullptr, *c2 = nullptr,
        *p2 = nullptr, *a3 = nullptr, *c3 = nullptr, *p3 = nullptr, *ab = nullptr, *bt = nullptr,
        *d3a = nullptr, *d3 = nullptr, *d2a = nullptr, *d2 = nullptr, *d1a = nullptr,
        *d1 = nullptr, *y = nullptr;
  float *ga1 = nullptr, *gc1 = nullptr, *gp1 = nullptr, *ga2 = nullptr, *gc2 = nullptr,
        *gp2 = nullptr, *ga3 = nullptr, *gc3 = nullptr, *gp3 = nullptr, *gab = nullptr,
        *gbt = nullptr, *gd3a = nullptr, *gd3 = nullptr, *gd2a = nullptr, *gd2 = nullptr,
        *gd1a = nullptr, *gd1 = nullptr, *gy = nullptr;
  unsigned char *arg1 = nullptr, *arg2 = nullptr, *arg3 = nullptr;
  __nv_bfloat16* planes = nullptr;   // a convolution input (or output gradient) split into terms
  __nv_bfloat16* wa = nullptr;       // a convolution's weight operand laid out as rows of K
  double* loss = nullptr;
  std::vector<void*> allocs;
};

namespace {

struct Net {
  slim_unet* u;
  int n;
  cudaStream_t s;
  long long P(int level) const {   // pixels at level 1..4
    return (long long)n * (u->H >> (level - 1)) * (u->W >> (level - 1));
  }
  int h(int level) const { return u->H >> (level - 1); }
  int w(int level) const { return u->W >> (level - 1); }
  const float* W_(int l) const { return u->eff + u->woff[l]; }
  const float* B_(int l) const { return u->eff + u->boff[l]; }
  float* gW(int l) const { return u->grad + u->woff[l]; }
  float* gB(int l) const { return u->grad + u->boff[l]; }

  cudaError_t conv(int l, const float* X, int level, float* Y, bool relu) const {
    const LayerSpec& L = kLayers[l];
    return conv3x3_fwd(X, n, L.i, h(level), w(level), W_(l), B_(l), L.o, relu, Y, s, u->planes,
                       u->wa);
  }
  // dY holds the gradient at the ReLU output; on return dX (if any) holds the
  // gradient at the layer input.
  cudaError_t conv_back(int l, const float* X, int level, const float* Yout, float* dY, float* dX) const {
    const LayerSpec& L = kLayers[l];
    const long long count = (long long)L.o * P(level);
    relu_mask_kernel<<<grid_for(count), kT, 0, s>>>(dY, Yout, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return conv3x3_bwd(X, dY, n, L.i, h(level), w(level), W_(l), L.o, gW(l), gB(l), dX, s,
                       u->planes, u->wa);
  }
  // transposed conv from level `lin` (input) to lin-1
  cudaError_t tconv(int l, const float* X, int lin, float* Y) const {
    const LayerSpec& L = kLayers[l];
    return tconv2x2_fwd(X, n, L.i, h(lin), w(lin), W_(l), B_(l), L.o, Y, s);
  }
  cudaError_t tconv_back(int l, const float* X, int lin, const float* dY, float* dX) const {
    const LayerSpec& L = kLayers[l];
    return tconv2x2_bwd(X, dY, n, L.i, h(lin), w(lin), W_(l), L.o, gW(l), gB(l), dX, s);
  }
  cudaError_t pool(const float* X, int level, float* Y, unsigned char* arg, int C) const {
    maxpool_kernel<<<grid_for((long long)C * P(level + 1)), kT, 0, s>>>(X, C, n, h(level), w(level), Y, arg);
    return cudaGetLastError();
  }
  cudaError_t pool_back(const float* dY, const unsigned char* arg, int level, float* dX, int C) const {
    maxpool_bwd_kernel<<<grid_for((long long)C * P(level + 1)), kT, 0, s>>>(dY, arg, C, n, h(level),
                                                                           w(level), dX);
    return cudaGetLastError();
  }

  cudaError_t forward() const {
    slim_unet& U = *u;
    cudaError_t e;
#define CKE(x) if ((e = (x)) != cudaSuccess) return e
    // the encoder output of each level goes to the lower rows of its concat buffer
    float* e1 = U.c1 + 32 * P(1);
    float* e2 = U.c2 + 64 * P(2);
    float* e3 = U.c3 + 128 * P(3);
    CKE(conv(L_ENC1A, U.x, 1, U.a1, true));
    CKE(conv(L_ENC1B, U.a1, 1, e1, true));
    CKE(pool(e1, 1, U.p1, U.arg1, 32));
    CKE(conv(L_ENC2A, U.p1, 2, U.a2, true));
    CKE(conv(L_ENC2B, U.a2, 2, e2, true));
    CKE(pool(e2, 2, U.p2, U.arg2, 64));
    CKE(conv(L_ENC3A, U.p2, 3, U.a3, true));
    CKE(conv(L_ENC3B, U.a3, 3, e3, true));
    CKE(pool(e3, 3, U.p3, U.arg3, 128));
    CKE(conv(L_BOTA, U.p3, 4, U.ab, true));
    CKE(conv(L_BOTB, U.ab, 4, U.bt, true));
    CKE(tconv(L_UP3, U.bt, 4, U.c3));
    CKE(conv(L_DEC3A, U.c3, 3, U.d3a, true));
    CKE(conv(L_DEC3B, U.d3a, 3, U.d3, true));
    CKE(tconv(L_UP2, U.d3, 3, U.c2));
    CKE(conv(L_DEC2A, U.c2, 2, U.d2a, true));
    CKE(conv(L_DEC2B, U.d2a, 2, U.d2, true));
    CKE(tconv(L_UP1, U.d2, 2, U.c1));
    CKE(conv(L_DEC1A, U.c1, 1, U.d1a, true));
    CKE(conv(L_DEC1B, U.d1a, 1, U.d1, true));
    return gemm<false, false>(1, (int)P(1), 32, W_(L_OUT), 32, U.d1, (int)P(1), U.y, (int)P(1),
                              B_(L_OUT), false, false, 1, s);
  }

  // Gradients of the loss whose gradient at y is in gy (grad buffer zeroed first).
  cudaError_t backward() const {
    slim_unet& U = *u;
    cudaError_t e;
    float* e1 = U.c1 + 32 * P(1);
    float* e2 = U.c2 + 64 * P(2);
    float* e3 = U.c3 + 128 * P(3);
    float* ge1 = U.gc1 + 32 * P(1);
    float* ge2 = U.gc2 + 64 * P(2);
    float* ge3 = U.gc3 + 128 * P(3);
    const int P1 = (int)P(1);
    // output 1x1 conv
    CKE((gemm<false, true>(1, 32, P1, U.gy, P1, U.d1, P1, gW(L_OUT), 32, nullptr, false, true,
                           wgrad_splits(1, 32, P1), s)));
    CKE(rowsum(U.gy, 1, P(1), gB(L_OUT), s));
    CKE((gemm<true, false>(32, P1, 1, W_(L_OUT), 32, U.gy, P1, U.gd1, P1, nullptr, false, false, 1, s)));
    // level 1 decoder
    CKE(conv_back(L_DEC1B, U.d1a, 1, U.d1, U.gd1, U.gd1a));
    CKE(conv_back(L_DEC1A, U.c1, 1, U.d1a, U.gd1a, U.gc1));
    CKE(tconv_back(L_UP1, U.d2, 2, U.gc1, U.gd2));
    CKE(conv_back(L_DEC2B, U.d2a, 2, U.d2, U.gd2, U.gd2a));
    CKE(conv_back(L_DEC2A, U.c2, 2, U.d2a, U.gd2a, U.gc2));
    CKE(tconv_back(L_UP2, U.d3, 3, U.gc2, U.gd3));
    CKE(conv_back(L_DEC3B, U.d3a, 3, U.d3, U.gd3, U.gd3a));
    CKE(conv_back(L_DEC3A, U.c3, 3, U.d3a, U.gd3a, U.gc3));
    CKE(tconv_back(L_UP3, U.bt, 4, U.gc3, U.gbt));
    CKE(conv_back(L_BOTB, U.ab, 4, U.bt, U.gbt, U.gab));
    CKE(conv_back(L_BOTA, U.p3, 4, U.ab, U.gab, U.gp3));
    // encoder: skip gradient (already in the concat gradient) + pooled gradient
    CKE(pool_back(U.gp3, U.arg3, 3, ge3, 128));
    CKE(conv_back(L_ENC3B, U.a3, 3, e3, ge3, U.ga3));
    CKE(conv_back(L_ENC3A, U.p2, 3, U.a3, U.ga3, U.gp2));
    CKE(pool_back(U.gp2, U.arg2, 2, ge2, 64));
    CKE(conv_back(L_ENC2B, U.a2, 2, e2, ge2, U.ga2));
    CKE(conv_back(L_ENC2A, U.p1, 2, U.a2, U.ga2, U.gp1));
    CKE(pool_back(U.gp1, U.arg1, 1, ge1, 32));
    CKE(conv_back(L_ENC1B, U.a1, 1, e1, ge1, U.ga1));
    CKE(conv_back(L_ENC1A, U.x, 1, U.a1, U.ga1, nullptr));
#undef CKE
    return cudaSuccess;
  }
};

void unet_free(slim_unet* u) {
  for (void* p : u->allocs) cudaFree(p);
  u->allocs.clear();
}

}  // namespace

extern "C" {

slim_status slim_unet_param_count(long long* count) {
  if (!count) return SLIM_EINVAL;
  long long c = 0;
  for (const LayerSpec& l : kLayers) c += weight_count(l) + (l.kind == kTconv ? l.o : l.o);
  *count = c;
  return SLIM_OK;
}

namespace {
bool layer_sizes_ok(int n, int ci, int H, int W, int co) {
  return n > 0 && ci > 0 && H > 0 && W > 0 && co > 0 && ci <= 65536 && co <= 65536 &&
         4LL * n * H * W < (1LL << 31);
}
slim_status layer_status(cudaError_t e) { return e == cudaSuccess ? SLIM_OK : SLIM_ECUDA; }
}  // namespace

namespace {
// Planes and weight-layout scratch of the standalone layer calls, one block
// from the stream-ordered pool (none when the planes do not apply).
struct PlanesScratch {
  __nv_bfloat16* p = nullptr;
  __nv_bfloat16* w = nullptr;
  cudaStream_t s;
  PlanesScratch(size_t planes, size_t weights, cudaStream_t st) : s(st) {
    if (!planes) return;
    const size_t off = (planes + 255) / 256 * 256;
    unsigned char* q = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&q), off + weights, s) != cudaSuccess) {
      cudaGetLastError();
      return;   // the convolution then gathers and splits in the CTA
    }
    p = reinterpret_cast<__nv_bfloat16*>(q);
    w = reinterpret_cast<__nv_bfloat16*>(q + off);
  }
  ~PlanesScratch() {
    if (p) cudaFreeAsync(p, s);
  }
};
}  // namespace

slim_status slim_unet_conv3x3(const float* x, int n, int c_in, int H, int W, const float* w,
                              const float* b, int c_out, int relu, float* y, void* stream) {
  if (!x || !w || !y || !layer_sizes_ok(n, c_in, H, W, c_out)) return SLIM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  PlanesScratch ps(planes_bytes(c_in, (long long)n * H * W), conv_weight_bytes(c_in, c_out), s);
  return layer_status(conv3x3_fwd(x, n, c_in, H, W, w, b, c_out, relu != 0, y, s, ps.p, ps.w));
}

slim_status slim_unet_conv3x3_grad(const float* x, const float* dy, int n, int c_in, int H, int W,
                                   const float* w, int c_out, float* dw, float* db, float* dx,
                                   void* stream) {
  if (!x || !dy || !w || !dw || !layer_sizes_ok(n, c_in, H, W, c_out)) return SLIM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  PlanesScratch ps(dx ? planes_bytes(c_out, (long long)n * H * W) : 0, conv_weight_bytes(c_in, c_out),
                   s);
  return layer_status(conv3x3_bwd(x, dy, n, c_in, H, W, w, c_out, dw, db, dx, s, ps.p, ps.w));
}

slim_status slim_unet_tconv2x2(const float* x, int n, int c_in, int H, int W, const float* w,
                               const float* b, int c_out, float* y, void* stream) {
  if (!x || !w || !y || !layer_sizes_ok(n, c_in, H, W, c_out)) return SLIM_EINVAL;
  return layer_status(tconv2x2_fwd(x, n, c_in, H, W, w, b, c_out, y, (cudaStream_t)stream));
}

slim_status slim_unet_tconv2x2_grad(const float* x, const float* dy, int n, int c_in, int H, int W,
                                    const float* w, int c_out, float* dw, float* db, float* dx,
                                    void* stream) {
  if (!x || !dy || !w || !dw || !layer_sizes_ok(n, c_in, H, W, c_out)) return SLIM_EINVAL;
  return layer_status(tconv2x2_bwd(x, dy, n, c_in, H, W, w, c_out, dw, db, dx, (cudaStream_t)stream));
}

slim_status slim_unet_create(int H, int W, int max_batch, slim_unet** out) {
  if (!out) return SLIM_EINVAL;
  *out = nullptr;
  if (H < 8 || W < 8 || H % 8 || W % 8 || max_batch < 1 || (long long)H * W * max_batch > (1LL << 24))
    return SLIM_EINVAL;
  slim_unet* u = new (std::nothrow) slim_unet();
  if (!u) return SLIM_ENOMEM;
  u->H = H;
  u->W = W;
  u->max_n = max_batch;
  long long off = 0;
  for (int l = 0; l < kNumLayers; ++l) {
    u->woff[l] = off;
    off += weight_count(kLayers[l]);
    u->boff[l] = off;
    off += kLayers[l].o;
  }
  u->nparams = off;
  const long long P1 = (long long)max_batch * H * W, P2 = P1 / 4, P3 = P1 / 16, P4 = P1 / 64;
  bool ok = true;
  auto fa = [&](float** p, long long count) {
    if (!ok) return;
    void* q = nullptr;
    if (cudaMalloc(&q, (size_t)count * sizeof(float)) != cudaSuccess) { ok = false; return; }
    u->allocs.push_back(q);
    *p = (float*)q;
  };
  auto ba = [&](unsigned char** p, long long count) {
    if (!ok) return;
    void* q = nullptr;
    if (cudaMalloc(&q, (size_t)count) != cudaSuccess) { ok = false; return; }
    u->allocs.push_back(q);
    *p = (unsigned char*)q;
  };
  fa(&u->master, off); fa(&u->eff, off); fa(&u->grad, off); fa(&u->m, off); fa(&u->v, off);
  ba(&u->is_w, off);
  fa(&u->x, P1); fa(&u->a1, 32 * P1); fa(&u->c1, 64 * P1); fa(&u->p1, 32 * P2);
  fa(&u->a2, 64 * P2); fa(&u->c2, 128 * P2); fa(&u->p2, 64 * P3); fa(&u->a3, 128 * P3);
  fa(&u->c3, 256 * P3); fa(&u->p3, 128 * P4); fa(&u->ab, 256 * P4); fa(&u->bt, 256 * P4);
  fa(&u->d3a, 128 * P3); fa(&u->d3, 128 * P3); fa(&u->d2a, 64 * P2); fa(&u->d2, 64 * P2);
  fa(&u->d1a, 32 * P1); fa(&u->d1, 32 * P1); fa(&u->y, P1);
  fa(&u->ga1, 32 * P1); fa(&u->gc1, 64 * P1); fa(&u->gp1, 32 * P2); fa(&u->ga2, 64 * P2);
  fa(&u->gc2, 128 * P2); fa(&u->gp2, 64 * P3); fa(&u->ga3, 128 * P3); fa(&u->gc3, 256 * P3);
  fa(&u->gp3, 128 * P4); fa(&u->gab, 256 * P4); fa(&u->gbt, 256 * P4); fa(&u->gd3a, 128 * P3);
  fa(&u->gd3, 128 * P3); fa(&u->gd2a, 64 * P2); fa(&u->gd2, 64 * P2); fa(&u->gd1a, 32 * P1);
  fa(&u->gd1, 32 * P1); fa(&u->gy, P1);
  ba(&u->arg1, 32 * P2); ba(&u->arg2, 64 * P3); ba(&u->arg3, 128 * P4);
  {
    // the largest planes any 3x3 convolution needs (its input forward, its
    // output gradient backward) at the level it runs on (kLayers order; 0:
    // not a 3x3 convolution)
    static const int kLevel[] = {1, 1, 2, 2, 3, 3, 4, 4, 0, 3, 3, 0, 2, 2, 0, 1, 1, 0};
    static_assert(sizeof(kLevel) / sizeof(kLevel[0]) == kNumLayers, "one level per layer");
    const long long Pl[5] = {0, P1, P2, P3, P4};
    size_t need = 0;
    for (int l = 0; l < kNumLayers; ++l) {
      if (!kLevel[l]) continue;
      const LayerSpec& L = kLayers[l];
      need = std::max(need, std::max(planes_bytes(L.i, Pl[kLevel[l]]), planes_bytes(L.o, Pl[kLevel[l]])));
    }
    unsigned char* q = nullptr;
    ba(&q, (long long)need);
    u->planes = reinterpret_cast<__nv_bfloat16*>(q);
    size_t wneed = 0;
    for (int l = 0; l < kNumLayers; ++l)
      if (kLayers[l].kind == kConv) wneed = std::max(wneed, conv_weight_bytes(kLayers[l].i, kLayers[l].o));
    q = nullptr;
    ba(&q, (long long)wneed);
    u->wa = reinterpret_cast<__nv_bfloat16*>(q);
  }
  if (ok) {
    void* q = nullptr;
    ok = cudaMalloc(&q, sizeof(double)) == cudaSuccess;
    if (ok) { u->allocs.push_back(q); u->loss = (double*)q; }
  }
  if (ok) {
    std::vector<unsigned char> isw((size_t)off, 0);
    for (int l = 0; l < kNumLayers; ++l)
      std::fill(isw.begin() + u->woff[l], isw.begin() + u->boff[l], 1);
    ok = cudaMemcpy(u->is_w, isw.data(), isw.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(u->master, 0, off * sizeof(float)) == cudaSuccess &&
         cudaMemset(u->eff, 0, off * sizeof(float)) == cudaSuccess &&
         cudaMemset(u->m, 0, off * sizeof(float)) == cudaSuccess &&
         cudaMemset(u->v, 0, off * sizeof(float)) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    unet_free(u);
    delete u;
    return SLIM_ENOMEM;
  }
  *out = u;
  return SLIM_OK;
}

void slim_unet_destroy(slim_unet* u) {
  if (!u) return;
  cudaDeviceSynchronize();
  unet_free(u);
  delete u;
}

slim_status slim_unet_set_params(slim_unet* u, const float* params, long long count) {
  if (!u || !params || count != u->nparams) return SLIM_EINVAL;
  if (cudaMemcpy(u->master, params, count * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(u->m, 0, count * sizeof(float)) != cudaSuccess ||
      cudaMemset(u->v, 0, count * sizeof(float)) != cudaSuccess)
    return SLIM_ECUDA;
  refresh_eff_kernel<<<grid_for(count), kT>>>(u->master, u->eff, u->is_w, count);
  u->t = 0;
  return cudaDeviceSynchronize() == cudaSuccess ? SLIM_OK : SLIM_ECUDA;
}

slim_status slim_unet_get_params(slim_unet* u, float* params, long long count) {
  if (!u || !params || count != u->nparams) return SLIM_EINVAL;
  return cudaMemcpy(params, u->master, count * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
             ? SLIM_OK : SLIM_ECUDA;
}

slim_status slim_unet_get_grads(slim_unet* u, float* grads, long long count) {
  if (!u || !grads || count != u->nparams) return SLIM_EINVAL;
  return cudaMemcpy(grads, u->grad, count * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
             ? SLIM_OK : SLIM_ECUDA;
}

slim_status slim_unet_forward(slim_unet* u, const float* x, float* y, int n, void* stream) {
  if (!u || !x || !y || n < 1 || n > u->max_n) return SLIM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const long long P1 = (long long)n * u->H * u->W;
  Net net{u, n, s};
  if (cudaMemcpyAsync(u->x, x, P1 * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SLIM_ECUDA;
  if (net.forward() != cudaSuccess) return SLIM_ECUDA;
  if (cudaMemcpyAsync(y, u->y, P1 * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SLIM_ECUDA;
  return SLIM_OK;
}

slim_status slim_unet_train_step(slim_unet* u, const float* x, const float* target, int n, float lr,
                                 double* loss, void* stream) {
  if (!u || !x || !target || n < 1 || n > u->max_n || !(lr >= 0.f)) return SLIM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const long long P1 = (long long)n * u->H * u->W;
  Net net{u, n, s};
  if (cudaMemcpyAsync(u->x, x, P1 * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(u->grad, 0, u->nparams * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(u->loss, 0, sizeof(double), s) != cudaSuccess)
    return SLIM_ECUDA;
  if (net.forward() != cudaSuccess) return SLIM_ECUDA;
  mse_kernel<<<grid_for(P1), kT, 0, s>>>(u->y, target, P1, u->gy, u->loss);
  if (cudaGetLastError() != cudaSuccess || net.backward() != cudaSuccess) return SLIM_ECUDA;
  u->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)std::pow(0.9, (double)u->t);
  const float c2 = 1.f - (float)std::pow(0.999, (double)u->t);
  adam_kernel<<<grid_for(u->nparams), kT, 0, s>>>(u->master, u->eff, u->grad, u->m, u->v, u->is_w,
                                                  u->nparams, lr, b1, b2, 1e-8f, c1, c2);
  if (cudaGetLastError() != cudaSuccess) return SLIM_ECUDA;
  if (loss) {
    double h = 0.0;
    if (cudaMemcpyAsync(&h, u->loss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SLIM_ECUDA;
    *loss = h / (double)P1;
  }
  return SLIM_OK;
}

}  // extern "C"

namespace slim {
int unet_height(const slim_unet* net) { return net->H; }
int unet_width(const slim_unet* net) { return net->W; }

// out = s * in (the warm start's input and output scaling).
cudaError_t unet_scale(const float* in, float* out, long long count, float s, cudaStream_t st) {
  scale_copy_kernel<<<grid_for(count), kT, 0, st>>>(in, out, count, s);
  return cudaGetLastError();
}
}  // namespace slim
