// Float32-accurate products on the tcgen05 tensor cores, the triangular
// inverse of a Cholesky factor built on them, and the matrix-vector products
// that apply that inverse (declarations and the arithmetic in slim_tc.cuh).
//
// One CTA computes a 128 x BN tile of C (BN = 128, or 64 for products too
// small to fill the GPU with the wide tile).  For each 64-wide slice of K its
// 256 threads load the float32 operand tiles (either storage order), split
// every value into three bfloat16 terms and store each term tile in the
// K-major, 128-byte-swizzled shared-memory layout the MMA reads.  One thread
// then issues the six term products of each 16-wide K step as tcgen05.mma
// (M = 128, N = BN, K = 16, float32 accumulation in tensor memory) and
// commits them to an mbarrier of that stage; with two stages the loads of
// slice s+1 overlap the MMAs of slice s.  After the last slice the eight
// warps read the accumulator from tensor memory (each warp its 32-lane
// quarter and half of the columns) and write alpha acc + beta C.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <cuda_bf16.h>

#include "slim_chol.cuh"
#include "slim_device.cuh"
#include "slim_grid.cuh"
#include "slim_lookahead.cuh"
#include "slim_tc.cuh"
#include "slim_tcgen05.cuh"

namespace slim {

namespace {

constexpr int kThreads = 256;
constexpr int kStages = 2;
constexpr int kTermA = kTcBM * kTcBK * 2;            // bytes of one bfloat16 term tile of A
constexpr unsigned kSpinLimit = 1u << 24;            // mbarrier polls before giving up

// The shape of a 128 x BN output tile.
template <int BN>
struct TcTile {
  static constexpr int kTermB = BN * kTcBK * 2;                 // bytes of one term tile of B
  static constexpr int kStageBytes = 3 * kTermA + 3 * kTermB;   // 72 KB (BN 64), 96 KB (128)
  static constexpr int kTmemCols = BN;                          // float32 accumulator: a column per n
  static constexpr int kHalfN = BN / 2;                         // accumulator columns per epilogue warp
  static constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024;
};

// PTX wrappers (slim_tcgen05.cuh), with this kernel's instruction shape
using t5::desc_sw128;
using t5::fence_barrier_init;
using t5::fence_proxy_async;
using t5::mbar_init;
using t5::mma_commit;
using t5::smem_u32;
using t5::tmem_alloc;
using t5::tmem_dealloc;
using t5::tmem_ld8;
__device__ __forceinline__ void tc_fence_before() { t5::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { t5::fence_after(); }
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return t5::mbar_wait(bar, parity, kSpinLimit);
}
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) { return desc_sw128(addr); }
// Instruction descriptor: M = 128, N = BN
template <int BN>
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  constexpr uint32_t kIdesc = t5::idesc_bf16(kTcBM, BN);
  t5::mma_bf16(tmem_d, adesc, bdesc, kIdesc, accumulate);
}

// ----------------------------------------------------------------------------
// Operand staging
// ----------------------------------------------------------------------------
// Split 8 consecutive float32 values into three 16-byte chunks of bfloat16
// terms (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); the
// differences are exact in float32).
__device__ __forceinline__ void split8(const float (&x)[8], uint4& t0, uint4& t1, uint4& t2) {
  uint32_t w0[4], w1[4], w2[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t h0[2], h1[2], h2[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float v = x[2 * q + e];
      const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(b0);
      const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(b1);
      const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
      h0[e] = __bfloat16_as_ushort(b0);
      h1[e] = __bfloat16_as_ushort(b1);
      h2[e] = __bfloat16_as_ushort(b2);
    }
    w0[q] = h0[0] | (h0[1] << 16);
    w1[q] = h1[0] | (h1[1] << 16);
    w2[q] = h2[0] | (h2[1] << 16);
  }
  t0 = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  t1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
  t2 = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

using t5::sw128_off;

// Stage rows [0, R) x k [k0, k0 + 64) of op(X) into the three term tiles at
// `dst` (term t at dst + t * R * 128).  op(X)[r][k] is X[(r0 + r) * ld + k]
// (km = 0) or X[k * ld + r0 + r] (km = 1); rows at or beyond `rows` are
// zero.  tri = 1 reads op(X)[r][k] as zero for k > r0 + r, tri = 2 for
// k < r0 + r (a triangular operand whose other triangle holds other data).
// R * 64 / 256 values per thread, in runs of 8 consecutive k (one 16-byte
// chunk per term each), loaded, split and stored one run at a time.
// A thread's share of one operand stage: R * 64 / 256 values of op(X) in
// runs of 8 consecutive k (one 16-byte chunk per bfloat16 term each).
//   K-contiguous rows (km = 0): eight lanes per 64-float row, two float4
//     each, so a warp reads four whole rows per pass (R / 32 passes);
//   K-strided rows (X[k][m], km = 1): consecutive lanes take consecutive rows
//     m, so every load reads a contiguous run of one k row.
// All of the stage's loads are issued first (load_operand), then the values
// are masked, split and stored (store_operand): one memory round trip per
// stage instead of one per run.
template <int R>
struct StageMap {
  static constexpr int kPer = R * kTcBK / kThreads;   // 32 (R = 128) or 16 (R = 64)
  __device__ __forceinline__ static void at(int km, int c, int& row, int& kc) {
    const int tid = threadIdx.x;
    if (km == 0) {
      row = (tid >> 3) + 32 * c;
      kc = 8 * (tid & 7);
    } else {
      row = tid % R;
      kc = (tid / R) * kPer + 8 * c;
    }
  }
};

template <int R>
__device__ __forceinline__ void load_operand(float (&v)[StageMap<R>::kPer], const float* X,
                                             long long ld, int km, int r0, int rows, int k0) {
  constexpr int kRuns = StageMap<R>::kPer / 8;
#pragma unroll
  for (int c = 0; c < kRuns; ++c) {
    int row, kc;
    StageMap<R>::at(km, c, row, kc);
    const int rg = r0 + row;
    if (rg >= rows) {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[8 * c + e] = 0.f;
    } else if (km == 0) {
      const float4* src = reinterpret_cast<const float4*>(X + (long long)rg * ld + k0 + kc);
      const float4 q0 = __ldg(src), q1 = __ldg(src + 1);
      v[8 * c + 0] = q0.x; v[8 * c + 1] = q0.y; v[8 * c + 2] = q0.z; v[8 * c + 3] = q0.w;
      v[8 * c + 4] = q1.x; v[8 * c + 5] = q1.y; v[8 * c + 6] = q1.z; v[8 * c + 7] = q1.w;
    } else {
      const float* src = X + (long long)(k0 + kc) * ld + rg;
#pragma unroll
      for (int e = 0; e < 8; ++e) v[8 * c + e] = __ldg(src + (long long)e * ld);
    }
  }
}

// tri = 1 reads op(X)[r][k] as zero for k > r0 + r, tri = 2 for k < r0 + r
// (a triangular operand whose other triangle holds other data).
template <int R>
__device__ __forceinline__ void store_operand(unsigned char* dst, const float (&v)[StageMap<R>::kPer],
                                              int km, int r0, int k0, int tri) {
  constexpr int kRuns = StageMap<R>::kPer / 8;
#pragma unroll
  for (int c = 0; c < kRuns; ++c) {
    int row, kc;
    StageMap<R>::at(km, c, row, kc);
    const int rg = r0 + row;
    float x8[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + kc + e;
      x8[e] = (tri == 1 && k > rg) || (tri == 2 && k < rg) ? 0.f : v[8 * c + e];
    }
    uint4 t0, t1, t2;
    split8(x8, t0, t1, t2);
    const uint32_t off = sw128_off(row, kc / 8);
    *reinterpret_cast<uint4*>(dst + off) = t0;
    *reinterpret_cast<uint4*>(dst + R * 128 + off) = t1;
    *reinterpret_cast<uint4*>(dst + 2 * R * 128 + off) = t2;
  }
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const TcProblem* probs, int* status) {
  using Tile = TcTile<BN>;
  constexpr int kStageBytes = Tile::kStageBytes, kTermB = Tile::kTermB;
  constexpr int kTmemCols = Tile::kTmemCols, kHalfN = Tile::kHalfN;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t s_bar[kStages];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const TcProblem pb = probs[blockIdx.z];
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * BN;
  if (m0 >= pb.M || n0 >= pb.N) return;   // uniform: the whole CTA leaves
  if (pb.c_lower && n0 >= m0 + kTcBM) return;   // wholly above the diagonal
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

  // K range of this tile (triangular operands contribute nothing outside it)
  int kbeg = 0, kend = pb.K;
  if (pb.k_from_n) kbeg = n0;
  if (pb.k_to_m) kend = min(kend, m0 + kTcBM);
  const int nchunk = kend > kbeg ? (kend - kbeg) / kTcBK : 0;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&s_bar[s]), 1);
    s_fail = 0;
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  for (int c = 0; c < nchunk; ++c) {
    const int st = c % kStages;
    unsigned char* sa = smem + st * kStageBytes;
    unsigned char* sb = sa + 3 * kTermA;
    if (c >= kStages) {
      // the MMAs of slice c - kStages read this stage: wait for their commit
      if (!mbar_wait(smem_u32(&s_bar[st]), (uint32_t)((c / kStages - 1) & 1))) s_fail = 1;
    }
    const int k0 = kbeg + c * kTcBK;
    {
      float va[StageMap<kTcBM>::kPer], vb[StageMap<BN>::kPer];
      load_operand<kTcBM>(va, pb.A, pb.lda, pb.a_km, m0, pb.M, k0);
      load_operand<BN>(vb, pb.B, pb.ldb, pb.b_kn, n0, pb.N, k0);
      store_operand<kTcBM>(sa, va, pb.a_km, m0, k0, pb.k_to_m ? 1 : 0);
      store_operand<BN>(sb, vb, pb.b_kn, n0, k0, pb.k_from_n ? 2 : 0);
    }
    fence_proxy_async();
    __syncthreads();
    if (s_fail) break;   // uniform after the barrier
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk) {
        // six term products a_i b_j, i + j <= 2, smallest first
        const int ta[6] = {2, 1, 0, 1, 0, 0};
        const int tb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint64_t ad = smem_desc_sw128(a0 + ta[q] * kTermA) + (uint64_t)(kk * 2);
          const uint64_t bd = smem_desc_sw128(b0 + tb[q] * kTermB) + (uint64_t)(kk * 2);
          mma_bf16<BN>(tmem, ad, bd, (c > 0 || kk > 0 || q > 0) ? 1u : 0u);
        }
      }
      mma_commit(smem_u32(&s_bar[st]));
    }
  }
  // wait for the last slice's products (commits complete in order)
  if (nchunk > 0 && !s_fail) {
    const int cl = nchunk - 1;
    if (!mbar_wait(smem_u32(&s_bar[cl % kStages]), (uint32_t)((cl / kStages) & 1))) s_fail = 1;
  }
  tc_fence_after();
  __syncthreads();
  if (s_fail) {
    if (tid == 0) set_status(status, SLIM_ETIMEOUT);
  } else {
    // epilogue: warp w reads lanes 32 (w % 4) .. +31 and half w / 4 of the
    // columns, 8 columns at a time
    const int q = warp & 3, h = warp >> 2;
    const int row = 32 * q + lane;
    if (pb.c_nm == 0) {
      // through shared memory (the operand stages are free once the last
      // commit has arrived), then whole rows of C in 16-byte stores
      constexpr int kCsLd = BN + 4;
      float* Cs = reinterpret_cast<float*>(smem);
#pragma unroll 1
      for (int g = 0; g < BN / 16; ++g) {
        float acc[8];
        if (nchunk > 0) {
          tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kHalfN * h + 8 * g), acc);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[i] = 0.f;
        }
        float4* dst = reinterpret_cast<float4*>(Cs + row * kCsLd + kHalfN * h + 8 * g);
        dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
      }
      __syncthreads();
      const bool vec = (pb.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(pb.C) & 15) == 0;
      // a row of C is BN / 4 16-byte pieces: BN / 4 threads per row
      constexpr int kPieces = BN / 4, kRowsPerPass = kThreads / kPieces;
      const int c4 = tid % kPieces, rr = tid / kPieces;
#pragma unroll 2
      for (int pass = 0; pass < kTcBM / kRowsPerPass; ++pass) {
        const int r = rr + kRowsPerPass * pass, m = m0 + r, n = n0 + 4 * c4;
        if (m >= pb.M || n >= pb.N) continue;
        const float4 a = *reinterpret_cast<const float4*>(Cs + r * kCsLd + 4 * c4);
        float* cp = pb.C + (long long)m * pb.ldc + n;
        if (vec && n + 3 < pb.N) {
          float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
          if (pb.beta != 0.f) o = *reinterpret_cast<const float4*>(cp);
          o.x = pb.alpha * a.x + pb.beta * o.x;
          o.y = pb.alpha * a.y + pb.beta * o.y;
          o.z = pb.alpha * a.z + pb.beta * o.z;
          o.w = pb.alpha * a.w + pb.beta * o.w;
          *reinterpret_cast<float4*>(cp) = o;
        } else {
          const float av[4] = {a.x, a.y, a.z, a.w};
          for (int e = 0; e < 4 && n + e < pb.N; ++e) {
            const float old = pb.beta != 0.f ? cp[e] : 0.f;
            cp[e] = pb.alpha * av[e] + pb.beta * old;
          }
        }
      }
    } else {
      // C stored transposed: consecutive lanes hold consecutive m, so each
      // column n is one contiguous 128-byte run per warp
      const int m = m0 + row;
#pragma unroll 1
      for (int g = 0; g < BN / 16; ++g) {
        float acc[8];
        if (nchunk > 0) {
          tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kHalfN * h + 8 * g), acc);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[i] = 0.f;
        }
        if (m >= pb.M) continue;
        const int nb = n0 + kHalfN * h + 8 * g;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = nb + j;
          if (n < pb.N) {
            float* cp = pb.C + (long long)n * pb.ldc + m;
            const float old = pb.beta != 0.f ? *cp : 0.f;
            *cp = pb.alpha * acc[j] + pb.beta * old;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ----------------------------------------------------------------------------
// Pre-split operands and the product that streams them
// ----------------------------------------------------------------------------
constexpr int kPlaneTileBytes = 3 * kTermA;   // the three term tiles of 128 rows x 64 k: 48 KB
using t5::bulk_g2s;
using t5::mbar_arrive;
using t5::mbar_arrive_expect_tx;

// One CTA per 128 x 64 tile of op(X): the staging code of tc_gemm_kernel,
// writing the term tiles to global memory instead of shared memory.
__global__ void __launch_bounds__(kThreads) tc_split_kernel(const TcSplitJob* jobs) {
  const TcSplitJob j = jobs[blockIdx.y];
  const int KT = j.K / kTcBK, RT = (j.rows + kTcBM - 1) / kTcBM;
  const int t = blockIdx.x;
  if (t >= RT * KT) return;
  const int rt = t / KT, kt = t - rt * KT;
  // tiles wholly in the zero triangle: no product reads them
  if (j.tri == 1 && kt * kTcBK > rt * kTcBM + kTcBM - 1) return;
  if (j.tri == 2 && kt * kTcBK + kTcBK - 1 < rt * kTcBM) return;
  float v[StageMap<kTcBM>::kPer];
  load_operand<kTcBM>(v, j.X, j.ld, j.km, rt * kTcBM, j.rows, kt * kTcBK);
  store_operand<kTcBM>(j.planes + (size_t)t * kPlaneTileBytes, v, j.km, rt * kTcBM, kt * kTcBK,
                       j.tri);
}

// Stage ring of the streaming product: A's three term tiles (48 KB) and B's
// (BN rows each); two stages, of 96 KB for BN = 128 and 72 KB for 64 (the
// narrow tile's 145 KB leave room on the SM for a factorisation CTA).
template <int BN>
struct PlaneTile {
  static constexpr int kTermB = BN * 128;
  static constexpr int kStageBytes = kPlaneTileBytes + 3 * kTermB;
  static constexpr int kStages = 2;
  static constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024;
};
constexpr int kPlaneThreads = 128;   // warp 0 lane 0 loads, warp 1 lane 0 issues; 4 warps store

// C tile (m0, n0) of 128 x BN.  The producer thread waits for a stage to be
// free (the MMAs that read it have committed to its `empty` barrier), arms
// its `full` barrier with the stage's byte count and issues the bulk copies;
// the MMA thread waits for `full`, issues the 24 term products of the slice
// and commits to `empty`, and after the last slice to `done`.  Every wait is
// bounded; after one runs out the CTA still waits (bounded) for its copies
// and products in flight before it frees tensor memory.
template <int BN>
__global__ void __launch_bounds__(kPlaneThreads, 1)
    tc_gemm_planes_kernel(const TcProblem* probs, int* status) {
  using Tile = PlaneTile<BN>;
  constexpr int S = Tile::kStages, kStageBytes = Tile::kStageBytes, kTermB = Tile::kTermB;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t s_full[S], s_empty[S], s_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail, s_issued;
  const TcProblem pb = probs[blockIdx.z];
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * BN;
  if (m0 >= pb.M || n0 >= pb.N) return;
  if (pb.c_lower && n0 >= m0 + kTcBM) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

  int kbeg = 0, kend = pb.K;
  if (pb.k_from_n) kbeg = n0;
  if (pb.k_to_m) kend = min(kend, m0 + kTcBM);
  const int nchunk = kend > kbeg ? (kend - kbeg) / kTcBK : 0;
  const int KT = pb.K / kTcBK, kt0 = kbeg / kTcBK;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(smem_u32(&s_full[st]), 1);
      mbar_init(smem_u32(&s_empty[st]), 1);
    }
    mbar_init(smem_u32(&s_done), 1);
    s_fail = 0;
    s_issued = 0;
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    const unsigned char* a_src = pb.a_planes + (size_t)(m0 / kTcBM) * KT * kPlaneTileBytes;
    const unsigned char* b_src = pb.b_planes + (size_t)(n0 / kTcBM) * KT * kPlaneTileBytes +
                                 (BN == 64 ? (size_t)((n0 / 64) & 1) * kTermB : 0);
    int c = 0;
    for (; c < nchunk; ++c) {
      const int st = c % S;
      if (c >= S && !mbar_wait(smem_u32(&s_empty[st]), (uint32_t)((c / S - 1) & 1))) {
        s_fail = 1;
        break;
      }
      const uint32_t sa = smem_u32(smem + st * kStageBytes), sb = sa + kPlaneTileBytes;
      const uint32_t full = smem_u32(&s_full[st]);
      const size_t kofs = (size_t)(kt0 + c) * kPlaneTileBytes;
      mbar_arrive_expect_tx(full, (uint32_t)kStageBytes);
      bulk_g2s(sa, a_src + kofs, kPlaneTileBytes, full);
      if (BN == kTcBM) {
        bulk_g2s(sb, b_src + kofs, kPlaneTileBytes, full);
      } else {
#pragma unroll
        for (int t = 0; t < 3; ++t)
          bulk_g2s(sb + t * kTermB, b_src + kofs + (size_t)t * kTermA, kTermB, full);
      }
    }
    s_issued = c;
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t kIdescN = t5::idesc_bf16(kTcBM, BN);
    for (int c = 0; c < nchunk; ++c) {
      const int st = c % S;
      if (!mbar_wait(smem_u32(&s_full[st]), (uint32_t)((c / S) & 1))) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(smem + st * kStageBytes), b0 = a0 + kPlaneTileBytes;
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk) {
        // six term products a_i b_j, i + j <= 2, smallest first
        const int ta[6] = {2, 1, 0, 1, 0, 0};
        const int tb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint64_t ad = smem_desc_sw128(a0 + ta[q] * kTermA) + (uint64_t)(kk * 2);
          const uint64_t bd = smem_desc_sw128(b0 + tb[q] * kTermB) + (uint64_t)(kk * 2);
          t5::mma_bf16(tmem, ad, bd, kIdescN, (c > 0 || kk > 0 || q > 0) ? 1u : 0u);
        }
      }
      mma_commit(smem_u32(&s_empty[st]));
    }
    // `done` completes once every product issued above has (at once if none was)
    if (nchunk > 0) {
      mma_commit(smem_u32(&s_done));
    } else {
      mbar_arrive(smem_u32(&s_done));
    }
  }
  __syncwarp();
  if (!mbar_wait(smem_u32(&s_done), 0u)) s_fail = 1;
  tc_fence_after();
  __syncthreads();
  if (s_fail) {
    if (tid == 0) {
      // copies still in flight land before the CTA leaves
      const int issued = s_issued;
      for (int c = issued - S > 0 ? issued - S : 0; c < issued; ++c)
        mbar_wait(smem_u32(&s_full[c % S]), (uint32_t)((c / S) & 1));
      set_status(status, SLIM_ETIMEOUT);
    }
  } else {
    // epilogue: warp w holds accumulator lanes (rows) 32 w .. 32 w + 31
    const int row = 32 * warp + lane;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
    if (pb.c_nm == 0) {
      // through shared memory (the stages are free: every product has completed),
      // then whole rows of C in 16-byte stores
      constexpr int kCsLd = BN + 4;
      float* Cs = reinterpret_cast<float*>(smem);
#pragma unroll 1
      for (int g = 0; g < BN / 8; ++g) {
        float acc[8];
        if (nchunk > 0) {
          tmem_ld8(trow + (uint32_t)(8 * g), acc);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[i] = 0.f;
        }
        float4* dst = reinterpret_cast<float4*>(Cs + row * kCsLd + 8 * g);
        dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
      }
      __syncthreads();
      const bool vec = (pb.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(pb.C) & 15) == 0;
      constexpr int kPieces = BN / 4, kRowsPerPass = kPlaneThreads / kPieces;
      const int c4 = tid % kPieces, rr = tid / kPieces;
#pragma unroll 4
      for (int pass = 0; pass < kTcBM / kRowsPerPass; ++pass) {
        const int r = rr + kRowsPerPass * pass, m = m0 + r, n = n0 + 4 * c4;
        if (m >= pb.M || n >= pb.N) continue;
        const float4 a = *reinterpret_cast<const float4*>(Cs + r * kCsLd + 4 * c4);
        float* cp = pb.C + (long long)m * pb.ldc + n;
        if (vec && n + 3 < pb.N) {
          float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
          if (pb.beta != 0.f) o = *reinterpret_cast<const float4*>(cp);
          o.x = pb.alpha * a.x + pb.beta * o.x;
          o.y = pb.alpha * a.y + pb.beta * o.y;
          o.z = pb.alpha * a.z + pb.beta * o.z;
          o.w = pb.alpha * a.w + pb.beta * o.w;
          *reinterpret_cast<float4*>(cp) = o;
        } else {
          const float av[4] = {a.x, a.y, a.z, a.w};
          for (int e = 0; e < 4 && n + e < pb.N; ++e) {
            const float old = pb.beta != 0.f ? cp[e] : 0.f;
            cp[e] = pb.alpha * av[e] + pb.beta * old;
          }
        }
      }
    } else {
      // C stored transposed: consecutive lanes hold consecutive m, so each
      // column n is one contiguous 128-byte run per warp
      const int m = m0 + row;
#pragma unroll 1
      for (int g = 0; g < BN / 8; ++g) {
        float acc[8];
        if (nchunk > 0) {
          tmem_ld8(trow + (uint32_t)(8 * g), acc);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[i] = 0.f;
        }
        if (m >= pb.M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + 8 * g + j;
          if (n < pb.N) {
            float* cp = pb.C + (long long)n * pb.ldc + m;
            const float old = pb.beta != 0.f ? *cp : 0.f;
            *cp = pb.alpha * acc[j] + pb.beta * old;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, BN);
  }
}

// ----------------------------------------------------------------------------
// Triangular inverse helpers
// ----------------------------------------------------------------------------
// X's diagonal tiles from the factor's tile inverses (zeros above the diagonal).
__global__ void trinv_diag_kernel(const float* W, float* X, int P, int T) {
  const int t = blockIdx.x;
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
    const int r = idx / 64, c = idx % 64;
    X[(size_t)(t * 64 + r) * P + t * 64 + c] = r >= c ? W[(size_t)t * 4096 + idx] : 0.f;
  }
}

// X[j][i] = X[i][j] for i > j: the strict upper triangle takes X^T.  32 x 32
// tiles through shared memory; tile (bi, bj) with bi >= bj.
__global__ void trinv_mirror_kernel(float* X, int P) {
  __shared__ float t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int r = ty; r < 32; r += 8) t[r][tx] = X[(size_t)(bi * 32 + r) * P + bj * 32 + tx];
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + tx, j = bj * 32 + r;   // element (i, j) of the lower triangle
    if (i > j) X[(size_t)j * P + i] = t[tx][r];
  }
}

// The products with X run one warp per row, eight consecutive rows per CTA.
// The CTA first stages the vector over the columns its rows touch in shared
// memory as float32, so the rows (the only large stream, read once) are the
// only global traffic.  A lane takes 16-byte pieces of the row, four in
// flight; float32 products in groups of four, groups summed in float64.
constexpr int kTrRows = kThreads / 32;     // rows per CTA
constexpr int kTrMaxP = 8192;              // largest order (the staged vector: p + 8 floats)

// Stage v[c0 .. c1) as float32 at s_v[c - c0'] where c0' = c0 & ~3 (so that
// 16-byte pieces of the row and of s_v line up).
__device__ __forceinline__ int stage_vec(const double* v, int c0, int c1, float* s_v) {
  const int ca = c0 & ~3;
  for (int c = ca + threadIdx.x; c < c1; c += blockDim.x) s_v[c - ca] = c >= c0 ? (float)v[c] : 0.f;
  __syncthreads();
  return ca;
}

// sum_{j=j0}^{j1-1} row[j] v[j] with v staged from column ca.
__device__ __forceinline__ double warp_row_dot(const float* __restrict__ row, const float* s_v,
                                               int ca, int j0, int j1, int lane) {
  double acc = 0.0;
  if (j1 <= j0) return 0.0;
  const int jh = min(j1, (j0 + 3) & ~3);
  if (j0 + lane < jh) acc = (double)(row[j0 + lane] * s_v[j0 + lane - ca]);
  for (int base = jh; base < j1; base += 512) {
    float4 a[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = base + 128 * t + 4 * lane;
      if (j + 3 < j1) a[t] = __ldg(reinterpret_cast<const float4*>(row + j));
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = base + 128 * t + 4 * lane;
      if (j + 3 < j1) {
        const float4 w = *reinterpret_cast<const float4*>(s_v + (j - ca));
        float g = a[t].x * w.x;
        g = fmaf(a[t].y, w.y, g);
        g = fmaf(a[t].z, w.z, g);
        g = fmaf(a[t].w, w.w, g);
        acc += (double)g;
      } else if (j < j1) {
        float g = 0.f;
        for (int e = j; e < j1; ++e) g = fmaf(row[e], s_v[e - ca], g);
        acc += (double)g;
      }
    }
  }
  return warp_sum(acc);
}

// y[i] = sum_{j=lo..i} X[i][j] v[j] for i in [lo, p).
__global__ void __launch_bounds__(kThreads) trinv_lower_kernel(const float* X, int P, int p,
                                                                int lo, const double* v,
                                                                double* y) {
  extern __shared__ __align__(16) float s_v[];   // p + 8 floats
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = lo + blockIdx.x * kTrRows;
  const int ilast = min(p - 1, i0 + kTrRows - 1);
  const int ca = stage_vec(v, lo, ilast + 1, s_v);
  const int i = i0 + warp;
  if (i >= p) return;
  const double d = warp_row_dot(X + (size_t)i * P, s_v, ca, lo, i + 1, lane);
  if (lane == 0) y[i] = d;
}

// z[j] (+)= sum_{i=max(j,lo)..p-1} X[i][j] y[i]: row j of the upper triangle
// holds X[i][j] at column i.
__global__ void __launch_bounds__(kThreads) trinv_upper_kernel(const float* X, int P, int p,
                                                                int lo, const double* y,
                                                                double* z, int accumulate) {
  extern __shared__ __align__(16) float s_v[];   // p + 8 floats
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = blockIdx.x * kTrRows;
  const int ca = stage_vec(y, max(j0, lo), p, s_v);
  const int j = j0 + warp;
  if (j >= p) return;
  const double d = warp_row_dot(X + (size_t)j * P, s_v, ca, max(j, lo), p, lane);
  if (lane == 0) z[j] = accumulate ? z[j] + d : d;
}

// ----------------------------------------------------------------------------
// The iterate chain of the pipelined tensor-core form as one cooperative
// launch: residual, the first solve, the refinement rounds and the scatter,
// each phase spread over every warp of the grid and separated by bounded grid
// barriers, so the chain waits for SMs once per step instead of once per
// kernel.  Rows go to warps cyclically (warp w of the grid takes rows w,
// w + W, ...), which balances the triangular rows; every CTA stages the
// vector of a phase in shared memory once.
// ----------------------------------------------------------------------------
struct IterTc {
  const StepInfo* info;
  const int* ext;        // [P] factored row -> extended row (-1: empty)
  const float* X;        // L^{-1} (lower) and L^{-T} (strict upper), P x P
  double* y;             // [P] intermediate of the products
  double* res;           // [P] refinement residual
  unsigned* bar;         // grid barrier (zeroed before the launch)
  int refine;            // refinement rounds
};

__device__ __forceinline__ int grid_warp() { return blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); }
__device__ __forceinline__ int grid_warps() { return gridDim.x * (kThreads / 32); }

// y[i] = sum_{j=lo..i} X[i][j] v[j] for i in [lo, p), rows cyclic over the grid's warps.
__device__ void coop_lower(const float* X, int P, int p, int lo, const double* v, double* y,
                           float* s_v) {
  const int ca = stage_vec(v, lo, p, s_v);
  const int lane = threadIdx.x & 31;
  for (int i = lo + grid_warp(); i < p; i += grid_warps()) {
    const double d = warp_row_dot(X + (size_t)i * P, s_v, ca, lo, i + 1, lane);
    if (lane == 0) y[i] = d;
  }
}

// z[j] (+)= sum_{i=max(j,lo)..p-1} X[i][j] y[i] for j in [0, p).
__device__ void coop_upper(const float* X, int P, int p, int lo, const double* y, double* z,
                           int accumulate, float* s_v) {
  const int ca = stage_vec(y, lo, p, s_v);
  const int lane = threadIdx.x & 31;
  for (int j = grid_warp(); j < p; j += grid_warps()) {
    const double d = warp_row_dot(X + (size_t)j * P, s_v, ca, max(j, lo), p, lane);
    if (lane == 0) z[j] = accumulate ? z[j] + d : d;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) iterate_tc_kernel(LaArgs<T> a, IterTc it) {
  extern __shared__ __align__(16) unsigned char smem_it[];
  float* s_v = reinterpret_cast<float*>(smem_it);
  __shared__ int s_flag;
  const int lane = threadIdx.x & 31;
  const int P = a.P, p = a.p, ell = a.ell;
  const int lo = (a.nslots - 1) * ell;   // the newest block's rows: the first right-hand side
  const long long k = it.info->k;
  const int tid_g = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;

  // residual r_k = A_k x - b_k from the stored taps into rhs[lo..p); zeros elsewhere
  for (int i = tid_g; i < P; i += nth)
    if (i < lo || i >= p) a.rhs[i] = 0.0;
  const int eslot = (int)((k - 1) % a.eslots);
  for (int w = grid_warp(); w < ell; w += grid_warps()) {
    const int q = eslot * ell + w;
    const int* rp = a.ring_pix + (size_t)q * a.taps;
    const double* rw = a.ring_w + (size_t)q * a.taps;
    T acc = T(0);
    for (int s2 = lane; s2 < a.N; s2 += 32) {
      const int pa = rp[2 * s2], pb = rp[2 * s2 + 1];
      if (pa >= 0) acc += (T)rw[2 * s2] * a.x[pa];
      if (pb >= 0) acc += (T)rw[2 * s2 + 1] * a.x[pb];
    }
    acc = warp_sum(acc);
    if (lane == 0) a.rhs[lo + w] = (double)(acc - a.b[a.ring_ids[q]]);
  }
  if (!grid_barrier(it.bar, a.status, &s_flag)) return;

  // first solve, z = X^T X rhs: rhs is zero above lo, so y is too
  coop_lower(it.X, P, p, lo, a.rhs, it.y, s_v);
  if (!grid_barrier(it.bar, a.status, &s_flag)) return;
  coop_upper(it.X, P, p, lo, it.y, a.z, 0, s_v);
  if (!grid_barrier(it.bar, a.status, &s_flag)) return;

  // refinement: res = rhs - lambda_k z - G z in float64, z += X^T X res
  const double lam = it.info->lam_k;
  for (int round = 0; round < it.refine; ++round) {
    double* s_z = reinterpret_cast<double*>(smem_it);
    int* s_ext = reinterpret_cast<int*>(s_z + P);
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
      s_z[j] = a.z[j];
      s_ext[j] = it.ext[j];
    }
    __syncthreads();
    for (int row = grid_warp(); row < P; row += grid_warps()) {
      const int ei = s_ext[row];
      double sum = 0.0;
      if (ei >= 0) {
        const double* g = a.G + (size_t)ei * a.Pe;
        for (int base = 0; base < P; base += 256) {
          double gv[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int j = base + 32 * t + lane;
            const int ej = j < P ? s_ext[j] : -1;
            gv[t] = ej >= 0 ? __ldg(g + ej) : 0.0;
          }
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int j = base + 32 * t + lane;
            if (j < P) sum += gv[t] * s_z[j];
          }
        }
      }
      sum = warp_sum(sum);
      if (lane == 0) it.res[row] = a.rhs[row] - lam * s_z[row] - sum;
    }
    if (!grid_barrier(it.bar, a.status, &s_flag)) return;
    coop_lower(it.X, P, p, 0, it.res, it.y, s_v);
    if (!grid_barrier(it.bar, a.status, &s_flag)) return;
    coop_upper(it.X, P, p, 0, it.y, a.z, 1, s_v);
    if (!grid_barrier(it.bar, a.status, &s_flag)) return;
  }

  // scatter x -= eta M_k^T z over the window's rows
  for (int q = grid_warp(); q < p; q += grid_warps()) {
    const int qe = it.ext[q];
    if (qe < 0) continue;
    const T c = (T)(-a.eta * a.z[q]);
    if (c == T(0)) continue;
    const int* rp = a.ring_pix + (size_t)qe * a.taps;
    const double* rw = a.ring_w + (size_t)qe * a.taps;
    for (int t = lane; t < a.taps; t += 32) {
      const int pix = rp[t];
      if (pix >= 0) atomicAdd(&a.x[pix], c * (T)(a.cinv ? rw[t] * a.cinv[pix] : rw[t]));
    }
  }
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

size_t tc_smem_bytes() { return TcTile<kTcBN>::kSmem; }

cudaError_t tc_prepare() {
  const void* fn[4] = {(const void*)tc_gemm_kernel<kTcBN>, (const void*)tc_gemm_kernel<kTcBNNarrow>,
                       (const void*)tc_gemm_planes_kernel<kTcBN>,
                       (const void*)tc_gemm_planes_kernel<kTcBNNarrow>};
  const size_t bytes[4] = {TcTile<kTcBN>::kSmem, TcTile<kTcBNNarrow>::kSmem,
                           PlaneTile<kTcBN>::kSmem, PlaneTile<kTcBNNarrow>::kSmem};
  for (int i = 0; i < 4; ++i) {
    cudaError_t e = cudaFuncSetAttribute(fn[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes[i]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Either tile runs one CTA per SM (two stages of 72 or 96 KB).  The wide
// tile splits each operand once per 128 x 128 outputs instead of 128 x 64; it
// is taken when its tiles fill every SM at least once, else the narrow tile,
// which has twice as many.
cudaError_t tc_gemm(const TcProblem* d_probs, int nprob, int max_m, int max_n, int* status,
                    cudaStream_t s) {
  if (nprob <= 0 || max_m <= 0 || max_n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long wide_tiles = (long long)nprob * cdiv(max_m, kTcBM) * cdiv(max_n, kTcBN);
  if (wide_tiles >= sms) {
    dim3 grid(cdiv(max_n, kTcBN), cdiv(max_m, kTcBM), nprob);
    tc_gemm_kernel<kTcBN><<<grid, kThreads, TcTile<kTcBN>::kSmem, s>>>(d_probs, status);
  } else {
    dim3 grid(cdiv(max_n, kTcBNNarrow), cdiv(max_m, kTcBM), nprob);
    tc_gemm_kernel<kTcBNNarrow><<<grid, kThreads, TcTile<kTcBNNarrow>::kSmem, s>>>(d_probs,
                                                                                status);
  }
  return cudaGetLastError();
}

size_t tc_plane_bytes(int rows, int K) {
  return (size_t)cdiv(rows, kTcBM) * (size_t)(K / kTcBK) * kPlaneTileBytes;
}

TcSplitJob tc_split_job_a(const TcProblem& p, unsigned char* a) {
  TcSplitJob j{};
  j.X = p.A;
  j.ld = p.lda;
  j.km = p.a_km;
  j.rows = p.M;
  j.K = p.K;
  j.tri = p.k_to_m ? 1 : 0;
  j.planes = a;
  return j;
}

TcSplitJob tc_split_job_b(const TcProblem& p, unsigned char* b) {
  TcSplitJob j{};
  j.X = p.B;
  j.ld = p.ldb;
  j.km = p.b_kn;   // op(B)^T[n][k] = B[n*ldb + k] (b_kn = 0) or B[k*ldb + n]
  j.rows = p.N;
  j.K = p.K;
  j.tri = p.k_from_n ? 2 : 0;
  j.planes = b;
  return j;
}

cudaError_t tc_split(const TcSplitJob* d_jobs, int njobs, int max_tiles, cudaStream_t s) {
  if (njobs <= 0 || max_tiles <= 0) return cudaSuccess;
  tc_split_kernel<<<dim3(max_tiles, njobs), kThreads, 0, s>>>(d_jobs);
  return cudaGetLastError();
}

cudaError_t tc_gemm_planes(const TcProblem* d_probs, int nprob, int max_m, int max_n,
                           int* status, cudaStream_t s) {
  if (nprob <= 0 || max_m <= 0 || max_n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long wide_tiles = (long long)nprob * cdiv(max_m, kTcBM) * cdiv(max_n, kTcBN);
  if (wide_tiles >= sms) {
    dim3 grid(cdiv(max_n, kTcBN), cdiv(max_m, kTcBM), nprob);
    tc_gemm_planes_kernel<kTcBN>
        <<<grid, kPlaneThreads, PlaneTile<kTcBN>::kSmem, s>>>(d_probs, status);
  } else {
    dim3 grid(cdiv(max_n, kTcBNNarrow), cdiv(max_m, kTcBM), nprob);
    tc_gemm_planes_kernel<kTcBNNarrow>
        <<<grid, kPlaneThreads, PlaneTile<kTcBNNarrow>::kSmem, s>>>(d_probs, status);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Triangular inverse
// ----------------------------------------------------------------------------
namespace {
struct Split {
  int a, m, b;
};
void collect_splits(int a, int b, int depth, std::vector<std::vector<Split>>& lv) {
  if (b - a <= 1) return;
  const int m = (a + b) / 2;
  if ((int)lv.size() <= depth) lv.resize(depth + 1);
  lv[depth].push_back({a, m, b});
  collect_splits(a, m, depth + 1, lv);
  collect_splits(m, b, depth + 1, lv);
}
}  // namespace

cudaError_t tri_inverse_plan(TriInvPlan* plan, int P, const float* L, const float* W, float* X) {
  (void)W;
  *plan = TriInvPlan{};
  if (P % 64) return cudaErrorInvalidValue;
  plan->P = P;
  plan->T = P / 64;
  std::vector<std::vector<Split>> lv;
  collect_splits(0, plan->T, 0, lv);
  // deepest level first: a split needs both halves inverted
  std::vector<TcProblem> probs;
  for (int d = (int)lv.size() - 1; d >= 0; --d) {
    const int first = (int)probs.size();
    int mm = 0, mn = 0;
    // product 1 of every split of this depth, then product 2
    for (const Split& sp : lv[d]) {
      const int r0 = sp.m * 64, c0 = sp.a * 64;
      const int M = (sp.b - sp.m) * 64, N = (sp.m - sp.a) * 64;
      TcProblem t1{};   // T1 = L21 X11 (rows m..b, cols a..m), stored transposed at (c0, r0)
      t1.A = L + (size_t)r0 * P + c0;
      t1.lda = P;
      t1.a_km = 0;
      t1.B = X + (size_t)c0 * P + c0;   // X11[k][n]
      t1.ldb = P;
      t1.b_kn = 1;
      t1.C = X + (size_t)c0 * P + r0;   // T1^T in the upper triangle
      t1.ldc = P;
      t1.c_nm = 1;
      t1.M = M;
      t1.N = N;
      t1.K = N;
      t1.k_from_n = 1;                   // X11 is lower triangular
      t1.alpha = 1.f;
      t1.beta = 0.f;
      probs.push_back(t1);
      mm = std::max(mm, M);
      mn = std::max(mn, N);
    }
    plan->level_first.push_back(first);
    plan->level_max_m.push_back(mm);
    plan->level_max_n.push_back(mn);
    const int second = (int)probs.size();
    for (const Split& sp : lv[d]) {
      const int r0 = sp.m * 64, c0 = sp.a * 64;
      const int M = (sp.b - sp.m) * 64, N = (sp.m - sp.a) * 64;
      TcProblem t2{};   // X21 = -X22 T1
      t2.A = X + (size_t)r0 * P + r0;   // X22[m][k]
      t2.lda = P;
      t2.a_km = 0;
      t2.B = X + (size_t)c0 * P + r0;   // T1^T[n][k]
      t2.ldb = P;
      t2.b_kn = 0;
      t2.C = X + (size_t)r0 * P + c0;
      t2.ldc = P;
      t2.c_nm = 0;
      t2.M = M;
      t2.N = N;
      t2.K = M;
      t2.k_to_m = 1;                     // X22 is lower triangular
      t2.alpha = -1.f;
      t2.beta = 0.f;
      probs.push_back(t2);
    }
    plan->level_first.push_back(second);
    plan->level_max_m.push_back(mm);
    plan->level_max_n.push_back(mn);
  }
  plan->level_first.push_back((int)probs.size());
  plan->nprob = (int)probs.size();
  if (probs.empty()) return cudaSuccess;
  // plane offsets: each launch's operands from the start of the scratch
  std::vector<TcSplitJob> jobs;
  std::vector<std::pair<size_t, size_t>> offs(probs.size());
  size_t scratch = 0;
  for (size_t l = 0; l + 1 < plan->level_first.size(); ++l) {
    plan->job_first.push_back((int)jobs.size());
    int max_tiles = 0;
    size_t at = 0;
    for (int i = plan->level_first[l]; i < plan->level_first[l + 1]; ++i) {
      const TcProblem& q = probs[i];
      offs[i].first = at;
      at += tc_plane_bytes(q.M, q.K);
      offs[i].second = at;
      at += tc_plane_bytes(q.N, q.K);
      max_tiles = std::max(max_tiles, std::max(cdiv(q.M, kTcBM), cdiv(q.N, kTcBM)) * (q.K / kTcBK));
      jobs.push_back(tc_split_job_a(q, nullptr));
      jobs.push_back(tc_split_job_b(q, nullptr));
    }
    plan->job_max_tiles.push_back(max_tiles);
    scratch = std::max(scratch, at);
  }
  plan->job_first.push_back((int)jobs.size());
  cudaError_t e = cudaMalloc(&plan->d_planes, scratch);
  if (e != cudaSuccess) return e;
  for (size_t i = 0; i < probs.size(); ++i) {
    probs[i].a_planes = plan->d_planes + offs[i].first;
    probs[i].b_planes = plan->d_planes + offs[i].second;
    jobs[2 * i].planes = plan->d_planes + offs[i].first;
    jobs[2 * i + 1].planes = plan->d_planes + offs[i].second;
  }
  e = cudaMalloc(&plan->d_jobs, jobs.size() * sizeof(TcSplitJob));
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->d_jobs, jobs.data(), jobs.size() * sizeof(TcSplitJob),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_probs, probs.size() * sizeof(TcProblem));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(plan->d_probs, probs.data(), probs.size() * sizeof(TcProblem),
                    cudaMemcpyHostToDevice);
}

void tri_inverse_plan_destroy(TriInvPlan* plan) {
  if (plan->d_probs) cudaFree(plan->d_probs);
  if (plan->d_jobs) cudaFree(plan->d_jobs);
  if (plan->d_planes) cudaFree(plan->d_planes);
  *plan = TriInvPlan{};
}

cudaError_t tri_inverse(const TriInvPlan& plan, const float* W, float* X, int* status,
                        cudaStream_t s) {
  trinv_diag_kernel<<<plan.T, 256, 0, s>>>(W, X, plan.P, plan.T);
  cudaError_t e = cudaGetLastError();
  // each entry of level_first opens one batched launch (product 1, product 2, ...),
  // its operands split into planes just before it
  for (size_t l = 0; e == cudaSuccess && l + 1 < plan.level_first.size(); ++l) {
    const int f = plan.level_first[l], n = plan.level_first[l + 1] - f;
    const int jf = plan.job_first[l], jn = plan.job_first[l + 1] - jf;
    e = tc_split(plan.d_jobs + jf, jn, plan.job_max_tiles[l], s);
    if (e == cudaSuccess)
      e = tc_gemm_planes(plan.d_probs + f, n, plan.level_max_m[l], plan.level_max_n[l], status, s);
  }
  if (e != cudaSuccess) return e;
  const int tb = plan.P / 32;
  trinv_mirror_kernel<<<dim3(tb, tb), dim3(32, 8), 0, s>>>(X, plan.P);
  return cudaGetLastError();
}

cudaError_t tc_chol_plan(TcCholPlan* plan, int P, float* L, const float* winv) {
  *plan = TcCholPlan{};
  if (P % 64) return cudaErrorInvalidValue;
  plan->P = P;
  plan->T = P / 64;
  std::vector<TcProblem> probs;
  for (int j = 0; j + 1 < plan->T; ++j) {
    const int r0 = (j + 1) * 64, c0 = j * 64, M = P - r0;
    TcProblem t{};   // L_ij = A_ij W_j^T, rows r0.. of panel column j, in place
    t.A = L + (size_t)r0 * P + c0;
    t.lda = P;
    t.B = winv + (size_t)j * 64 * 64;   // op(B)[k][n] = W_j[n][k]
    t.ldb = 64;
    t.C = L + (size_t)r0 * P + c0;      // one CTA owns all 64 columns of its rows
    t.ldc = P;
    t.M = M;
    t.N = 64;
    t.K = 64;
    t.alpha = 1.f;
    probs.push_back(t);
    TcProblem u{};   // A_trail -= L_p L_p^T on the lower tiles
    u.A = L + (size_t)r0 * P + c0;
    u.lda = P;
    u.B = L + (size_t)r0 * P + c0;      // op(B)[k][n] = L_p[n][k]
    u.ldb = P;
    u.C = L + (size_t)r0 * P + r0;
    u.ldc = P;
    u.M = M;
    u.N = M;
    u.K = 64;
    u.alpha = -1.f;
    u.beta = 1.f;
    u.c_lower = 1;
    probs.push_back(u);
  }
  if (probs.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(&plan->d_probs, probs.size() * sizeof(TcProblem));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(plan->d_probs, probs.data(), probs.size() * sizeof(TcProblem),
                    cudaMemcpyHostToDevice);
}

void tc_chol_plan_destroy(TcCholPlan* plan) {
  if (plan->d_probs) cudaFree(plan->d_probs);
  *plan = TcCholPlan{};
}

cudaError_t tc_cholesky(const TcCholPlan& plan, float* L, float* winv, int* status,
                        cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < plan.T && e == cudaSuccess; ++j) {
    e = chol_potrf_tile(L, plan.P, j, winv, status, s);
    if (e != cudaSuccess || j + 1 == plan.T) break;
    const int M = plan.P - (j + 1) * 64;
    e = tc_gemm(plan.d_probs + 2 * j, 1, M, 64, status, s);
    if (e == cudaSuccess) e = tc_gemm(plan.d_probs + 2 * j + 1, 1, M, M, status, s);
  }
  return e;
}

cudaError_t trinv_lower(const float* X, int P, int p, int lo, const double* v, double* y,
                        cudaStream_t s) {
  const int rows = p - lo;
  if (rows <= 0) return cudaSuccess;
  if (p > kTrMaxP) return cudaErrorInvalidValue;
  trinv_lower_kernel<<<cdiv(rows, kTrRows), kThreads, (size_t)(p + 8) * sizeof(float), s>>>(
      X, P, p, lo, v, y);
  return cudaGetLastError();
}

cudaError_t trinv_upper(const float* X, int P, int p, int lo, const double* y, double* z,
                        int accumulate, cudaStream_t s) {
  if (p > kTrMaxP) return cudaErrorInvalidValue;
  trinv_upper_kernel<<<cdiv(p, kTrRows), kThreads, (size_t)(p + 8) * sizeof(float), s>>>(
      X, P, p, lo, y, z, accumulate);
  return cudaGetLastError();
}

size_t iterate_tc_smem(int P) { return (size_t)P * (sizeof(double) + sizeof(int)) + 64; }

template <typename T>
cudaError_t iterate_tc_prepare(int P, int num_sms, int* grid) {
  const size_t smem = iterate_tc_smem(P);
  cudaError_t e = cudaFuncSetAttribute(iterate_tc_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iterate_tc_kernel<T>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = std::min(kIterTcCtas, per_sm * num_sms);
  return cudaSuccess;
}

template <typename T>
cudaError_t iterate_tc(const LaArgs<T>& a, const StepInfo* info, const int* ext, const float* X,
                       double* y, double* res, unsigned* bar, int refine, int grid,
                       cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  LaArgs<T> args = a;
  IterTc it{info, ext, X, y, res, bar, refine};
  void* params[] = {&args, &it};
  return cudaLaunchCooperativeKernel((const void*)iterate_tc_kernel<T>, dim3(grid),
                                     dim3(kThreads), params, iterate_tc_smem(a.P), s);
}

template cudaError_t iterate_tc_prepare<float>(int, int, int*);
template cudaError_t iterate_tc_prepare<double>(int, int, int*);
template cudaError_t iterate_tc<float>(const LaArgs<float>&, const StepInfo*, const int*,
                                       const float*, double*, double*, unsigned*, int, int,
                                       cudaStream_t);
template cudaError_t iterate_tc<double>(const LaArgs<double>&, const StepInfo*, const int*,
                                        const float*, double*, double*, unsigned*, int, int,
                                        cudaStream_t);

// ----------------------------------------------------------------------------
// C ABI: the product and the inverse factor on their own
// ----------------------------------------------------------------------------
namespace {
__global__ void tc_form_f32_kernel(const double* G, int p, double lam, float* L, int P) {
  const long long total = (long long)P * P;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / P), j = (int)(idx % P);
    double v = 0.0;
    if (i < p && j < p) v = G[(size_t)i * p + j] + (i == j ? lam : 0.0);
    else if (i == j) v = 1.0;
    L[idx] = (float)v;
  }
}
__global__ void tc_copy_out_kernel(const float* X, int P, int p, float* out) {
  const long long total = (long long)p * p;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x)
    out[idx] = X[(size_t)(idx / p) * P + idx % p];
}
slim_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SLIM_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SLIM_ENOMEM : SLIM_ECUDA;
}
}  // namespace
}  // namespace slim

using namespace slim;

namespace {
// The product's work space comes from a stream-ordered pool of the library's
// own, one per device, whose release threshold is the maximum: memory freed
// at the end of a call stays mapped for the next one instead of going back to
// the driver at each synchronisation.
cudaError_t workspace_pool(cudaMemPool_t* pool) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) {
    *pool = it->second;
    return cudaSuccess;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t p = nullptr;
  e = cudaMemPoolCreate(&p, &props);
  if (e != cudaSuccess) return e;
  uint64_t keep = UINT64_MAX;
  e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e != cudaSuccess) {
    cudaMemPoolDestroy(p);
    return e;
  }
  pools[dev] = p;
  *pool = p;
  return cudaSuccess;
}
}  // namespace

extern "C" slim_status slim_tc_matmul(int M, int N, int K, const float* A, long long lda,
                                      int a_km, const float* B, long long ldb, int b_kn, float* C,
                                      long long ldc, int c_nm, float alpha, float beta,
                                      int a_lower, int b_lower, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 64 || K % 64 || lda < 1 || ldb < 1 || ldc < 1)
    return SLIM_EINVAL;
  if ((a_km | b_kn | c_nm | a_lower | b_lower) & ~1) return SLIM_EINVAL;
  // float4 loads of K-contiguous rows need 16-byte rows
  if ((!a_km && (lda % 4 || reinterpret_cast<uintptr_t>(A) % 16)) ||
      (!b_kn && (ldb % 4 || reinterpret_cast<uintptr_t>(B) % 16)))
    return SLIM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TcProblem pb{};
  pb.A = A; pb.lda = lda; pb.a_km = a_km;
  pb.B = B; pb.ldb = ldb; pb.b_kn = b_kn;
  pb.C = C; pb.ldc = ldc; pb.c_nm = c_nm;
  pb.M = M; pb.N = N; pb.K = K;
  pb.k_to_m = a_lower; pb.k_from_n = b_lower;
  pb.alpha = alpha; pb.beta = beta;
  // one allocation from the library's stream-ordered pool: the problem, the
  // status word, the split jobs and both operands' planes
  static_assert(sizeof(TcProblem) <= 256 && 2 * sizeof(TcSplitJob) <= 512, "workspace layout");
  const size_t a_bytes = tc_plane_bytes(M, K), b_bytes = tc_plane_bytes(N, K);
  const size_t o_st = 256, o_jobs = 512, o_a = 1024, o_b = o_a + a_bytes;
  unsigned char* ws = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = tc_prepare();
  if (e == cudaSuccess) e = workspace_pool(&pool);
  if (e == cudaSuccess)
    e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ws), o_b + b_bytes, pool, s);
  if (e != cudaSuccess) return from_cuda(e);
  pb.a_planes = ws + o_a;
  pb.b_planes = ws + o_b;
  const TcSplitJob jobs[2] = {tc_split_job_a(pb, ws + o_a), tc_split_job_b(pb, ws + o_b)};
  TcProblem* d_pb = reinterpret_cast<TcProblem*>(ws);
  int* d_st = reinterpret_cast<int*>(ws + o_st);
  TcSplitJob* d_jobs = reinterpret_cast<TcSplitJob*>(ws + o_jobs);
  e = cudaMemcpyAsync(d_pb, &pb, sizeof(pb), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_jobs, jobs, sizeof(jobs), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_st, 0, sizeof(int), s);
  const int max_tiles = cdiv(std::max(M, N), kTcBM) * (K / kTcBK);
  if (e == cudaSuccess) e = tc_split(d_jobs, 2, max_tiles, s);
  if (e == cudaSuccess) e = tc_gemm_planes(d_pb, 1, M, N, d_st, s);
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, d_st, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t ef = cudaFreeAsync(ws, s);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  slim_status st = from_cuda(e);
  return st != SLIM_OK ? st : (hs ? (slim_status)hs : SLIM_OK);
}

extern "C" slim_status slim_chol_inverse(const double* G, int p, double lambda, float* X,
                                         void* stream) {
  if (!G || !X || p < 1 || p > 16384 || !(lambda >= 0.0)) return SLIM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = (p + 63) / 64 * 64;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return from_cuda(cudaErrorUnknown);
  CholPlan plan;
  TriInvPlan tp;
  float *L = nullptr, *Xf = nullptr;
  int* d_st = nullptr;
  cudaError_t e = chol_plan_create(&plan, P, 64, 1, sms);
  if (e == cudaSuccess) e = cudaMalloc(&L, (size_t)P * P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&Xf, (size_t)P * P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_st, sizeof(int));
  if (e == cudaSuccess) e = tc_prepare();
  if (e == cudaSuccess) e = tri_inverse_plan(&tp, P, L, (const float*)plan.d_winv, Xf);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_st, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    const long long total = (long long)P * P;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    tc_form_f32_kernel<<<grid, 256, 0, s>>>(G, p, lambda, L, P);
    e = cudaGetLastError();
  }
  TcCholPlan cp;
  if (e == cudaSuccess) e = chol_potrf_tile_prepare();
  if (e == cudaSuccess) e = tc_chol_plan(&cp, P, L, (const float*)plan.d_winv);
  if (e == cudaSuccess) e = tc_cholesky(cp, L, (float*)plan.d_winv, d_st, s);
  if (e == cudaSuccess) e = tri_inverse(tp, (const float*)plan.d_winv, Xf, d_st, s);
  if (e == cudaSuccess) {
    const long long total = (long long)p * p;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    tc_copy_out_kernel<<<grid, 256, 0, s>>>(Xf, P, p, X);
    e = cudaGetLastError();
  }
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, d_st, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  slim_status st = from_cuda(e);
  tri_inverse_plan_destroy(&tp);
  tc_chol_plan_destroy(&cp);
  chol_plan_destroy(&plan);
  cudaFree(L);
  cudaFree(Xf);
  cudaFree(d_st);
  return st != SLIM_OK ? st : (hs ? (slim_status)hs : SLIM_OK);
}
