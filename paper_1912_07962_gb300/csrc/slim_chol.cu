// Tiled Cholesky factorisation and triangular solves of K = lambda_k I + G.
//
// One persistent launch factors K: CTAs claim tasks of the right-looking tiled
// algorithm (POTRF of a diagonal tile, TRSM of a panel tile, a GEMM update of
// a trailing tile) through an atomic ticket, in an order where every task
// depends only on earlier ones, and wait for their inputs on per-tile counters.
// Tile counter (i,k) counts the updates applied to tile (i,k) plus one when the
// tile is final, so "tile (i,k) final" is counter == k+1.  A claimed task is
// always runnable once the tasks claimed before it finish, so progress never
// depends on which CTAs the hardware schedules; every wait is still bounded
// and gives up with SLIM_ETIMEOUT (and tells the other CTAs to stop).
//
// The solves chain diagonal blocks the same way: CTA i of the forward solve
// subtracts L_ij y_j as each y_j is published, then applies L_ii^{-1}; the
// backward solve runs the transposed chain from the last block.
#include <algorithm>
#include <type_traits>

#include <cooperative_groups.h>

#include "slim_chol.cuh"
#include "slim_device.cuh"

namespace slim {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kSpinLimit = 1u << 22;   // ~seconds of polling before giving up

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// CTA-wide bounded wait until f[q] >= t[q] for q < nf (nf <= 3), the flags
// polled in parallel by threads 0..nf-1.  Returns false if a wait ran out or
// another CTA asked everyone to stop.
__device__ bool cta_wait(const int* f0, int t0, const int* f1, int t1, const int* f2, int t2,
                         int nf, int* abort_flag, int* status, int* s_ok3) {
  const int tid = threadIdx.x;
  if (tid < 3) {
    int ok = 1;
    if (tid < nf) {
      const int* f = tid == 0 ? f0 : (tid == 1 ? f1 : f2);
      const int tg = tid == 0 ? t0 : (tid == 1 ? t1 : t2);
      unsigned it = 0;
      while (ld_acquire(f) < tg) {
        if (ld_acquire(abort_flag)) { ok = 0; break; }
        if (++it > kSpinLimit) {
          set_status(status, SLIM_ETIMEOUT);
          atomicExch(abort_flag, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
      __threadfence();
    }
    s_ok3[tid] = ok;
  }
  __syncthreads();
  const int ok = s_ok3[0] & s_ok3[1] & s_ok3[2];
  __syncthreads();
  return ok != 0;
}

__device__ bool cta_wait(const int* flag, int target, int* abort_flag, int* status, int* s_ok3) {
  return cta_wait(flag, target, flag, 0, flag, 0, 1, abort_flag, status, s_ok3);
}

__device__ __forceinline__ void cta_publish(int* flag, int add = 1) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add(flag, add);
  }
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <typename T>
__device__ __forceinline__ void stcg(T* p, T v) { __stcg(p, v); }

// Load TM consecutive values from (16-byte aligned) shared memory.
template <typename T, int TM>
__device__ __forceinline__ void lds_vec(T (&v)[TM], const T* p) {
  if constexpr (sizeof(T) == 4 && TM == 4) {
    float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (sizeof(T) == 8 && TM == 2) {
    double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int a = 0; a < TM; ++a) v[a] = p[a];
  }
}

__host__ __device__ constexpr int gemm_ld(int nb) { return nb + 4; }   // padded row of a staged tile
constexpr int kPanelLd = 20;   // 16 panel columns + pad, 16-byte rows

// A factorisation CTA holds three NB x gemm_ld(NB) tiles in shared memory:
//   As, Bs  GEMM operands staged transposed (k-major)
//   S       a tile staged as is: the GEMM's C operand, or the diagonal tile
// The diagonal factorisation reuses Bs for the inverse and As for the
// factored panel and the partial sums of the inverse.
// The float32 factor with 64 x 64 tiles also runs grouped updates, whose
// operands are two 64 x (128 + 4) tiles staged transposed.
template <typename T>
__host__ __device__ constexpr size_t factor_smem_bytes(int nb) {
  return (sizeof(T) == 4 && nb == 64)
             ? (size_t)2 * nb * (2 * nb + 4) * sizeof(T) > (size_t)3 * nb * gemm_ld(nb) * sizeof(T)
                   ? (size_t)2 * nb * (2 * nb + 4) * sizeof(T)
                   : (size_t)3 * nb * gemm_ld(nb) * sizeof(T)
             : (size_t)3 * nb * gemm_ld(nb) * sizeof(T);
}

template <typename T>
using vec16_t = typename std::conditional<sizeof(T) == 4, float4, double2>::type;

// One NB x NB tile (row-major, leading dimension ld) in registers, in EV x EV
// blocks (EV values per 16 bytes): block b covers rows (b / (NB/EV))*EV..,
// columns (b % (NB/EV))*EV..; a row's blocks are read by consecutive threads.
template <typename T, int NB>
struct TileRegs {
  using V = vec16_t<T>;
  static constexpr int EV = 16 / sizeof(T);
  static constexpr int QB = NB / EV;                            // blocks per row
  static constexpr int NBLKS = QB * QB;
  static constexpr int BPT = (NBLKS + kThreads - 1) / kThreads;  // blocks per thread
  V v[BPT][EV];
  __device__ void load(const T* A, int ld) {
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
      const int b = threadIdx.x + t * kThreads;
      if (b < NBLKS) {
        const int rq = b / QB, qq = b % QB;
#pragma unroll
        for (int e = 0; e < EV; ++e)
          v[t][e] = __ldcg(reinterpret_cast<const V*>(A + (size_t)(rq * EV + e) * ld + qq * EV));
      }
    }
  }
  // As[q][r] = A[r][q]: each EV x EV block transposed in registers
  __device__ void store_t(T* As) const {
    constexpr int LD = gemm_ld(NB);
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
      const int b = threadIdx.x + t * kThreads;
      if (b < NBLKS) {
        const int rq = b / QB, qq = b % QB;
#pragma unroll
        for (int e = 0; e < EV; ++e) {
          V o;
          T* po = reinterpret_cast<T*>(&o);
#pragma unroll
          for (int f = 0; f < EV; ++f) po[f] = reinterpret_cast<const T*>(&v[t][f])[e];
          *reinterpret_cast<V*>(As + (size_t)(qq * EV + e) * LD + rq * EV) = o;
        }
      }
    }
  }
  // As[q][col0 + r] = A[r][q] with row length ld (a tile of a wider operand)
  __device__ void store_t_ld(T* As, int ld, int col0) const {
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
      const int b = threadIdx.x + t * kThreads;
      if (b < NBLKS) {
        const int rq = b / QB, qq = b % QB;
#pragma unroll
        for (int e = 0; e < EV; ++e) {
          V o;
          T* po = reinterpret_cast<T*>(&o);
#pragma unroll
          for (int f = 0; f < EV; ++f) po[f] = reinterpret_cast<const T*>(&v[t][f])[e];
          *reinterpret_cast<V*>(As + (size_t)(qq * EV + e) * ld + col0 + rq * EV) = o;
        }
      }
    }
  }
  __device__ void store_n(T* S) const {
    constexpr int LD = gemm_ld(NB);
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
      const int b = threadIdx.x + t * kThreads;
      if (b < NBLKS) {
        const int rq = b / QB, qq = b % QB;
#pragma unroll
        for (int e = 0; e < EV; ++e)
          *reinterpret_cast<V*>(S + (size_t)(rq * EV + e) * LD + qq * EV) = v[t][e];
      }
    }
  }
};

// Stage A and B transposed into As, Bs and (if C) C as is into S, then
// barrier.  With one block per thread all loads are in flight together;
// larger tiles are staged one after another to bound the registers.
template <typename T, int NB>
__device__ void stage_tiles(const T* A, int lda, const T* B, int ldb, const T* C, int ldc, T* As,
                            T* Bs, T* S) {
  if constexpr (TileRegs<T, NB>::BPT == 1) {
    TileRegs<T, NB> ra, rb, rc;
    ra.load(A, lda);
    rb.load(B, ldb);
    if (C) rc.load(C, ldc);
    ra.store_t(As);
    rb.store_t(Bs);
    if (C) rc.store_n(S);
  } else {
    TileRegs<T, NB> rt;
    rt.load(A, lda);
    rt.store_t(As);
    rt.load(B, ldb);
    rt.store_t(Bs);
    if (C) {
      rt.load(C, ldc);
      rt.store_n(S);
    }
  }
  __syncthreads();
}

// acc = (A B^T) for the thread's TM x TM block: thread (ty,tx) owns rows
// ty*TM.., columns tx*TM..; each k step reads two contiguous vectors.
template <typename T, int NB>
__device__ __forceinline__ void gemm_core(const T* As, const T* Bs, T (&acc)[NB / 16][NB / 16]) {
  constexpr int LD = gemm_ld(NB);
  constexpr int TM = NB / 16;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
#pragma unroll 8
  for (int q = 0; q < NB; ++q) {
    T av[TM], bv[TM];
    lds_vec<T, TM>(av, As + q * LD + ty * TM);
    lds_vec<T, TM>(bv, Bs + q * LD + tx * TM);
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] += av[a] * bv[b];
  }
}

// 16-byte streaming store of EV values.
template <typename T>
__device__ __forceinline__ void st_vec16(T* p, const T (&v)[16 / sizeof(T)]) {
  if constexpr (sizeof(T) == 4)
    __stcg(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  else
    __stcg(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
}

// Store a thread's TM values of row r (columns tx*TM..) to global memory.
template <typename T, int TM>
__device__ __forceinline__ void st_row(T* p, const T (&v)[TM]) {
  if constexpr (TM * sizeof(T) == 16) {
    st_vec16<T>(p, v);
  } else {
#pragma unroll
    for (int b = 0; b < TM; ++b) stcg(p + b, v[b]);
  }
}

// out = sign * A B^T (+ C if C): the TRSM (B = inverse diagonal tile) and the
// trailing update (C = the tile itself, sign -1) of the tiled algorithm.
template <typename T, int NB>
__device__ __noinline__ void task_gemm(T* out, int ldo, const T* A, int lda, const T* B, int ldb, const T* C,
                          T sign, T* As, T* Bs, T* S) {
  constexpr int LD = gemm_ld(NB);
  constexpr int TM = NB / 16;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  stage_tiles<T, NB>(A, lda, B, ldb, C, ldo, As, Bs, S);
  T acc[TM][TM];
  gemm_core<T, NB>(As, Bs, acc);
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int r = ty * TM + a;
    T o[TM];
#pragma unroll
    for (int b = 0; b < TM; ++b) o[b] = sign * acc[a][b] + (C ? S[r * LD + tx * TM + b] : T(0));
    st_row<T, TM>(out + (size_t)r * ldo + tx * TM, o);
  }
  __syncthreads();
}

// C -= A B^T for a 2x2 group of 64 x 64 tiles (float32): C is the 128 x 128
// block at the group's top-left tile, A and B the 128 x 64 blocks of column
// k at rows i and m (leading dimension P).  Thread (ty, tx) owns rows ty*8..,
// columns tx*8..; the products are summed from zero and subtracted from C
// once, as in the single-tile update (C is large next to the Schur complement
// it leaves, so it must not take the rounding of every product).  Like every
// tile read of the factorisation, C is read around L1 (tiles change under
// other SMs).
template <int NB>
__device__ __noinline__ void task_gemm_group(float* C, int P, const float* A, const float* B,
                                             float* As, float* Bs) {
  constexpr int LD2 = 2 * NB + 4;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  {
    TileRegs<float, NB> r0, r1;
    r0.load(A, P);
    r1.load(A + (size_t)NB * P, P);
    r0.store_t_ld(As, LD2, 0);
    r1.store_t_ld(As, LD2, NB);
    r0.load(B, P);
    r1.load(B + (size_t)NB * P, P);
    r0.store_t_ld(Bs, LD2, 0);
    r1.store_t_ld(Bs, LD2, NB);
  }
  __syncthreads();
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 4
  for (int q = 0; q < NB; ++q) {
    const float4 a0 = *reinterpret_cast<const float4*>(As + q * LD2 + ty * 8);
    const float4 a1 = *reinterpret_cast<const float4*>(As + q * LD2 + ty * 8 + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(Bs + q * LD2 + tx * 8);
    const float4 b1 = *reinterpret_cast<const float4*>(Bs + q * LD2 + tx * 8 + 4);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    float* row = C + (size_t)(ty * 8 + a) * P + tx * 8;
    float4 c0 = __ldcg(reinterpret_cast<const float4*>(row));
    float4 c1 = __ldcg(reinterpret_cast<const float4*>(row + 4));
    c0.x -= acc[a][0]; c0.y -= acc[a][1]; c0.z -= acc[a][2]; c0.w -= acc[a][3];
    c1.x -= acc[a][4]; c1.y -= acc[a][5]; c1.z -= acc[a][6]; c1.w -= acc[a][7];
    __stcg(reinterpret_cast<float4*>(row), c0);
    __stcg(reinterpret_cast<float4*>(row + 4), c1);
  }
  __syncthreads();
}

// CTA-wide bounded wait for the 8 counters of a grouped update of tiles
// (i..i+1, m..m+1) at step k: the four operand tiles of column k final
// (counter k+1), the four output tiles with the k earlier updates applied.
__device__ bool cta_wait_group(const int* cnt, int Tt, int i, int m, int k, int* abort_flag,
                               int* status, int* s_ok8) {
  const int tid = threadIdx.x;
  if (tid < 8) {
    const int q = tid & 3;
    const int* f;
    int tg;
    if (tid < 4) {
      const int row = q == 0 ? i : q == 1 ? i + 1 : q == 2 ? m : m + 1;
      f = cnt + row * Tt + k;
      tg = k + 1;
    } else {
      f = cnt + (i + (q >> 1)) * Tt + m + (q & 1);
      tg = k;
    }
    int ok = 1;
    unsigned it = 0;
    while (ld_acquire(f) < tg) {
      if (ld_acquire(abort_flag)) { ok = 0; break; }
      if (++it > kSpinLimit) {
        set_status(status, SLIM_ETIMEOUT);
        atomicExch(abort_flag, 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_ok8[tid] = ok;
  }
  __syncthreads();
  int ok = 1;
#pragma unroll
  for (int q = 0; q < 8; ++q) ok &= s_ok8[q];
  __syncthreads();
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ void pivot(T d, T& s, T& rs, int* status) {
  if (!(d > T(0))) {
    set_status(status, SLIM_ENOTPD);
    d = T(1);
  }
  if constexpr (sizeof(T) == 4) {
    // hardware reciprocal square root (a few ulp): the float32 factor only
    // preconditions the float64-residual refinement
    rs = rsqrtf(d);
    s = d * rs;
  } else {
    rs = rsqrt_pivot(d, status);
    s = d * rs;
  }
}

// One warp: factor the 16 x 16 block D (lower triangle, leading dimension
// ld) in place and write its inverse X (lower, zeros above).  Lane l holds
// row l in registers; step c broadcasts the pivot and column c by shuffles
// (right-looking: a_lj -= l_lc l_jc for c < j <= l).  Then lane l forms
// column l of the inverse by forward substitution,
//   X_il = -(sum_{q=l}^{i-1} L_iq X_ql) / L_ii,  X_ll = 1 / L_ll.
// Lanes 16..31 mirror lanes 0..15.
template <typename T>
__device__ __noinline__ void diag_block(T* D, int ld, T* X, int ldx, int* status) {
  const int lane = threadIdx.x & 31, l = lane & 15;
  T a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = (j <= l) ? D[l * ld + j] : T(0);
  T my_rs = T(0);   // 1 / L_ll
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const T d = __shfl_sync(0xffffffffu, a[c], c);
    T s, rs;
    pivot(d, s, rs, status);
    if (l == c) my_rs = rs;
    const T lc = (l > c) ? a[c] * rs : T(0);
    a[c] = (l == c) ? s : lc;
#pragma unroll
    for (int j = c + 1; j < 16; ++j) {
      const T bj = __shfl_sync(0xffffffffu, lc, j);
      if (l >= j) a[j] -= lc * bj;
    }
  }
  if (lane < 16) {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j <= l) D[l * ld + j] = a[j];
  }
  __syncwarp();
  // rows of L are read back from shared memory (one broadcast load each)
  T x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const T rs_i = __shfl_sync(0xffffffffu, my_rs, i);
    T sum = T(0);
#pragma unroll
    for (int q = 0; q < i; ++q) sum += D[i * ld + q] * x[q];
    x[i] = (i == l) ? rs_i : (i > l ? -sum * rs_i : T(0));
  }
  if (lane < 16) {
#pragma unroll
    for (int i = 0; i < 16; ++i) X[i * ldx + l] = x[i];
  }
  __syncwarp();
}

// Float64 tile factorisation: factor the NB x NB tile In (lower triangle,
// leading dimension ld_in; read once at the start) into Lkk and write its
// inverse (lower, zeros above) to W.  Non-positive pivots set SLIM_ENOTPD
// and are replaced by 1 so the factorisation still completes without NaNs.
//
// Right-looking elimination on the unscaled Schur complements,
//   S[i][q] -= (S[i][c] / d_c) S[q][c]   for c < q <= i,
// with the tile in registers (thread (ty,tx) owns rows ty+16u, columns
// tx+16v) and column c broadcast through a double-buffered shared column: one
// barrier per column.  The column's owners publish it as soon as it is final.
// float: every thread forms 1/d_c itself (correctly rounded reciprocal), and
// the update runs unpredicated (rows/columns <= c get zero multipliers; the
// upper triangle receives values that are never read).  double: the narrow
// float64 pipe makes per-thread reciprocals costly, so the owner of the next
// pivot divides once and shares 1/d with the column, and only lower-triangle
// entries are updated.
// The inverse is blocked in 16 x 16 blocks: diagonal blocks in parallel, then
// one block diagonal at a time, W_ij = -W_ii (sum_{k=j}^{i-1} L_ik W_kj).
template <typename T, int NB>
__device__ void potrf_elim(const T* In, int ld_in, T* Lkk, int ld, T* W, T* S, T* Ls,
                           int* status) {
  constexpr int LD = NB + 1;
  constexpr int TM = NB / 16;
  constexpr bool kF64 = sizeof(T) == 8;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  // shared layout (S and Ls hold NB*(NB+4) values each; the scratch of the
  // inverse follows Ls and may overlap In, which is no longer read then):
  //   S:  the tile, NB x LD, then sqrt(d_c) and 1/sqrt(d_c) (2*NB)
  //   Ls: the double-buffered column (2*(NB+1), the last entry 1/d for
  //       float64) during the elimination, then the inverse W (NB x LD)
  T* colbuf = Ls;
  T* sd = S + NB * LD;
  T* rsd = sd + NB;
  T a[TM][TM];
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TM; ++v) a[u][v] = In[(ty + 16 * u) * ld_in + tx + 16 * v];
  for (int i = tid; i < NB; i += kThreads) colbuf[i] = In[i * ld_in];
  if (kF64 && tid == 0) {
    const T d0 = In[0];
    colbuf[NB] = d0 > T(0) ? T(1) / d0 : T(1);
  }
  __syncthreads();
  for (int c = 0; c < NB; ++c) {
    const T* col = colbuf + (c & 1) * (NB + 1);
    T inv_d;
    if constexpr (kF64) {
      inv_d = col[NB];
    } else {
      const T d = col[c];
      inv_d = d > T(0) ? __frcp_rn(d) : T(1);
    }
    T cr[TM], cq[TM];
#pragma unroll
    for (int u = 0; u < TM; ++u) cr[u] = (ty + 16 * u > c) ? col[ty + 16 * u] * inv_d : T(0);
#pragma unroll
    for (int v = 0; v < TM; ++v) cq[v] = (tx + 16 * v > c) ? col[tx + 16 * v] : T(0);
    T* nxt = colbuf + ((c + 1) & 1) * (NB + 1);
#pragma unroll
    for (int v = 0; v < TM; ++v) {
      const int cl = tx + 16 * v;
#pragma unroll
      for (int u = 0; u < TM; ++u) {
        if constexpr (kF64) {
          if (cl > c && cl <= ty + 16 * u) a[u][v] -= cr[u] * cq[v];
        } else {
          a[u][v] -= cr[u] * cq[v];
        }
      }
      if (cl == c + 1) {
#pragma unroll
        for (int u = 0; u < TM; ++u) {
          nxt[ty + 16 * u] = a[u][v];
          if (kF64 && ty + 16 * u == c + 1) nxt[NB] = a[u][v] > T(0) ? T(1) / a[u][v] : T(1);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TM; ++v) S[(ty + 16 * u) * LD + tx + 16 * v] = a[u][v];
  __syncthreads();
  if (tid < NB) {
    T d = S[tid * LD + tid];
    if (!(d > T(0))) {
      set_status(status, SLIM_ENOTPD);
      d = T(1);
    }
    const T r = sqrt(d);
    sd[tid] = r;
    rsd[tid] = T(1) / r;
  }
  __syncthreads();
  // scale the columns: L[c][c] = sqrt(d_c), L[i][c] = S[i][c] / sqrt(d_c)
  for (int idx = tid; idx < NB * NB; idx += kThreads) {
    const int i = idx / NB, c = idx % NB;
    S[i * LD + c] = (i == c) ? sd[c] : (i > c ? S[i * LD + c] * rsd[c] : T(0));
  }
  __syncthreads();
  constexpr int NBLK = NB / 16;
  constexpr int TPB = kThreads / NBLK;      // threads per diagonal block
  constexpr int TPC = TPB / 16;             // threads per column of a block
  T* Wt = Ls;
  for (int idx = tid; idx < NB * NB; idx += kThreads) {
    const int i = idx / NB, c = idx % NB;
    if (i / 16 != c / 16 || i < c) Wt[i * LD + c] = T(0);
  }
  {
    const int blk = tid / TPB, jl = (tid % TPB) / TPC, sub = tid % TPC;
    const int base = blk * 16, j = base + jl;
    for (int il = 0; il < 16; ++il) {
      const int i = base + il;
      T sacc = T(0);
      if (il > jl)
        for (int q = j + sub; q < i; q += TPC) sacc += S[i * LD + q] * Wt[q * LD + j];
#pragma unroll
      for (int o = TPC / 2; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o, TPC);
      __syncwarp();
      if (sub == 0 && il >= jl) Wt[i * LD + j] = (il == jl) ? rsd[j] : -sacc * rsd[i];
      __syncwarp();
    }
  }
  __syncthreads();
  T* Tmp = Ls + NB * gemm_ld(NB);   // sum_k L_ik W_kj, 16 x 16 per block of a diagonal
  for (int d = 1; d < NBLK; ++d) {
    const int nblk = NBLK - d;          // blocks (i, i-d) on this diagonal
    for (int idx = tid; idx < nblk * 256; idx += kThreads) {
      const int bi = idx / 256, e = idx % 256, r = e / 16, c = e % 16;
      const int i = bi + d, j = bi;
      T acc = T(0);
      for (int k = j; k < i; ++k)
#pragma unroll 4
        for (int q = 0; q < 16; ++q)
          acc += S[(i * 16 + r) * LD + k * 16 + q] * Wt[(k * 16 + q) * LD + j * 16 + c];
      Tmp[idx] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < nblk * 256; idx += kThreads) {
      const int bi = idx / 256, e = idx % 256, r = e / 16, c = e % 16;
      const int i = bi + d, j = bi;
      T acc = T(0);
#pragma unroll 4
      for (int q = 0; q < 16; ++q) acc += Wt[(i * 16 + r) * LD + i * 16 + q] * Tmp[bi * 256 + q * 16 + c];
      Wt[(i * 16 + r) * LD + j * 16 + c] = -acc;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < NB * NB; idx += kThreads) {
    const int r = idx / NB, c = idx % NB;
    stcg(Lkk + (size_t)r * ld + c, S[r * LD + c]);
    stcg(W + (size_t)r * NB + c, Wt[r * LD + c]);
  }
  __syncthreads();
}

// Factor the diagonal tile held in S (lower triangle of K_kk after its
// updates) and write L_kk (zeros above the diagonal) to Lg and its inverse
// to Wg.  Blocked by 16 columns: warp 0 factors and inverts the 16 x 16
// diagonal block, the CTA forms the panel below it, L_P = S_P D^{-T}, and
// updates the trailing lower triangle, S -= L_P L_P^T (three barriers per
// panel).  Then the off-diagonal blocks of the inverse, one block diagonal
// at a time: W_ij = -W_ii sum_{k=j}^{i-1} L_ik W_kj.
// Non-positive pivots set SLIM_ENOTPD and are replaced by 1, so the
// factorisation still completes without NaNs.
template <typename T, int NB>
__device__ void potrf_smem(T* S, T* Wt, T* Pn, T* Tmp, T* Lg, int ld, T* Wg, int* status) {
  constexpr int LD = gemm_ld(NB);
  constexpr int LP = kPanelLd;
  constexpr int NBLK = NB / 16;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ty = tid / 16, tx = tid % 16;
  for (int idx = tid; idx < NB * NB; idx += kThreads) {
    const int i = idx / NB, c = idx % NB;
    if (i / 16 < c / 16) Wt[i * LD + c] = T(0);
  }
  for (int pb = 0; pb < NBLK; ++pb) {
    const int c0 = 16 * pb;
    if (warp == 0) diag_block<T>(S + c0 * LD + c0, LD, Wt + c0 * LD + c0, LD, status);
    __syncthreads();
    const int rows = NB - c0 - 16;
    if (rows == 0) break;
    for (int idx = tid; idx < rows * 16; idx += kThreads) {
      const int r = c0 + 16 + idx / 16, c = idx % 16;
      const T* sr = S + r * LD + c0;
      const T* dc = Wt + (c0 + c) * LD + c0;   // row c of D^{-1}, zeros above the diagonal
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < 16; q += 16 / sizeof(T)) {
        constexpr int EV = 16 / sizeof(T);
        T sv[EV], dv[EV];
        lds_vec<T, EV>(sv, sr + q);
        lds_vec<T, EV>(dv, dc + q);
#pragma unroll
        for (int e = 0; e < EV; ++e) acc += sv[e] * dv[e];
      }
      Pn[r * LP + c] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NBLK; ++u) {
      const int r = ty + 16 * u;
      if (r < c0 + 16) continue;
#pragma unroll
      for (int v = 0; v < NBLK; ++v) {
        const int c = tx + 16 * v;
        if (c < c0 + 16 || c > r) continue;
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < 16; q += 16 / sizeof(T)) {
          constexpr int EV = 16 / sizeof(T);
          T pr[EV], pc[EV];
          lds_vec<T, EV>(pr, Pn + r * LP + q);
          lds_vec<T, EV>(pc, Pn + c * LP + q);
#pragma unroll
          for (int e = 0; e < EV; ++e) acc += pr[e] * pc[e];
        }
        S[r * LD + c] -= acc;
      }
    }
    for (int idx = tid; idx < rows * 16; idx += kThreads) {
      const int r = c0 + 16 + idx / 16, c = idx % 16;
      S[r * LD + c0 + c] = Pn[r * LP + c];
    }
    __syncthreads();
  }
  constexpr int EVI = 16 / sizeof(T);
#pragma unroll
  for (int d = 1; d < NBLK; ++d) {
    const int nblk = NBLK - d;   // blocks (i, i-d) on this block diagonal
    for (int idx = tid; idx < nblk * 256; idx += kThreads) {
      const int bi = idx / 256, e = idx % 256, r = e / 16, c = e % 16;
      const int i = bi + d, j = bi;
      T acc = T(0);
#pragma unroll
      for (int kk = 0; kk < d; ++kk) {
        const int k = j + kk;
#pragma unroll
        for (int q = 0; q < 16; q += EVI) {
          T sv[EVI];
          lds_vec<T, EVI>(sv, S + (i * 16 + r) * LD + k * 16 + q);
#pragma unroll
          for (int f = 0; f < EVI; ++f) acc += sv[f] * Wt[(k * 16 + q + f) * LD + j * 16 + c];
        }
      }
      Tmp[idx] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < nblk * 256; idx += kThreads) {
      const int bi = idx / 256, e = idx % 256, r = e / 16, c = e % 16;
      const int i = bi + d;
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < 16; q += EVI) {
        T wv[EVI];
        lds_vec<T, EVI>(wv, Wt + (i * 16 + r) * LD + i * 16 + q);
#pragma unroll
        for (int f = 0; f < EVI; ++f) acc += wv[f] * Tmp[bi * 256 + (q + f) * 16 + c];
      }
      Wt[(i * 16 + r) * LD + bi * 16 + c] = -acc;
    }
    __syncthreads();
  }
  constexpr int EV = 16 / sizeof(T);
  for (int idx = tid; idx < NB * NB / EV; idx += kThreads) {
    const int r = idx / (NB / EV), c = (idx % (NB / EV)) * EV;
    T lo[EV], wo[EV];
#pragma unroll
    for (int e = 0; e < EV; ++e) {
      lo[e] = (c + e <= r) ? S[r * LD + c + e] : T(0);
      wo[e] = Wt[r * LD + c + e];
    }
    st_vec16(Lg + (size_t)r * ld + c, lo);
    st_vec16(Wg + (size_t)r * NB + c, wo);
  }
  __syncthreads();
}

// float32, NB = 64: the tile factorisation laid out for latency.  The 64
// pivots of a tile are a chain that no blocking shortens, so the chain runs
// in one warp with the 16 x 16 diagonal block in registers, and everything
// else runs on the other warps in its shadow.
constexpr int kLd64 = 68;       // gemm_ld(64)
constexpr int kLtLd = 17;       // transposed diagonal factor, 16 x 17

// One warp: the 16 x 16 diagonal block at (c0, c0) of S, minus the product of
// the previous panel's rows with themselves when `upd` (Pn rows c0..c0+15,
// 16 columns), factored in registers and inverted.  Lane l (and its mirror
// l + 16) holds row l.  Pivot c: the diagonal element comes from lane c, each
// lane scales its own column-c entry and the scaled column reaches the other
// rows by shuffles; entries above the diagonal carry values that are never
// read.  The inverse X = D^{-1} is formed column by column (lane l: column l)
// right-looking, X_ql = -(sum_{i<q} L_qi X_il) / L_qq.  L_D goes to S, X to
// Wt (block (c0, c0)).  Non-positive pivots set SLIM_ENOTPD and are replaced
// by 1.
__device__ __forceinline__ void diag16_f32(float* S, float* Wt, const float* Pn, bool upd, int c0,
                                        float* Lt, int* status) {
  const int lane = threadIdx.x & 31, l = lane & 15;
  float* srow = S + (c0 + l) * kLd64 + c0;
  float a[16];
#pragma unroll
  for (int q = 0; q < 16; q += 4) {
    const float4 v = *reinterpret_cast<const float4*>(srow + q);
    a[q] = v.x; a[q + 1] = v.y; a[q + 2] = v.z; a[q + 3] = v.w;
  }
  if (upd) {
    float pr[16];
    const float* prow = Pn + (c0 + l) * kPanelLd;
#pragma unroll
    for (int q = 0; q < 16; q += 4) {
      const float4 v = *reinterpret_cast<const float4*>(prow + q);
      pr[q] = v.x; pr[q + 1] = v.y; pr[q + 2] = v.z; pr[q + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float* pj = Pn + (c0 + j) * kPanelLd;
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        const float4 v = *reinterpret_cast<const float4*>(pj + q);
        acc += pr[q] * v.x;
        acc += pr[q + 1] * v.y;
        acc += pr[q + 2] * v.z;
        acc += pr[q + 3] * v.w;
      }
      a[j] -= acc;
    }
  }
  bool bad = false;
  float my_rs = 1.f;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const float d = __shfl_sync(0xffffffffu, a[c], c);
    const bool ok = d > 0.f;
    bad |= !ok;
    const float dd = ok ? d : 1.f;
    const float rs = rsqrtf(dd);
    if (l == c) my_rs = rs;
    const float lc = (l == c ? dd : a[c]) * rs;
    a[c] = lc;
#pragma unroll
    for (int j = c + 1; j < 16; ++j) a[j] -= lc * __shfl_sync(0xffffffffu, lc, j);
  }
  if (bad && lane == 0) set_status(status, SLIM_ENOTPD);
  if (lane < 16) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j <= l) srow[j] = a[j];
      Lt[j * kLtLd + l] = j <= l ? a[j] : 0.f;   // Lt[q][i] = L_iq
    }
  }
  __syncwarp();
  float rsv[16], sacc[16], x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    rsv[i] = __shfl_sync(0xffffffffu, my_rs, i);
    sacc[i] = 0.f;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    x[q] = q == l ? rsv[q] : (q > l ? -rsv[q] * sacc[q] : 0.f);
#pragma unroll
    for (int i = q + 1; i < 16; ++i) sacc[i] += Lt[q * kLtLd + i] * x[q];
  }
  if (lane < 16) {
#pragma unroll
    for (int i = 0; i < 16; ++i) Wt[(c0 + i) * kLd64 + c0 + l] = x[i];
  }
  __syncwarp();
}

// Factor the 64 x 64 tile in S (lower triangle) into L_kk (to S, then Lg) and
// its inverse W (Wt, then Wg), blocked by 16 columns, two barriers per block:
//   B(pb), all warps: the panel below block pb, L_P = S_P X_pb^T, into Pn;
//          and W's row-block pb, W_pb,j = -X_pb T_pb,j (j < pb).
//   C(pb), warp 0: the next diagonal block, updated by the panel, factored
//          and inverted (X_pb+1);  warps 1-7 meanwhile: the rest of the
//          trailing update S -= L_P L_P^T, the panel copied into S, and
//          T_pb+1,j = sum_{k=j..pb} L_pb+1,k W_k,j for the next row-block of W.
// Shared scratch: Pn (64 x 20), Tmp (3 blocks of 16 x 16), Lt (16 x 17).
__device__ __noinline__ void potrf_la_f32(float* S, float* Wt, float* Pn, float* Tmp, float* Lt, float* Lg,
                             int ld, float* Wg, int* status) {
  constexpr int LD = kLd64, LP = kPanelLd;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int idx = tid; idx < 64 * 64; idx += kThreads) {
    const int i = idx / 64, c = idx % 64;
    if (i / 16 < c / 16) Wt[i * LD + c] = 0.f;
  }
  if (warp == 0) diag16_f32(S, Wt, Pn, false, 0, Lt, status);
  __syncthreads();
  for (int pb = 0; pb < 4; ++pb) {
    const int c0 = 16 * pb;
    const int rows = 48 - c0;
    // B(pb)
    for (int idx = tid; idx < rows * 16; idx += kThreads) {
      const int r = c0 + 16 + idx / 16, c = idx % 16;
      const float* sr = S + r * LD + c0;
      const float* xc = Wt + (c0 + c) * LD + c0;   // row c of X_pb, zeros above the diagonal
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        const float4 u = *reinterpret_cast<const float4*>(sr + q);
        const float4 v = *reinterpret_cast<const float4*>(xc + q);
        acc += u.x * v.x;
        acc += u.y * v.y;
        acc += u.z * v.z;
        acc += u.w * v.w;
      }
      Pn[r * LP + c] = acc;
    }
    for (int idx = tid; idx < pb * 256; idx += kThreads) {
      const int j = idx / 256, e = idx % 256, rr = e / 16, cc = e % 16;
      const float* xr = Wt + (c0 + rr) * LD + c0;
      const float* t = Tmp + j * 256 + cc;
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 16; ++q) acc += xr[q] * t[q * 16];
      Wt[(c0 + rr) * LD + 16 * j + cc] = -acc;
    }
    __syncthreads();
    if (pb == 3) break;
    // C(pb)
    const int n0 = c0 + 16;   // first row / column of the trailing matrix
    if (warp == 0) {
      diag16_f32(S, Wt, Pn, true, n0, Lt, status);
    } else {
      const int t = tid - 32, nt = kThreads - 32;
      // trailing blocks (bi, bj), pb+1 <= bj <= bi <= 3, except (pb+1, pb+1)
      const int nb = 3 - pb;                  // block rows of the trailing matrix
      const int nblk = nb * (nb + 1) / 2 - 1;
      for (int idx = t; idx < nblk * 256; idx += nt) {
        int b = idx / 256 + 1;                // triangle index, 0 is (pb+1, pb+1)
        int bi = 0;
        while (b > bi) b -= ++bi;
        const int r = n0 + 16 * bi + (idx % 256) / 16, c = n0 + 16 * b + idx % 16;
        const float* pr = Pn + r * LP;
        const float* pc = Pn + c * LP;
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < 16; q += 4) {
          const float4 u = *reinterpret_cast<const float4*>(pr + q);
          const float4 v = *reinterpret_cast<const float4*>(pc + q);
          acc += u.x * v.x;
          acc += u.y * v.y;
          acc += u.z * v.z;
          acc += u.w * v.w;
        }
        S[r * LD + c] -= acc;
      }
      for (int idx = t; idx < rows * 16; idx += nt) {
        const int r = n0 + idx / 16, q = idx % 16;
        S[r * LD + c0 + q] = Pn[r * LP + q];
      }
      // T_{pb+1, j} for j <= pb; L_{pb+1, pb} is still in Pn
      for (int idx = t; idx < (pb + 1) * 256; idx += nt) {
        const int j = idx / 256, rr = (idx % 256) / 16, cc = idx % 16;
        const int r = n0 + rr;
        float acc = 0.f;
        for (int k = j; k <= pb; ++k) {
          const float* lr = k < pb ? S + r * LD + 16 * k : Pn + r * LP;
          const float* wc = Wt + 16 * k * LD + 16 * j + cc;
#pragma unroll
          for (int q = 0; q < 16; ++q) acc += lr[q] * wc[q * LD];
        }
        Tmp[j * 256 + rr * 16 + cc] = acc;
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < 64 * 16; idx += kThreads) {
    const int r = idx / 16, c = (idx % 16) * 4;
    float lo[4], wo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      lo[e] = (c + e <= r) ? S[r * LD + c + e] : 0.f;
      wo[e] = Wt[r * LD + c + e];
    }
    st_vec16(Lg + (size_t)r * ld + c, lo);
    st_vec16(Wg + (size_t)r * 64 + c, wo);
  }
  __syncthreads();
}

// Factor the diagonal tile staged in S (float32: blocked by 16 columns;
// float64: CTA-wide elimination, where the narrow float64 pipe makes one
// warp's serial 16 x 16 factorisations slow).
template <typename T, int NB>
__device__ __forceinline__ void potrf_tile(T* S, T* As, T* Bs, T* Lg, int ld, T* Wg, int* status) {
  if constexpr (sizeof(T) == 8)
    potrf_elim<T, NB>(S, gemm_ld(NB), Lg, ld, Wg, As, Bs, status);
  else if constexpr (NB == 64)
    potrf_la_f32(S, Bs, As, As + 64 * kPanelLd, As + 64 * kPanelLd + 3 * 256, Lg, ld, Wg, status);
  else
    potrf_smem<T, NB>(S, Bs, As, As + NB * kPanelLd, Lg, ld, Wg, status);
}

// The critical path of panel k in one task (i = k+1): L_ik = A_ik W_k^T
// (published at once for the trailing updates), then A_ii -= L_ik L_ik^T with
// L_ik kept in shared memory, then the factorisation of tile (i,i).
template <typename T, int NB>
__device__ __noinline__ void task_panel(T* t_ik, T* t_ii, int P, const T* w_k, T* w_i, int* flag_ik, T* As,
                           T* Bs, T* S, int* status) {
  constexpr int LD = gemm_ld(NB);
  constexpr int TM = NB / 16;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  stage_tiles<T, NB>(t_ik, P, w_k, NB, t_ii, P, As, Bs, S);
  T acc[TM][TM];
  gemm_core<T, NB>(As, Bs, acc);
  __syncthreads();   // every thread is done reading As
#pragma unroll
  for (int a = 0; a < TM; ++a) st_row<T, TM>(t_ik + (size_t)(ty * TM + a) * P + tx * TM, acc[a]);
  // As[c][r] = X[r][c]: the thread's TM rows of column c are contiguous
#pragma unroll
  for (int b = 0; b < TM; ++b) {
    T col[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) col[a] = acc[a][b];
    if constexpr (TM * sizeof(T) == 16) {
      vec16_t<T> o;
      T* po = reinterpret_cast<T*>(&o);
#pragma unroll
      for (int a = 0; a < TM; ++a) po[a] = col[a];
      *reinterpret_cast<vec16_t<T>*>(As + (tx * TM + b) * LD + ty * TM) = o;
    } else {
#pragma unroll
      for (int a = 0; a < TM; ++a) As[(tx * TM + b) * LD + ty * TM + a] = col[a];
    }
  }
  cta_publish(flag_ik);
  gemm_core<T, NB>(As, As, acc);
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) S[(ty * TM + a) * LD + tx * TM + b] -= acc[a][b];
  __syncthreads();
  potrf_tile<T, NB>(S, As, Bs, t_ii, P, w_i, status);
}

// Factor diagonal tile (k,k) when nothing precedes it (k = 0).
template <typename T, int NB>
__device__ __noinline__ void task_potrf(T* Lkk, int P, T* w_k, T* As, T* Bs, T* S, int* status) {
  TileRegs<T, NB> rc;
  rc.load(Lkk, P);
  rc.store_n(S);
  __syncthreads();
  potrf_tile<T, NB>(S, As, Bs, Lkk, P, w_k, status);
}

// Run task tk of the factorisation of L (P x P, Tt x Tt tiles): wait for its
// inputs on the tile counters, compute, publish.  Returns false when a wait
// ran out or another CTA asked everyone to stop.
template <typename T, int NB>
__device__ __forceinline__ bool run_factor_task(const CholTask tk, T* L, int P, int Tt, int* cnt,
                                                T* winv, int* status, int* abort_flag, T* As,
                                                T* Bs, T* S, int* s_ok3, int* s_ok8) {
  const int i = tk.i, m = tk.m, k = tk.k;
  bool ok = true;
  if (tk.type == kUpd) {
    ok = cta_wait(&cnt[i * Tt + k], k + 1, &cnt[m * Tt + k], k + 1, &cnt[i * Tt + m], k, 3,
                  abort_flag, status, s_ok3);
    if (ok) {
      T* tile_im = L + (size_t)i * NB * P + (size_t)m * NB;
      const T* Lik = L + (size_t)i * NB * P + (size_t)k * NB;
      const T* Lmk = L + (size_t)m * NB * P + (size_t)k * NB;
      task_gemm<T, NB>(tile_im, P, Lik, P, Lmk, P, tile_im, T(-1), As, Bs, S);
      cta_publish(&cnt[i * Tt + m]);
    }
  } else if (tk.type == kUpd4) {
    ok = cta_wait_group(cnt, Tt, i, m, k, abort_flag, status, s_ok8);
    if (ok) {
      if constexpr (sizeof(T) == 4 && NB == 64) {
        task_gemm_group<NB>(L + (size_t)i * NB * P + (size_t)m * NB, P,
                            L + (size_t)i * NB * P + (size_t)k * NB,
                            L + (size_t)m * NB * P + (size_t)k * NB, As, As + NB * (2 * NB + 4));
      } else {
        set_status(status, SLIM_EINVAL);   // the list holds no groups for this factor
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        red_release_add(&cnt[i * Tt + m], 1);
        red_release_add(&cnt[i * Tt + m + 1], 1);
        red_release_add(&cnt[(i + 1) * Tt + m], 1);
        red_release_add(&cnt[(i + 1) * Tt + m + 1], 1);
      }
    }
  } else if (tk.type == kTrsm) {
    ok = cta_wait(&cnt[m * Tt + m], m + 1, &cnt[i * Tt + m], m, nullptr, 0, 2, abort_flag,
                  status, s_ok3);
    if (ok) {
      T* tile_im = L + (size_t)i * NB * P + (size_t)m * NB;
      task_gemm<T, NB>(tile_im, P, tile_im, P, winv + (size_t)m * NB * NB, NB, nullptr, T(1),
                       As, Bs, S);
      cta_publish(&cnt[i * Tt + m]);
    }
  } else if (tk.type == kPanel) {
    ok = cta_wait(&cnt[k * Tt + k], k + 1, &cnt[i * Tt + k], k, &cnt[i * Tt + i], k, 3,
                  abort_flag, status, s_ok3);
    if (ok) {
      task_panel<T, NB>(L + (size_t)i * NB * P + (size_t)k * NB,
                        L + (size_t)i * NB * P + (size_t)i * NB, P, winv + (size_t)k * NB * NB,
                        winv + (size_t)i * NB * NB, &cnt[i * Tt + k], As, Bs, S, status);
      cta_publish(&cnt[i * Tt + i], 2);
    }
  } else {
    ok = cta_wait(&cnt[k * Tt + k], k, abort_flag, status, s_ok3);
    if (ok) {
      task_potrf<T, NB>(L + (size_t)k * NB * P + (size_t)k * NB, P, winv + (size_t)k * NB * NB,
                        As, Bs, S, status);
      cta_publish(&cnt[k * Tt + k]);
    }
  }
  return ok;
}

// R: the register cap per thread.  255 when one CTA has the SM to itself:
// below that the task code keeps values across its non-inlined calls in
// memory, and the chain of diagonal tiles runs about 1.5x slower; 128 lets two
// CTAs, or a factorisation CTA and other kernels, share an SM.
constexpr int kRegsWide = 255, kRegsShared = 128;

template <typename T, int NB, int R>
__global__ void __maxnreg__(R) chol_factor_kernel(T* L, int P, int Tt,
                                                               const CholTask* tasks, int ntasks,
                                                               int* cnt, int* ticket, T* winv,
                                                               int* status, int* abort_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);
  T* Bs = As + NB * gemm_ld(NB);
  T* S = Bs + NB * gemm_ld(NB);
  __shared__ int s_task, s_ok3[3], s_ok8[8];
  __shared__ CholTask s_desc;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int t = atomicAdd(ticket, 1);
    s_task = t;
    if (t < ntasks) s_desc = tasks[t];
  }
  __syncthreads();
  for (;;) {
    const int t = s_task;
    if (t >= ntasks) return;
    const CholTask tk = s_desc;
    // thread 32 claims the next ticket while the CTA works on this one; the
    // claimed task is started only after this one finishes, which keeps the
    // claim order a valid execution order
    int next = 0;
    if (tid == 32) next = atomicAdd(ticket, 1);
    __syncthreads();
    const bool ok = run_factor_task<T, NB>(tk, L, P, Tt, cnt, winv, status, abort_flag, As, Bs, S,
                                           s_ok3, s_ok8);
    __syncthreads();
    if (tid == 32) {
      s_task = ok ? next : ntasks;
      if (ok && next < ntasks) s_desc = tasks[next];
    }
    __syncthreads();
  }
}

// Many factorisations in one persistent launch: the CTAs claim (problem,
// task) pairs from one merged queue in which every problem's tasks keep
// their own order, so a claimed task depends only on tasks of its problem
// claimed before it and the launch always makes progress.
template <typename T, int NB, int R>
__global__ void __maxnreg__(R) chol_factor_batch_kernel(
    const FactorJob* jobs, const int2* queue, int nqueue, int* ticket, int* abort_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);
  T* Bs = As + NB * gemm_ld(NB);
  T* S = Bs + NB * gemm_ld(NB);
  __shared__ int s_task, s_ok3[3], s_ok8[8];
  __shared__ int2 s_q;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int t = atomicAdd(ticket, 1);
    s_task = t;
    if (t < nqueue) s_q = queue[t];
  }
  __syncthreads();
  for (;;) {
    const int t = s_task;
    if (t >= nqueue) return;
    const int2 q = s_q;
    const FactorJob jb = jobs[q.x];
    const CholTask tk = jb.tasks[q.y];
    int next = 0;
    if (tid == 32) next = atomicAdd(ticket, 1);
    __syncthreads();
    const bool ok = run_factor_task<T, NB>(tk, reinterpret_cast<T*>(jb.L), jb.P, jb.T, jb.cnt,
                                           reinterpret_cast<T*>(jb.winv), jb.status, abort_flag,
                                           As, Bs, S, s_ok3, s_ok8);
    __syncthreads();
    if (tid == 32) {
      s_task = ok ? next : nqueue;
      if (ok && next < nqueue) s_q = queue[next];
    }
    __syncthreads();
  }
}

// One diagonal tile on its own (the launch-per-panel factorisation): factor
// tile (j, j) of L in place and write its inverse to winv[j].
__global__ void __launch_bounds__(kThreads) chol_potrf_tile_kernel(float* L, int P, int j,
                                                                    float* winv, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* As = reinterpret_cast<float*>(smem_raw);
  float* Bs = As + 64 * gemm_ld(64);
  float* S = Bs + 64 * gemm_ld(64);
  task_potrf<float, 64>(L + (size_t)j * 64 * P + (size_t)j * 64, P, winv + (size_t)j * 64 * 64,
                        As, Bs, S, status);
}

// Row-split GEMV pieces: thread (r = tid/TPR, sub = tid%TPR) owns columns
// sub*CPT .. sub*CPT+CPT-1 of row r.  Tiles are loaded into registers before
// the wait for the vector they multiply, hiding the L2 latency of the tile.
template <typename T, int NB>
struct RowPart {
  static constexpr int TPR = kThreads / NB;
  static constexpr int CPT = NB / TPR;
  T v[CPT];
  // 16-byte loads (the rows of a tile start on 16-byte boundaries: ld and the
  // tile offsets are multiples of 4 floats / 2 doubles)
  __device__ void load(const T* M, int ld) {
    const int r = threadIdx.x / TPR, sub = threadIdx.x % TPR;
    const T* p = M + (size_t)r * ld + sub * CPT;
    if constexpr ((CPT * sizeof(T)) % 16 == 0) {
      constexpr int EV = 16 / sizeof(T);
#pragma unroll
      for (int q = 0; q < CPT; q += EV) {
        const vec16_t<T> t = __ldcg(reinterpret_cast<const vec16_t<T>*>(p + q));
        const T* pt = reinterpret_cast<const T*>(&t);
#pragma unroll
        for (int e = 0; e < EV; ++e) v[q + e] = pt[e];
      }
    } else {
#pragma unroll
      for (int q = 0; q < CPT; ++q) v[q] = ldcg(p + q);
    }
  }
  // acc[r] += sign * (M v)[r]
  __device__ void apply(const T* vec, T* acc, T sign) const {
    const int r = threadIdx.x / TPR, sub = threadIdx.x % TPR;
    T s = T(0);
#pragma unroll
    for (int q = 0; q < CPT; ++q) s += v[q] * vec[sub * CPT + q];
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
    if (sub == 0) acc[r] += sign * s;
  }
};

// Column-split transposed GEMV: thread (a = tid%NB, ch = tid/NB) owns rows
// ch*RPC .. ch*RPC+RPC-1 of column a; partial sums meet in shared memory.
template <typename T, int NB>
struct ColPart {
  static constexpr int CH = kThreads / NB;
  static constexpr int RPC = NB / CH;
  T v[RPC];
  __device__ void load(const T* M, int ld) {
    const int a = threadIdx.x % NB, ch = threadIdx.x / NB;
#pragma unroll
    for (int q = 0; q < RPC; ++q) v[q] = ldcg(M + (size_t)(ch * RPC + q) * ld + a);
  }
  // acc[a] += sign * (M^T vec)[a]; `part` holds kThreads partial sums
  __device__ void apply(const T* vec, T* acc, T sign, T* part) const {
    const int a = threadIdx.x % NB, ch = threadIdx.x / NB;
    T s = T(0);
#pragma unroll
    for (int q = 0; q < RPC; ++q) s += v[q] * vec[ch * RPC + q];
    part[ch * NB + a] = s;
    __syncthreads();
    if (threadIdx.x < NB) {
      T t = T(0);
#pragma unroll
      for (int c = 0; c < CH; ++c) t += part[c * NB + threadIdx.x];
      acc[threadIdx.x] += sign * t;
    }
  }
};

template <typename T, int NB>
__global__ void __launch_bounds__(kThreads) chol_fwd_kernel(const T* L, int P, int Tt,
                                                            const T* winv, const double* v, T* y,
                                                            int* fflag, int* ticket, int* status,
                                                            int* abort_flag) {
  __shared__ T acc[NB], vec[NB], out[NB];
  __shared__ int s_task, s_ok3[3];
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(ticket, 1);
    __syncthreads();
    const int i = s_task;
    __syncthreads();
    if (i >= Tt) return;
    RowPart<T, NB> wpart, lpart;
    wpart.load(winv + (size_t)i * NB * NB, NB);
    if (threadIdx.x < NB) acc[threadIdx.x] = (T)v[i * NB + threadIdx.x];
    for (int j = 0; j < i; ++j) {
      lpart.load(L + (size_t)i * NB * P + (size_t)j * NB, P);
      if (!cta_wait(&fflag[j], 1, abort_flag, status, s_ok3)) return;
      if (threadIdx.x < NB) vec[threadIdx.x] = ldcg(y + j * NB + threadIdx.x);
      __syncthreads();
      lpart.apply(vec, acc, T(-1));
      __syncthreads();
    }
    if (threadIdx.x < NB) out[threadIdx.x] = T(0);
    __syncthreads();
    wpart.apply(acc, out, T(1));
    __syncthreads();
    if (threadIdx.x < NB) stcg(y + i * NB + threadIdx.x, out[threadIdx.x]);
    cta_publish(&fflag[i]);
  }
}

template <typename T, int NB>
__global__ void __launch_bounds__(kThreads) chol_bwd_kernel(const T* L, int P, int Tt,
                                                            const T* winv, const T* y, T* zt,
                                                            double* z, int* bflag, int* ticket,
                                                            int* status, int* abort_flag) {
  __shared__ T acc[NB], vec[NB], out[NB];
  __shared__ T part[kThreads];
  __shared__ int s_task, s_ok3[3];
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= Tt) return;
    const int i = Tt - 1 - t;
    ColPart<T, NB> wpart, lpart;
    wpart.load(winv + (size_t)i * NB * NB, NB);
    if (threadIdx.x < NB) acc[threadIdx.x] = ldcg(y + i * NB + threadIdx.x);
    for (int j = Tt - 1; j > i; --j) {
      lpart.load(L + (size_t)j * NB * P + (size_t)i * NB, P);
      if (!cta_wait(&bflag[j], 1, abort_flag, status, s_ok3)) return;
      if (threadIdx.x < NB) vec[threadIdx.x] = ldcg(zt + j * NB + threadIdx.x);
      __syncthreads();
      lpart.apply(vec, acc, T(-1), part);
      __syncthreads();
    }
    if (threadIdx.x < NB) out[threadIdx.x] = T(0);
    __syncthreads();
    wpart.apply(acc, out, T(1), part);
    __syncthreads();
    if (threadIdx.x < NB) {
      stcg(zt + i * NB + threadIdx.x, out[threadIdx.x]);
      z[i * NB + threadIdx.x] = (double)out[threadIdx.x];
    }
    cta_publish(&bflag[i]);
  }
}

// ---------------------------------------------------------------------------
// Both triangular solves of L L^T z = v in one thread-block cluster.
//
// Tile row i belongs to CTA i mod C.  Every CTA keeps the whole of y (and
// then z) in its shared memory.  The owner of a tile row sends its NB values
// to every other CTA of the cluster with one bulk copy each (distributed
// shared memory); the copy completes a per-row mbarrier in the receiving CTA,
// on which that CTA waits.  While waiting for row j-1, a CTA has already
// folded rows < j-1 into its accumulator (batches of tiles with all loads in
// flight), so each link of the chain costs one NB x NB matrix-vector product
// and one copy.  Every wait is bounded; before leaving, each CTA waits for all
// copies addressed to it.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return done != 0;
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
// Copy `bytes` (multiple of 16, 16-byte aligned) from this CTA's shared memory
// to the CTA whose addresses are dst / bar; the copy completes that CTA's mbarrier.
__device__ __forceinline__ void bulk_copy_to(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "r"(src), "r"(bytes), "r"(bar) : "memory");
}

constexpr int kSolveBatch = 4;   // tiles folded per batch

// CTA-wide bounded wait until the rows [j0, j1) owned by other CTAs have
// arrived (their mbarriers in this CTA completed).
__device__ bool cluster_wait_rows(uint64_t* bars, int j0, int j1, int C, int rank, unsigned limit,
                                  int* abort_flag, int* status, int* s_ok) {
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int j = j0; ok && j < j1; ++j) {
      if (j % C == rank) continue;
      unsigned it = 0;
      while (!mbar_try_wait(&bars[j], 0)) {
        if (++it > limit) {
          set_status(status, SLIM_ETIMEOUT);
          atomicExch(abort_flag, 1);
          ok = 0;
          break;
        }
        if ((it & 255u) == 0 && ld_acquire(abort_flag)) {
          ok = 0;
          break;
        }
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  const int ok = *s_ok;
  __syncthreads();
  return ok != 0;
}

// Transposed GEMV piece: thread (a = tid%NB, ch = tid/NB) holds rows
// ch*RPC .. ch*RPC+RPC-1 of column a of a tile (a warp reads whole rows of the
// tile, coalesced); (M^T vec)[a] is the sum of the CH partial sums of column a.
template <typename T, int NB>
struct TPart {
  static constexpr int CH = kThreads / NB;
  static constexpr int RPC = NB / CH;
  T v[RPC];
  __device__ void load(const T* M, int ld) {
    const int a = threadIdx.x % NB, ch = threadIdx.x / NB;
#pragma unroll
    for (int q = 0; q < RPC; ++q) v[q] = ldcg(M + (size_t)(ch * RPC + q) * ld + a);
  }
  // partial sum of column a over this thread's rows of vec (shared memory)
  __device__ T dot(const T* vec) const {
    const int ch = threadIdx.x / NB;
    T s = T(0);
    constexpr int EV = (RPC * sizeof(T)) % 16 == 0 ? 16 / (int)sizeof(T) : 1;
    T x[EV];
#pragma unroll
    for (int q = 0; q < RPC; q += EV) {
      lds_vec<T, EV>(x, vec + ch * RPC + q);
#pragma unroll
      for (int e = 0; e < EV; ++e) s += v[q + e] * x[e];
    }
    return s;
  }
};

// Partial sum of row r over this thread's columns of vec (RowPart layout).
template <typename T, int NB>
__device__ __forceinline__ T row_dot(const RowPart<T, NB>& m, const T* vec) {
  constexpr int CPT = RowPart<T, NB>::CPT;
  constexpr int EV = (CPT * sizeof(T)) % 16 == 0 ? 16 / (int)sizeof(T) : 1;
  const int sub = threadIdx.x % RowPart<T, NB>::TPR;
  T s = T(0);
  T x[EV];
#pragma unroll
  for (int q = 0; q < CPT; q += EV) {
    lds_vec<T, EV>(x, vec + sub * CPT + q);
#pragma unroll
    for (int e = 0; e < EV; ++e) s += m.v[q + e] * x[e];
  }
  return s;
}

// Store one value into a peer CTA's shared memory; the store completes that
// CTA's mbarrier by sizeof(value) bytes.
__device__ __forceinline__ void st_async_peer(uint32_t addr, float val, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
               ::"r"(addr), "r"(__float_as_uint(val)), "r"(bar) : "memory");
}
__device__ __forceinline__ void st_async_peer(uint32_t addr, double val, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
               ::"r"(addr), "l"(__double_as_longlong(val)), "r"(bar) : "memory");
}

// Bounded wait of the calling thread for a row's arrival.
__device__ __forceinline__ void thread_wait_row(uint64_t* bar, int* abort_flag, int* status) {
  unsigned it = 0;
  while (!mbar_try_wait(bar, 0)) {
    if (++it > kSpinLimit) {
      set_status(status, SLIM_ETIMEOUT);
      atomicExch(abort_flag, 1);
      return;
    }
    if ((it & 255u) == 0 && ld_acquire(abort_flag)) return;
  }
}

template <typename T, int NB>
__global__ void __launch_bounds__(kThreads) chol_solve_cluster_kernel(
    const T* L, int P, int Tt, const T* winv, const double* v, double* z, int* status,
    int* abort_flag, int i0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* y = reinterpret_cast<T*>(smem_raw);     // [P] forward solution
  T* zt = y + P;                              // [P] backward solution
  uint64_t* fbar = reinterpret_cast<uint64_t*>(zt + P);   // [Tt] arrival of y rows
  uint64_t* bbar = fbar + Tt;                             // [Tt] arrival of z rows
  __shared__ __align__(16) T acc[NB];
  __shared__ T part[kThreads];
  __shared__ int s_ok;
  using RP = RowPart<T, NB>;
  using TP = TPart<T, NB>;
  constexpr int TPR = RP::TPR, CPT = RP::CPT;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, r = tid / TPR, sub = tid % TPR;
  if (tid == 0) {
    for (int i = 0; i < Tt; ++i) {
      mbar_init(&fbar[i], 1);
      mbar_init(&bbar[i], 1);
      if (i % C != rank) {   // rows sent by other CTAs: one arrival expecting NB values
        if (i >= i0) mbar_expect_tx(&fbar[i], NB * sizeof(T));   // y rows above i0 are not sent
        mbar_expect_tx(&bbar[i], NB * sizeof(T));
      }
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // v is zero above tile i0, hence so is y: every CTA holds those rows as zero
  for (int q = tid; q < i0 * NB; q += kThreads) y[q] = T(0);
  cl.sync();   // every CTA's barriers exist before anyone sends
  bool ok = true;
  // The owner of row i finishes it with one barrier on the chain: every thread
  // waits for row i-1 itself, the rows' accumulators meet in shared memory,
  // and the lanes holding the results store them into every peer.
  // forward: y_i = W_i (v_i - sum_{i0<=j<i} L_ij y_j), from the first tile
  // i >= i0 this CTA owns
  for (int i = i0 + ((rank - i0) % C + C) % C; ok && i < Tt; i += C) {
    RP wp, lastp;
    wp.load(winv + (size_t)i * NB * NB, NB);
    if (i > i0) lastp.load(L + (size_t)i * NB * P + (size_t)(i - 1) * NB, P);
    T s = T(0);
    for (int j = i0; j + 1 < i; j += kSolveBatch) {   // rows i0 .. i-2, batches in flight
      const int nj = min(kSolveBatch, i - 1 - j);
      RP bp[kSolveBatch];
#pragma unroll
      for (int u = 0; u < kSolveBatch; ++u)
        if (u < nj) bp[u].load(L + (size_t)i * NB * P + (size_t)(j + u) * NB, P);
      if (!cluster_wait_rows(fbar, j, j + nj, C, rank, kSpinLimit, abort_flag, status, &s_ok)) {
        ok = false;
        break;
      }
#pragma unroll
      for (int u = 0; u < kSolveBatch; ++u)
        if (u < nj) s += row_dot<T, NB>(bp[u], y + (j + u) * NB);
    }
    if (!ok) break;
    if (i > i0) {
      if ((i - 1) % C != rank) thread_wait_row(&fbar[i - 1], abort_flag, status);
      s += row_dot<T, NB>(lastp, y + (i - 1) * NB);
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
    if (sub == 0) acc[r] = (T)v[i * NB + r] - s;
    __syncthreads();
    T w = row_dot<T, NB>(wp, acc);
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o, TPR);
    // the TPR lanes of row r all hold w: each stores it into every TPR-th peer
    if (sub == 0) y[i * NB + r] = w;
    {
      const uint32_t la = smem_u32(y + i * NB + r), lb = smem_u32(&fbar[i]);
      for (int d = sub; d < C; d += TPR)
        if (d != rank) st_async_peer(map_to_rank(la, d), w, map_to_rank(lb, d));
    }
    __syncthreads();
  }
  // backward: z_i = W_i^T (y_i - sum_{j>i} L_ji^T z_j); column sums meet in
  // shared memory (one barrier each)
  const int a = tid % NB, ch = tid / NB;
  const int last = Tt - 1 - ((Tt - 1 - rank) % C + C) % C;   // largest i = rank (mod C)
  for (int i = last; ok && i >= 0; i -= C) {
    TP wp, nextp;
    wp.load(winv + (size_t)i * NB * NB, NB);
    if (i + 1 < Tt) nextp.load(L + (size_t)(i + 1) * NB * P + (size_t)i * NB, P);
    T s = T(0);
    for (int j = Tt - 1; j > i + 1; j -= kSolveBatch) {   // rows > i+1, batches in flight
      const int nj = min(kSolveBatch, j - i - 1);         // tiles j, j-1, .., j-nj+1
      TP bp[kSolveBatch];
#pragma unroll
      for (int u = 0; u < kSolveBatch; ++u)
        if (u < nj) bp[u].load(L + (size_t)(j - u) * NB * P + (size_t)i * NB, P);
      if (!cluster_wait_rows(bbar, j - nj + 1, j + 1, C, rank, kSpinLimit, abort_flag, status,
                             &s_ok)) {
        ok = false;
        break;
      }
#pragma unroll
      for (int u = 0; u < kSolveBatch; ++u)
        if (u < nj) s += bp[u].dot(zt + (j - u) * NB);
    }
    if (!ok) break;
    if (i + 1 < Tt) {
      if ((i + 1) % C != rank) thread_wait_row(&bbar[i + 1], abort_flag, status);
      s += nextp.dot(zt + (i + 1) * NB);
    }
    part[ch * NB + a] = s;
    __syncthreads();
    if (tid < NB) {
      T t = T(0);
#pragma unroll
      for (int c = 0; c < TP::CH; ++c) t += part[c * NB + tid];
      acc[tid] = y[i * NB + tid] - t;
    }
    __syncthreads();
    part[ch * NB + a] = wp.dot(acc);
    __syncthreads();
    {
      // the CH threads of column a form the same sum: each stores it into
      // every CH-th peer
      T w = T(0);
#pragma unroll
      for (int c = 0; c < TP::CH; ++c) w += part[c * NB + a];
      if (ch == 0) {
        zt[i * NB + a] = w;
        z[i * NB + a] = (double)w;
      }
      const uint32_t la = smem_u32(zt + i * NB + a), lb = smem_u32(&bbar[i]);
      for (int d = ch; d < C; d += TP::CH)
        if (d != rank) st_async_peer(map_to_rank(la, d), w, map_to_rank(lb, d));
    }
    __syncthreads();
  }
  // wait for every store addressed to this CTA before leaving (briefly when a
  // wait already ran out: the rows still missing will not come)
  const unsigned drain = ok ? kSpinLimit : (kSpinLimit >> 8);
  cluster_wait_rows(fbar, i0, Tt, C, rank, drain, abort_flag, status, &s_ok);
  cluster_wait_rows(bbar, 0, Tt, C, rank, drain, abort_flag, status, &s_ok);
  cl.sync();   // no CTA leaves while others may still store into its shared memory
}

template <typename T>
size_t solve_cluster_smem(int P, int Tt) {
  return 2 * (size_t)P * sizeof(T) + 2 * (size_t)Tt * sizeof(uint64_t);   // Tt >= super-rows
}

// Largest cluster (16, else 8) that fits the solve, or 0 when none does, or
// when the lower triangle of L is over half of L2 (64 MB): the cluster's 16
// SMs then stream L from DRAM at a fraction of its bandwidth, while the
// chained solve (a CTA per tile row across the GPU) folds with all SMs.
template <typename T, int NB>
int pick_solve_cluster(int P, int Tt) {
  constexpr int kMaxSmem = 200 * 1024;   // allowance set once for every plan
  constexpr size_t kMaxTriangle = 64u << 20;
  if ((size_t)P * P / 2 * sizeof(T) > kMaxTriangle) return 0;
  const size_t smem = solve_cluster_smem<T>(P, Tt);
  if (smem > (size_t)kMaxSmem) return 0;
  auto kern = chol_solve_cluster_kernel<T, NB>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const bool np = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess;
  cudaGetLastError();
  for (int C : {16, 8}) {
    if (C > 8 && !np) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = C;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) return C;
    cudaGetLastError();
  }
  return 0;
}

template <typename T, int NB>
cudaError_t launch_solve_cluster(const CholPlan& p, const void* L, const double* v, double* z,
                                 int* status, cudaStream_t s, int i0) {
  int* abort_flag = p.d_sync + p.T * p.T + 2 * p.T + 3;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.cluster);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = solve_cluster_smem<T>(p.P, p.T);
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = p.cluster;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, chol_solve_cluster_kernel<T, NB>, (const T*)L, p.P, p.T,
                            (const T*)p.d_winv, v, z, status, abort_flag, i0);
}

template <typename T, int NB>
size_t factor_smem() { return factor_smem_bytes<T>(NB); }

template <typename T, int NB>
cudaError_t launch_factor(const CholPlan& p, void* L, int* status, cudaStream_t s) {
  int* cnt = p.d_sync;
  int* ticket = p.d_sync + p.T * p.T + 2 * p.T;
  int* abort_flag = ticket + 3;
  if (p.wide)
    chol_factor_kernel<T, NB, kRegsWide><<<p.grid, kThreads, factor_smem<T, NB>(), s>>>(
        (T*)L, p.P, p.T, p.d_tasks, p.ntasks, cnt, ticket, (T*)p.d_winv, status, abort_flag);
  else
    chol_factor_kernel<T, NB, kRegsShared><<<p.grid, kThreads, factor_smem<T, NB>(), s>>>(
        (T*)L, p.P, p.T, p.d_tasks, p.ntasks, cnt, ticket, (T*)p.d_winv, status, abort_flag);
  return cudaGetLastError();
}

// opt in to the factor kernels' shared memory
template <typename T, int NB>
cudaError_t factor_smem_optin() {
  const int bytes = (int)factor_smem<T, NB>();
  cudaError_t e = cudaFuncSetAttribute(chol_factor_kernel<T, NB, kRegsWide>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_factor_kernel<T, NB, kRegsShared>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_factor_batch_kernel<T, NB, kRegsWide>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_factor_batch_kernel<T, NB, kRegsShared>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

template <typename T, int NB>
void launch_factor_batch(const CholBatch& b, int* ticket, int* abort_flag, cudaStream_t s) {
  if (b.wide)
    chol_factor_batch_kernel<T, NB, kRegsWide><<<b.grid, kThreads, factor_smem<T, NB>(), s>>>(
        b.d_jobs, b.d_queue, b.nqueue, ticket, abort_flag);
  else
    chol_factor_batch_kernel<T, NB, kRegsShared><<<b.grid, kThreads, factor_smem<T, NB>(), s>>>(
        b.d_jobs, b.d_queue, b.nqueue, ticket, abort_flag);
}

template <typename T, int NB>
cudaError_t launch_solve(const CholPlan& p, const void* L, const double* v, double* z,
                         int* status, cudaStream_t s) {
  int* fflag = p.d_sync + p.T * p.T;
  int* bflag = fflag + p.T;
  int* ticket = bflag + p.T;
  int* abort_flag = ticket + 3;
  int grid = p.T < p.grid ? p.T : p.grid;
  chol_fwd_kernel<T, NB><<<grid, kThreads, 0, s>>>((const T*)L, p.P, p.T, (const T*)p.d_winv, v,
                                                    (T*)p.d_y, fflag, ticket + 1, status,
                                                    abort_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  chol_bwd_kernel<T, NB><<<grid, kThreads, 0, s>>>((const T*)L, p.P, p.T, (const T*)p.d_winv,
                                                    (const T*)p.d_y, (T*)p.d_y + p.P, z, bflag,
                                                    ticket + 2, status, abort_flag);
  return cudaGetLastError();
}

}  // namespace

cudaError_t chol_batch_create(CholBatch* b, const std::vector<const CholPlan*>& plans,
                              const std::vector<void*>& Ls, const std::vector<int*>& statuses,
                              int num_sms, int ctas_per_sm) {
  *b = CholBatch{};
  if (plans.empty()) return cudaSuccess;
  b->is_f32 = plans[0]->is_f32;
  b->nb = plans[0]->nb;
  b->plans = plans;
  std::vector<FactorJob> jobs;
  struct Item { double key; int job, task; };
  std::vector<Item> items;
  for (size_t j = 0; j < plans.size(); ++j) {
    const CholPlan* p = plans[j];
    if (p->is_f32 != b->is_f32 || p->nb != b->nb) return cudaErrorInvalidValue;
    jobs.push_back(FactorJob{Ls[j], p->P, p->T, p->d_tasks, p->d_sync, p->d_winv, statuses[j]});
    for (int t = 0; t < p->ntasks; ++t)
      items.push_back(Item{(t + 0.5) / p->ntasks, (int)j, t});
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const Item& x, const Item& y) { return x.key < y.key; });
  std::vector<int2> queue(items.size());
  for (size_t q = 0; q < items.size(); ++q) queue[q] = make_int2(items[q].job, items[q].task);
  b->njobs = (int)jobs.size();
  b->nqueue = (int)queue.size();
  b->wide = ctas_per_sm <= 1;
  b->grid = num_sms * (b->wide ? 1 : ctas_per_sm);
  cudaError_t e = cudaMalloc(&b->d_jobs, jobs.size() * sizeof(FactorJob));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, queue.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ticket, 2 * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_jobs, jobs.data(), jobs.size() * sizeof(FactorJob), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_queue, queue.data(), queue.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  if (b->is_f32) return b->nb == 64 ? factor_smem_optin<float, 64>() : factor_smem_optin<float, 32>();
  return b->nb == 64 ? factor_smem_optin<double, 64>() : factor_smem_optin<double, 32>();
}

void chol_batch_destroy(CholBatch* b) {
  cudaFree(b->d_jobs);
  cudaFree(b->d_queue);
  cudaFree(b->d_ticket);
  *b = CholBatch{};
}

cudaError_t chol_factor_batch(const CholBatch& b, cudaStream_t s) {
  if (b.nqueue == 0) return cudaSuccess;
  cudaError_t e;
  // tile counters start at zero for every factorisation, and so do the
  // merged queue's ticket and abort flag
  for (const CholPlan* p : b.plans)
    if ((e = cudaMemsetAsync(p->d_sync, 0, chol_sync_words(p->T) * sizeof(int), s)) != cudaSuccess)
      return e;
  if ((e = cudaMemsetAsync(b.d_ticket, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
  int* ticket = b.d_ticket;
  int* abort_flag = b.d_ticket + 1;
  if (b.is_f32) {
    if (b.nb == 64) launch_factor_batch<float, 64>(b, ticket, abort_flag, s);
    else launch_factor_batch<float, 32>(b, ticket, abort_flag, s);
  } else {
    if (b.nb == 64) launch_factor_batch<double, 64>(b, ticket, abort_flag, s);
    else launch_factor_batch<double, 32>(b, ticket, abort_flag, s);
  }
  return cudaGetLastError();
}

cudaError_t chol_potrf_tile_prepare() {
  return cudaFuncSetAttribute(chol_potrf_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)factor_smem<float, 64>());
}

cudaError_t chol_potrf_tile(float* L, int P, int j, float* winv, int* status, cudaStream_t s) {
  chol_potrf_tile_kernel<<<1, kThreads, factor_smem<float, 64>(), s>>>(L, P, j, winv, status);
  return cudaGetLastError();
}

cudaError_t chol_plan_configure(CholPlan* plan, int P, int nb, int is_f32, int num_sms,
                                int ctas_per_sm, int wide) {
  *plan = CholPlan{};
  if (P % nb) return cudaErrorInvalidValue;
  plan->P = P;
  plan->nb = nb;
  plan->T = P / nb;
  plan->is_f32 = is_f32;
  plan->wide = wide < 0 ? (ctas_per_sm <= 1) : (wide != 0);
  plan->grid = (plan->wide ? 1 : ctas_per_sm) * num_sms;
  if (is_f32)
    plan->cluster = nb == 64 ? pick_solve_cluster<float, 64>(P, plan->T)
                             : pick_solve_cluster<float, 32>(P, plan->T);
  else
    plan->cluster = nb == 64 ? pick_solve_cluster<double, 64>(P, plan->T)
                             : pick_solve_cluster<double, 32>(P, plan->T);
  if (is_f32) return nb == 64 ? factor_smem_optin<float, 64>() : factor_smem_optin<float, 32>();
  return nb == 64 ? factor_smem_optin<double, 64>() : factor_smem_optin<double, 32>();
}

cudaError_t chol_plan_create(CholPlan* plan, int P, int nb, int is_f32, int num_sms,
                             int ctas_per_sm, int wide) {
  cudaError_t e = chol_plan_configure(plan, P, nb, is_f32, num_sms, ctas_per_sm, wide);
  if (e != cudaSuccess) return e;
  std::vector<CholTask> tasks = build_chol_tasks(plan->T, is_f32 && nb == 64);
  plan->ntasks = (int)tasks.size();
  size_t es = is_f32 ? sizeof(float) : sizeof(double);
  if ((e = cudaMalloc(&plan->d_tasks, tasks.size() * sizeof(CholTask))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(plan->d_tasks, tasks.data(), tasks.size() * sizeof(CholTask),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  size_t nsync = chol_sync_words(plan->T);
  if ((e = cudaMalloc(&plan->d_sync, nsync * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMemset(plan->d_sync, 0, nsync * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&plan->d_winv, (size_t)plan->T * nb * nb * es)) != cudaSuccess) return e;
  return cudaMalloc(&plan->d_y, 2 * (size_t)P * es);
}

void chol_plan_destroy(CholPlan* plan) {
  cudaFree(plan->d_tasks);
  cudaFree(plan->d_sync);
  cudaFree(plan->d_winv);
  cudaFree(plan->d_y);
  *plan = CholPlan{};
}

cudaError_t chol_factor(const CholPlan& p, void* L, int* status, cudaStream_t s) {
  // counters and tickets start at zero for every factorisation
  cudaError_t e = cudaMemsetAsync(p.d_sync, 0, chol_sync_words(p.T) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (p.is_f32) return p.nb == 64 ? launch_factor<float, 64>(p, L, status, s)
                                  : launch_factor<float, 32>(p, L, status, s);
  return p.nb == 64 ? launch_factor<double, 64>(p, L, status, s)
                    : launch_factor<double, 32>(p, L, status, s);
}

cudaError_t chol_solve(const CholPlan& p, const void* L, const double* v, double* z, int* status,
                       cudaStream_t s, int first_tile) {
  if (p.cluster) {
    const int i0 = std::max(0, std::min(first_tile, p.T - 1));
    if (p.is_f32) return p.nb == 64 ? launch_solve_cluster<float, 64>(p, L, v, z, status, s, i0)
                                    : launch_solve_cluster<float, 32>(p, L, v, z, status, s, i0);
    return p.nb == 64 ? launch_solve_cluster<double, 64>(p, L, v, z, status, s, i0)
                      : launch_solve_cluster<double, 32>(p, L, v, z, status, s, i0);
  }
  // reset the solve flags and tickets, keep the factor's abort flag
  int* fflag = p.d_sync + p.T * p.T;
  cudaError_t e = cudaMemsetAsync(fflag, 0, (2 * p.T + 3) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (p.is_f32) return p.nb == 64 ? launch_solve<float, 64>(p, L, v, z, status, s)
                                  : launch_solve<float, 32>(p, L, v, z, status, s);
  return p.nb == 64 ? launch_solve<double, 64>(p, L, v, z, status, s)
                    : launch_solve<double, 32>(p, L, v, z, status, s);
}

}  // namespace slim
