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

// CTA-wide bounded wait until *flag >= target.  Returns false if the wait ran
// out or another CTA asked everyone to stop.
__device__ bool cta_wait(const int* flag, int target, int* abort_flag, int* status, int* s_ok) {
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned it = 0;
    while (ld_acquire(flag) < target) {
      if (ld_acquire(abort_flag)) { ok = 0; break; }
      if (++it > kSpinLimit) {
        set_status(status, SLIM_ETIMEOUT);
        atomicExch(abort_flag, 1);
        ok = 0;
        break;
      }
      __nanosleep(40);
    }
    *s_ok = ok;
  }
  __syncthreads();
  int ok = *s_ok;
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ void cta_publish(int* flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add(flag, 1);
  }
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <typename T>
__device__ __forceinline__ void stcg(T* p, T v) { __stcg(p, v); }

// out = beta*C + sign * A B^T for NB x NB tiles (row-major, leading dimension
// ldA/ldB/ldC).  A and B are staged transposed (k-major) in shared memory.
template <typename T, int NB>
__device__ void tile_gemm_nt(T* out, const T* C, int ldC, const T* A, int ldA, const T* B, int ldB,
                             bool beta, T sign, T* As, T* Bs) {
  constexpr int LD = NB + 1;
  constexpr int TM = NB / 16;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += kThreads) {
    int r = idx / NB, q = idx % NB;
    As[q * LD + r] = ldcg(A + (size_t)r * ldA + q);
    Bs[q * LD + r] = ldcg(B + (size_t)r * ldB + q);
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  T acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
#pragma unroll 4
  for (int q = 0; q < NB; ++q) {
    T av[TM], bv[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) av[a] = As[q * LD + ty + 16 * a];
#pragma unroll
    for (int b = 0; b < TM; ++b) bv[b] = Bs[q * LD + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) {
      int r = ty + 16 * a, c = tx + 16 * b;
      T v = sign * acc[a][b];
      if (beta) v += ldcg(C + (size_t)r * ldC + c);
      stcg(out + (size_t)r * ldC + c, v);
    }
  __syncthreads();
}

// Factor the NB x NB diagonal tile at Lkk in place (lower triangle) and write
// its inverse (lower, zeros above) to W.  Non-positive pivots set SLIM_ENOTPD
// and are replaced by 1 so the factorisation still completes without NaNs.
template <typename T, int NB>
__device__ void tile_potrf(T* Lkk, int ld, T* W, T* S, T* Ls, int* status) {
  constexpr int LD = NB + 1;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += kThreads) {
    int r = idx / NB, c = idx % NB;
    S[r * LD + c] = ldcg(Lkk + (size_t)r * ld + c);
  }
  // right-looking elimination on the unscaled Schur complements:
  // S[i][q] -= S[i][c] S[q][c] / d_c for c < q <= i
  for (int c = 0; c < NB; ++c) {
    __syncthreads();
    T d = S[c * LD + c];
    if (!(d > T(0))) d = T(1);
    const T inv_d = T(1) / d;
    const int w = NB - c - 1;
    for (int idx = tid; idx < w * w; idx += kThreads) {
      int i = c + 1 + idx / w, q = c + 1 + idx % w;
      if (q <= i) S[i * LD + q] -= S[i * LD + c] * S[q * LD + c] * inv_d;
    }
  }
  __syncthreads();
  // scale the columns: L[c][c] = sqrt(d_c), L[i][c] = S[i][c] / sqrt(d_c)
  for (int idx = tid; idx < NB * NB; idx += kThreads) {
    int i = idx / NB, c = idx % NB;
    T d = S[c * LD + c];
    if (!(d > T(0))) {
      if (i == c) set_status(status, SLIM_ENOTPD);
      d = T(1);
    }
    T sd = sqrt(d);
    T v = (i == c) ? sd : (i > c ? S[i * LD + c] / sd : T(0));
    Ls[i * LD + c] = v;
  }
  __syncthreads();
  // inverse of the lower-triangular tile, one column per group of TPC lanes:
  // W[j][j] = 1/L[j][j];  W[i][j] = -(sum_{q=j}^{i-1} L[i][q] W[q][j]) / L[i][i]
  constexpr int TPC = kThreads / NB;
  const int j = tid / TPC, sub = tid % TPC;
  for (int i = 0; i < NB; ++i) {
    T s = T(0);
    if (i > j)
      for (int q = j + sub; q < i; q += TPC) s += Ls[i * LD + q] * S[q * LD + j];
    // every lane takes part in the reduction (groups of one warp differ in branch)
#pragma unroll
    for (int o = TPC / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPC);
    T v = (i < j) ? T(0) : (i == j ? T(1) / Ls[j * LD + j] : -s / Ls[i * LD + i]);
    __syncwarp();
    if (sub == 0) S[i * LD + j] = v;   // S now holds W column by column
    __syncwarp();
  }
  __syncthreads();
  for (int idx = tid; idx < NB * NB; idx += kThreads) {
    int r = idx / NB, c = idx % NB;
    stcg(Lkk + (size_t)r * ld + c, Ls[r * LD + c]);
    stcg(W + (size_t)r * NB + c, S[r * LD + c]);
  }
  __syncthreads();
}

template <typename T, int NB>
__global__ void __launch_bounds__(kThreads) chol_factor_kernel(T* L, int P, int Tt,
                                                               const CholTask* tasks, int ntasks,
                                                               int* cnt, int* ticket, T* winv,
                                                               int* status, int* abort_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);
  T* Bs = As + NB * (NB + 1);
  __shared__ int s_task, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= ntasks) return;
    const CholTask tk = tasks[t];
    const int i = tk.i, m = tk.m, k = tk.k;
    T* tile_im = L + (size_t)i * NB * P + (size_t)m * NB;
    if (tk.type == kUpd) {
      if (!cta_wait(&cnt[i * Tt + k], k + 1, abort_flag, status, &s_ok)) return;
      if (!cta_wait(&cnt[m * Tt + k], k + 1, abort_flag, status, &s_ok)) return;
      if (!cta_wait(&cnt[i * Tt + m], k, abort_flag, status, &s_ok)) return;
      const T* Lik = L + (size_t)i * NB * P + (size_t)k * NB;
      const T* Lmk = L + (size_t)m * NB * P + (size_t)k * NB;
      tile_gemm_nt<T, NB>(tile_im, tile_im, P, Lik, P, Lmk, P, true, T(-1), As, Bs);
      cta_publish(&cnt[i * Tt + m]);
    } else if (tk.type == kTrsm) {
      if (!cta_wait(&cnt[m * Tt + m], m + 1, abort_flag, status, &s_ok)) return;
      if (!cta_wait(&cnt[i * Tt + m], m, abort_flag, status, &s_ok)) return;
      const T* Wm = winv + (size_t)m * NB * NB;
      tile_gemm_nt<T, NB>(tile_im, nullptr, P, tile_im, P, Wm, NB, false, T(1), As, Bs);
      cta_publish(&cnt[i * Tt + m]);
    } else {
      if (!cta_wait(&cnt[k * Tt + k], k, abort_flag, status, &s_ok)) return;
      T* Lkk = L + (size_t)k * NB * P + (size_t)k * NB;
      tile_potrf<T, NB>(Lkk, P, winv + (size_t)k * NB * NB, As, Bs, status);
      cta_publish(&cnt[k * Tt + k]);
    }
  }
}

// out[r] = sign * sum_c M[r][c] v[c] (+ acc[r] if accumulate), one NB x NB tile;
// rows split over TPR lanes.  v and acc in shared memory.
template <typename T, int NB>
__device__ void tile_gemv(const T* M, int ld, const T* v, T* acc, T sign) {
  constexpr int TPR = kThreads / NB;
  constexpr int CPT = NB / TPR;
  const int r = threadIdx.x / TPR, sub = threadIdx.x % TPR;
  T s = T(0);
#pragma unroll 4
  for (int q = 0; q < CPT; ++q) {
    int c = sub * CPT + q;
    s += ldcg(M + (size_t)r * ld + c) * v[c];
  }
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
  __syncthreads();
  if (sub == 0) acc[r] += sign * s;
  __syncthreads();
}

// out[a] += sign * sum_c M[c][a] v[c]  (transposed tile), partial sums in `part`.
template <typename T, int NB>
__device__ void tile_gemv_t(const T* M, int ld, const T* v, T* acc, T sign, T* part) {
  constexpr int CH = kThreads / NB;
  constexpr int RPC = NB / CH;
  const int a = threadIdx.x % NB, ch = threadIdx.x / NB;
  T s = T(0);
#pragma unroll 4
  for (int q = 0; q < RPC; ++q) {
    int c = ch * RPC + q;
    s += ldcg(M + (size_t)c * ld + a) * v[c];
  }
  part[ch * NB + a] = s;
  __syncthreads();
  if (threadIdx.x < NB) {
    T t = T(0);
#pragma unroll
    for (int c = 0; c < CH; ++c) t += part[c * NB + threadIdx.x];
    acc[threadIdx.x] += sign * t;
  }
  __syncthreads();
}

template <typename T, int NB>
__global__ void __launch_bounds__(kThreads) chol_fwd_kernel(const T* L, int P, int Tt,
                                                            const T* winv, const double* v, T* y,
                                                            int* fflag, int* ticket, int* status,
                                                            int* abort_flag) {
  __shared__ T acc[NB], vec[NB], out[NB];
  __shared__ int s_task, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(ticket, 1);
    __syncthreads();
    const int i = s_task;
    __syncthreads();
    if (i >= Tt) return;
    if (threadIdx.x < NB) acc[threadIdx.x] = (T)v[i * NB + threadIdx.x];
    __syncthreads();
    for (int j = 0; j < i; ++j) {
      if (!cta_wait(&fflag[j], 1, abort_flag, status, &s_ok)) return;
      if (threadIdx.x < NB) vec[threadIdx.x] = ldcg(y + j * NB + threadIdx.x);
      __syncthreads();
      tile_gemv<T, NB>(L + (size_t)i * NB * P + (size_t)j * NB, P, vec, acc, T(-1));
    }
    if (threadIdx.x < NB) out[threadIdx.x] = T(0);
    __syncthreads();
    tile_gemv<T, NB>(winv + (size_t)i * NB * NB, NB, acc, out, T(1));
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
  __shared__ int s_task, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= Tt) return;
    const int i = Tt - 1 - t;
    if (threadIdx.x < NB) acc[threadIdx.x] = ldcg(y + i * NB + threadIdx.x);
    __syncthreads();
    for (int j = Tt - 1; j > i; --j) {
      if (!cta_wait(&bflag[j], 1, abort_flag, status, &s_ok)) return;
      if (threadIdx.x < NB) vec[threadIdx.x] = ldcg(zt + j * NB + threadIdx.x);
      __syncthreads();
      tile_gemv_t<T, NB>(L + (size_t)j * NB * P + (size_t)i * NB, P, vec, acc, T(-1), part);
    }
    if (threadIdx.x < NB) out[threadIdx.x] = T(0);
    __syncthreads();
    tile_gemv_t<T, NB>(winv + (size_t)i * NB * NB, NB, acc, out, T(1), part);
    if (threadIdx.x < NB) {
      stcg(zt + i * NB + threadIdx.x, out[threadIdx.x]);
      z[i * NB + threadIdx.x] = (double)out[threadIdx.x];
    }
    cta_publish(&bflag[i]);
  }
}

template <typename T, int NB>
size_t factor_smem() { return 2 * NB * (NB + 1) * sizeof(T); }

template <typename T, int NB>
cudaError_t launch_factor(const CholPlan& p, void* L, int* status, cudaStream_t s) {
  int* cnt = p.d_sync;
  int* ticket = p.d_sync + p.T * p.T + 2 * p.T;
  int* abort_flag = ticket + 3;
  chol_factor_kernel<T, NB><<<p.grid, kThreads, factor_smem<T, NB>(), s>>>(
      (T*)L, p.P, p.T, p.d_tasks, p.ntasks, cnt, ticket, (T*)p.d_winv, status, abort_flag);
  return cudaGetLastError();
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

std::vector<CholTask> build_chol_tasks(int T) {
  std::vector<CholTask> t;
  for (int k = 0; k < T; ++k) {
    t.push_back({kPotrf, (uint16_t)k, (uint16_t)k, (uint16_t)k});
    for (int i = k + 1; i < T; ++i) t.push_back({kTrsm, (uint16_t)i, (uint16_t)k, (uint16_t)k});
    // updates from panel k; column k+1 first so the next panel can start early
    for (int m = k + 1; m < T; ++m)
      for (int i = m; i < T; ++i) t.push_back({kUpd, (uint16_t)i, (uint16_t)m, (uint16_t)k});
  }
  return t;
}

cudaError_t chol_plan_create(CholPlan* plan, int P, int nb, int is_f32, int num_sms) {
  *plan = CholPlan{};
  if (P % nb) return cudaErrorInvalidValue;
  plan->P = P;
  plan->nb = nb;
  plan->T = P / nb;
  plan->is_f32 = is_f32;
  std::vector<CholTask> tasks = build_chol_tasks(plan->T);
  plan->ntasks = (int)tasks.size();
  size_t es = is_f32 ? sizeof(float) : sizeof(double);
  cudaError_t e;
  if ((e = cudaMalloc(&plan->d_tasks, tasks.size() * sizeof(CholTask))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(plan->d_tasks, tasks.data(), tasks.size() * sizeof(CholTask),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  size_t nsync = (size_t)plan->T * plan->T + 2 * plan->T + 4;
  if ((e = cudaMalloc(&plan->d_sync, nsync * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMemset(plan->d_sync, 0, nsync * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&plan->d_winv, (size_t)plan->T * nb * nb * es)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&plan->d_y, 2 * (size_t)P * es)) != cudaSuccess) return e;
  plan->grid = 2 * num_sms;
  // opt in to the shared memory the factor kernel needs
  if (is_f32) {
    if (nb == 64)
      e = cudaFuncSetAttribute(chol_factor_kernel<float, 64>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)factor_smem<float, 64>());
    else
      e = cudaFuncSetAttribute(chol_factor_kernel<float, 32>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)factor_smem<float, 32>());
  } else {
    if (nb == 64)
      e = cudaFuncSetAttribute(chol_factor_kernel<double, 64>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)factor_smem<double, 64>());
    else
      e = cudaFuncSetAttribute(chol_factor_kernel<double, 32>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)factor_smem<double, 32>());
  }
  return e;
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
  size_t nsync = (size_t)p.T * p.T + 2 * p.T + 4;
  cudaError_t e = cudaMemsetAsync(p.d_sync, 0, nsync * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (p.is_f32) return p.nb == 64 ? launch_factor<float, 64>(p, L, status, s)
                                  : launch_factor<float, 32>(p, L, status, s);
  return p.nb == 64 ? launch_factor<double, 64>(p, L, status, s)
                    : launch_factor<double, 32>(p, L, status, s);
}

cudaError_t chol_solve(const CholPlan& p, const void* L, const double* v, double* z, int* status,
                       cudaStream_t s) {
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
