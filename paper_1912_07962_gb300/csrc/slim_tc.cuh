// Float32-accurate matrix products on the Blackwell tensor cores (tcgen05),
// and the triangular inverse built on them.
//
// A float32 operand x enters as three bfloat16 terms x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1), which carry its 24 significant
// bits.  A product a b is accumulated as the six term products a_i b_j with
// i + j <= 2 (the dropped ones are below 2^-24 relative), each a tcgen05.mma
// of kind f16 (bfloat16 inputs, float32 accumulator in tensor memory).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "slim_lookahead.cuh"

namespace slim {

// One product of a batched launch: C = alpha op(A) op(B) + beta C, op(A) M x K,
// op(B) K x N, float32 in global memory.
struct TcProblem {
  const float* A;
  long long lda;     // a_km = 0: op(A)[m][k] = A[m*lda + k]; 1: A[k*lda + m]
  const float* B;
  long long ldb;     // b_kn = 0: op(B)[k][n] = B[n*ldb + k]; 1: B[k*ldb + n]
  float* C;
  long long ldc;     // c_nm = 0: C[m*ldc + n]; 1: C[n*ldc + m]
  int M, N, K;       // K a multiple of 64
  int a_km, b_kn, c_nm;
  int k_from_n;      // op(B) lower triangular (op(B)[k][n] = 0 for k < n; whatever the storage
                     // holds there is read as zero): an output tile's K loop starts at its first column
  int k_to_m;        // op(A) lower triangular (op(A)[m][k] = 0 for k > m, likewise masked): an
                     // output tile's K loop ends after its last row
  float alpha, beta; // beta = 0: C is not read
  int c_lower;       // 1: only output tiles that reach the lower triangle (some n <= m) are
                     // computed; tiles wholly above the diagonal are left alone
  // tc_gemm_planes only: op(A) and op(B)^T split in advance by tc_split (A and
  // B are then not read; the masks were applied by the split)
  const unsigned char* a_planes;
  const unsigned char* b_planes;
};

constexpr int kTcBM = 128;   // output rows per CTA (the MMA's M)
constexpr int kTcBN = 128;   // output columns per CTA (the MMA's N), wide tile
constexpr int kTcBNNarrow = 64;   // narrow tile, for products with few wide tiles
constexpr int kTcBK = 64;    // K per pipeline stage (128-byte bfloat16 rows)

// Launch the products probs[0..nprob) (a device array) with a grid covering
// max_m x max_n outputs; CTAs beyond a problem's own M x N return at once.
// A bounded wait that runs out records SLIM_ETIMEOUT in *status.
cudaError_t tc_gemm(const TcProblem* d_probs, int nprob, int max_m, int max_n, int* status,
                    cudaStream_t s);
// The same products from operands split in advance.  An operand op(X),
// rows x K, is stored as "planes": 128-row x 64-k tiles, each of its three
// bfloat16 term tiles the exact 16 KB image of the 128-byte-swizzled K-major
// shared-memory layout the MMA reads, the three terms of a tile consecutive
// (48 KB).  Tile (rt, kt) starts at byte (rt * (K / 64) + kt) * 49152; rows
// at or beyond `rows` are zero.  Each CTA then streams its tiles with bulk
// copies (cp.async.bulk into a ring of shared-memory stages, one producer
// thread, one MMA thread), so splitting costs one pass over each operand
// instead of one per tile of C.
struct TcSplitJob {
  const float* X;
  long long ld;      // km = 0: op(X)[r][k] = X[r*ld + k] (16-byte aligned rows); 1: X[k*ld + r]
  int km;
  int rows, K;       // K a multiple of 64
  int tri;           // 1: op(X)[r][k] read as zero for k > r; 2: for k < r (the tiles wholly
                     // in the zero triangle are not written: the products never read them)
  unsigned char* planes;
};
size_t tc_plane_bytes(int rows, int K);
// The split jobs of op(A) and op(B)^T of problem p, planes at a and b.
TcSplitJob tc_split_job_a(const TcProblem& p, unsigned char* a);
TcSplitJob tc_split_job_b(const TcProblem& p, unsigned char* b);
// Split jobs[0..njobs) (a device array); max_tiles = the largest
// ceil(rows / 128) * (K / 64) among them.
cudaError_t tc_split(const TcSplitJob* d_jobs, int njobs, int max_tiles, cudaStream_t s);
cudaError_t tc_gemm_planes(const TcProblem* d_probs, int nprob, int max_m, int max_n,
                           int* status, cudaStream_t s);

// Dynamic shared memory of one wide-tile CTA (both tile widths are opted in by
// tc_prepare, once per process).
size_t tc_smem_bytes();
cudaError_t tc_prepare();

// Inverse of a lower-triangular factor L (P x P row-major float32, P = T nb,
// nb = 64) whose diagonal tiles' inverses W_j are given (T tiles of 64 x 64,
// row-major, zero above the diagonal): X = L^{-1} in the lower triangle of the
// P x P buffer X (diagonal included) and X^T in its strict upper triangle.
// The recursion splits the tile range [a, b) at m = (a + b) / 2:
//   X11 = inv(L11), X22 = inv(L22),  X21 = -X22 (L21 X11),
// all blocks of one recursion depth in one batched launch per product (a
// split pass of its operands, then tc_gemm_planes); the intermediate L21 X11
// is held, transposed, in X's upper triangle.
struct TriInvPlan {
  int P = 0, T = 0;
  std::vector<int> level_first;       // problems of depth d: [level_first[d], level_first[d+1])
  std::vector<int> level_max_m, level_max_n;
  TcProblem* d_probs = nullptr;       // 2 per split: (L21 X11) and (-X22 T1)
  int nprob = 0;
  // the operands of each batched launch, split into planes just before it
  std::vector<int> job_first, job_max_tiles;   // jobs of launch l: [job_first[l], job_first[l+1])
  TcSplitJob* d_jobs = nullptr;
  unsigned char* d_planes = nullptr;           // scratch, shared by the launches in turn
};
// Plan for order P; L, W and X are bound now (the plan's problems point at them).
cudaError_t tri_inverse_plan(TriInvPlan* plan, int P, const float* L, const float* W, float* X);
void tri_inverse_plan_destroy(TriInvPlan* plan);
cudaError_t tri_inverse(const TriInvPlan& plan, const float* W, float* X, int* status,
                        cudaStream_t s);

// Right-looking blocked Cholesky of the float32 matrix L (P x P row-major, its
// lower triangle, P = 64 T) with one launch per step of each 64-wide panel j:
//   diagonal tile:  L_jj = chol(A_jj), W_j = L_jj^{-1}     (one CTA, SIMT)
//   panel:          L_ij = A_ij W_j^T for all i > j      (one tensor-core product, in place)
//   trailing:       A_il -= L_ij L_lj^T for all i >= l > j (one tensor-core product, the
//                   tiles that reach the lower triangle)
// The factor replaces L's lower triangle; W goes to winv (T tiles of 64 x 64).
// Entries above the diagonal of L's tiles are work space.
struct TcCholPlan {
  int P = 0, T = 0;
  TcProblem* d_probs = nullptr;       // 2 per panel: the panel's TRSM and its trailing update
};
cudaError_t tc_chol_plan(TcCholPlan* plan, int P, float* L, const float* winv);
void tc_chol_plan_destroy(TcCholPlan* plan);
cudaError_t tc_cholesky(const TcCholPlan& plan, float* L, float* winv, int* status,
                        cudaStream_t s);

// Matrix-vector products with the triangular inverse held as above (lower: X,
// strict upper: X^T), rows and columns in [0, p):
//   y[i]  = sum_{j = lo..i} X[i][j] v[j]        for i in [lo, p)   (trinv_lower)
//   z[j] (+)= sum_{i = max(j, lo)..p-1} X[i][j] y[i]   for j in [0, p)   (trinv_upper)
// lo: v is zero below index lo (the right-hand side's first nonzero row), so y
// is zero there too.  float32 products, float64 sums across the row.
cudaError_t trinv_lower(const float* X, int P, int p, int lo, const double* v, double* y,
                        cudaStream_t s);
cudaError_t trinv_upper(const float* X, int P, int p, int lo, const double* y, double* z,
                        int accumulate, cudaStream_t s);

// The iterate chain of the pipelined tensor-core form for step `info` (plain
// slimLS: no slimTik terms; C_k may be diagonal) as one cooperative launch of
// `grid` CTAs: r_k into rhs, z = X^T X rhs, `refine` rounds of
// res = rhs - lambda_k z - G z (float64) and z += X^T X res, then
// x -= eta M_k^T z.  y and res are work vectors of P doubles; bar two
// unsigned ints (zeroed here).  A grid barrier that runs out records
// SLIM_ETIMEOUT.  iterate_tc_prepare opts in to the shared memory for order P
// and gives the grid (at most kIterTcCtas CTAs, one per SM of a GB300, all co-resident).
constexpr int kIterTcCtas = 152;
size_t iterate_tc_smem(int P);
template <typename T>
cudaError_t iterate_tc_prepare(int P, int num_sms, int* grid);
template <typename T>
cudaError_t iterate_tc(const LaArgs<T>& a, const StepInfo* info, const int* ext, const float* X,
                       double* y, double* res, unsigned* bar, int refine, int grid,
                       cudaStream_t s);

}  // namespace slim
