// C ABI of libslim.so: context management and the step driver.
#include <cmath>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/slim.h"
#include "slim_chol.cuh"
#include "slim_kernels.cuh"
#include "slim_lookahead.cuh"
#include "slim_lsqr.cuh"
#include "slim_olbfgs.cuh"
#include "slim_frames.cuh"
#include "slim_unet.cuh"
#include "slim_rays.cuh"
#include "slim_tc.cuh"
#include "slim_tikl.cuh"

using namespace slim;

constexpr int kMaxBuf = 11;   // lookahead D <= 10: D+1 factor buffers

struct slim_ctx {
  // configuration
  int N = 0, n_views = 0, D = 0;
  long long n = 0, m = 0;
  int precision = SLIM_PREC_FP64, solver = SLIM_SOLVE_FP64, refine_iters = 2, use_graph = 0;
  int a_mode = 0;                 // 0 rows from the projector, 1/2 stored float32/bfloat16 rows
  CsrStore csr;
  int dim = 2, Dv = 1, kind = SLIM_BLOCKS_VIEWS, steps_per_view = 1;
  int S = 0, cap = 0;             // 3D: slices and the largest slice block solved
  int* d_slice_cnt = nullptr;
  int* d_slice_rows = nullptr;
  int ramp = 0, r = 0, nslots = 1, ell = 0, p = 0, P = 0, taps = 0, nb = 32;
  int decay_after = 0;             // 1/k decay of the damping after this step (0: none)
  int tile = 0, ctas_per_sm = 1;
  int cps_auto = 1;   // ctas_per_sm left to the library (0 in the step options)
  double lam = 0.0, eta = 1.0;
  unsigned long long seed = 0;
  std::vector<ViewGeom> h_views;
  // device state
  ViewGeom* d_views = nullptr;
  StepInfo* d_info = nullptr;
  long long* d_done = nullptr;
  int* d_status = nullptr;
  void* d_x = nullptr;
  void* d_b = nullptr;
  int* d_ring_ids = nullptr;
  int* d_ring_pix = nullptr;
  double* d_ring_w = nullptr;
  int* d_map_ray = nullptr;
  double* d_map_w = nullptr;
  double* d_G = nullptr;
  void* d_L = nullptr;
  double* d_rhs = nullptr;
  double* d_z = nullptr;
  double* d_dz = nullptr;
  int lsqr_max_iter = 0;
  double lsqr_tol = 0.0;
  double tik_lambda = 0.0;         // slimTik: lam_tik of Eq. (TLS1) (0: slimLS)
  int tik_reading = 0;             // count of Tikhonov rows: 0 blocks of M_k, 1 r
  double* d_cinv = nullptr;        // [n] 1/c of C_k = diag(c); null: C_k = I
  // slimTik with a lower-bidiagonal L (slim_set_tik_bidiag); null: C_k = I or diagonal
  double* d_tl_d0inv = nullptr;    // [n] 1 / d0
  double* d_tl_d1 = nullptr;       // [n]
  double* d_tl_U = nullptr;        // [ell * n] W a_i^T of the new block's rows
  double* d_tl_UT = nullptr;       // [n * ell]
  double* d_tl_v = nullptr;        // [n]
  // capture stage of a batch step: 0 the whole step; 1 up to K = lambda I + G
  // (the batch factors every problem in one merged launch); 2 from the
  // solves on
  int stage = 0;
  int cyclic = 0;                  // view blocks in the random cyclic order
  int distinct = 0;                // random-ray blocks of distinct rays (Floyd)
  int* d_perm = nullptr;           // [n_views] the current epoch's permutation (cyclic)
  long long* d_perm_epoch = nullptr;
  double* d_cinvh = nullptr;       // [n] c^{-1/2} (the LSQR form's column scaling)
  // 3D with random view directions (frames given): general Joseph rows, Gram
  // from voxel lists, the tiled dense solve
  bool general3d = false;
  std::vector<FrameGeom> h_frames;
  FrameGeom* d_frames = nullptr;
  int* d_vnext = nullptr;          // [ell * taps] voxel-list links of the new block
  int olbfgs_memory = 0;           // pairs of the olbfgs comparator
  int ray_lanes = 32;              // threads per ray: random-ray march and scatter
  int pair_window = 32;            // pair Gram: longer windows go to the whole warp
  double* d_olb = nullptr;         // its scratch: g, S, Y, u, S^T Y, Y^T Y, partial sums
  int* d_olb_state = nullptr;      // its pair bookkeeping
  double* d_lsqr = nullptr;        // LSQR scratch: u [p], v, w, s, tmp [n], partial sums, stats [3]
  unsigned* d_lsqr_bar = nullptr;  // its grid barrier
  double* d_res = nullptr;
  double* d_ref = nullptr;
  double* d_err = nullptr;
  CholPlan plan;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool has_data = false;
  long long h_k = 0;
  int num_sms = 0;
  bool timing = false;
  bool capturing = false;
  cudaEvent_t ev[8] = {};
  // pipelined form (lookahead D > 0): geometry chain D steps ahead
  int lookahead = 0, eslots = 0, Pe = 0, nbuf = 1;
  long long h_g = 0;                 // geometry steps enqueued
  long long* d_gdone = nullptr;      // geometry steps prepared (device)
  StepInfo* d_info_buf = nullptr;    // [nbuf]
  int* d_ext = nullptr;              // [nbuf * P] ring index -> extended row
  void* d_Lb[kMaxBuf] = {};
  CholPlan planb[kMaxBuf];
  // SLIM_SOLVE_MIXED_TC: X = L^{-1} per buffer (X^T in its upper triangle)
  void* d_Xb[kMaxBuf] = {};
  TriInvPlan tplan[kMaxBuf];
  TcCholPlan cplan[kMaxBuf];         // launch-per-panel tensor-core factorisation
  double* d_ty = nullptr;            // [P] intermediate of the products with X
  unsigned* d_coop_bar = nullptr;    // grid barrier of the cooperative iterate chain
  int coop_grid = 0;                 // its CTAs (0: the chain runs kernel by kernel)
  cudaStream_t xs = nullptr, gs = nullptr, fs[kMaxBuf] = {};
  cudaGraphExec_t g1_exec[kMaxBuf] = {}, g2_exec[kMaxBuf] = {}, gx_exec[kMaxBuf] = {};
  cudaEvent_t ev_user = nullptr, ev_g1 = nullptr, ev_g2[kMaxBuf] = {}, ev_x[kMaxBuf] = {};
  cudaEvent_t la_ev[10] = {};
  // launch log (timing on): event pairs around factor and iterate launches
  static constexpr int kLog = 512;
  std::vector<cudaEvent_t> log_f, log_x;   // 2*kLog each
  long long log_nf = 0, log_nx = 0, log_f0 = 0, log_x0 = 0;
  std::string err;
};

namespace {

size_t elem(int precision) { return precision == SLIM_PREC_FP32 ? sizeof(float) : sizeof(double); }

slim_status fail(slim_ctx* c, slim_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

slim_status cuda_fail(slim_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  if (c) c->err = m;
  return e == cudaErrorMemoryAllocation ? SLIM_ENOMEM : SLIM_ECUDA;
}

#define CK(call, where)                                    \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

template <typename TI, typename TO>
__global__ void convert_kernel(const TI* in, TO* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

// Copy n values of dtype `src_dtype` (host or device) into a device array of
// precision `dst_prec`, converting if needed.
cudaError_t copy_in(void* dst, int dst_f32, const void* src, int src_dtype, int on_device,
                    long long n, cudaStream_t s) {
  const bool same = (src_dtype == SLIM_F32) == (dst_f32 != 0);
  const size_t sb = src_dtype == SLIM_F32 ? 4 : 8;
  if (same)
    return cudaMemcpyAsync(dst, src, n * sb, on_device ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice, s);
  const void* dsrc = src;
  void* tmp = nullptr;
  cudaError_t e;
  if (!on_device) {
    if ((e = cudaMallocAsync(&tmp, n * sb, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(tmp, src, n * sb, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    dsrc = tmp;
  }
  int grid = (int)std::min<long long>((n + 255) / 256, 4096);
  if (grid < 1) grid = 1;
  if (src_dtype == SLIM_F32)
    convert_kernel<float, double><<<grid, 256, 0, s>>>((const float*)dsrc, (double*)dst, n);
  else
    convert_kernel<double, float><<<grid, 256, 0, s>>>((const double*)dsrc, (float*)dst, n);
  e = cudaGetLastError();
  if (tmp) cudaFreeAsync(tmp, s);
  return e;
}

cudaError_t copy_out(void* dst, int dst_dtype, int on_device, const void* src, int src_f32,
                     long long n, cudaStream_t s) {
  const bool same = (dst_dtype == SLIM_F32) == (src_f32 != 0);
  const size_t db = dst_dtype == SLIM_F32 ? 4 : 8;
  if (same) {
    cudaError_t e = cudaMemcpyAsync(dst, src, n * db, on_device ? cudaMemcpyDeviceToDevice
                                                                : cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
  }
  void* ddst = dst;
  void* tmp = nullptr;
  cudaError_t e;
  if (!on_device) {
    if ((e = cudaMallocAsync(&tmp, n * db, s)) != cudaSuccess) return e;
    ddst = tmp;
  }
  int grid = (int)std::min<long long>((n + 255) / 256, 4096);
  if (grid < 1) grid = 1;
  if (src_f32)
    convert_kernel<float, double><<<grid, 256, 0, s>>>((const float*)src, (double*)ddst, n);
  else
    convert_kernel<double, float><<<grid, 256, 0, s>>>((const double*)src, (float*)ddst, n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (tmp) {
    if ((e = cudaMemcpyAsync(dst, tmp, n * db, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    cudaFreeAsync(tmp, s);
  }
  return cudaStreamSynchronize(s);
}

template <typename T>
StepArgs<T> make_args(slim_ctx* c) {
  StepArgs<T> a;
  a.info = c->d_info;
  a.done = c->d_done;
  a.views = c->d_views;
  a.N = c->N;
  a.D = c->D;
  a.n_views = c->n_views;
  a.n = c->n;
  a.m = c->m;
  a.ell = c->ell;
  a.nslots = c->nslots;
  a.r = c->r;
  a.P = c->P;
  a.p = c->p;
  a.taps = c->taps;
  a.seed = c->seed;
  a.lam = c->lam;
  a.eta = c->eta;
  a.ramp = c->ramp;
  a.decay_after = c->decay_after;
  a.ring_ids = c->d_ring_ids;
  a.ring_pix = c->d_ring_pix;
  a.ring_w = c->d_ring_w;
  a.map_ray = c->d_map_ray;
  a.map_w = c->d_map_w;
  a.G = c->d_G;
  a.rhs = c->d_rhs;
  a.z = c->d_z;
  a.x = (T*)c->d_x;
  a.b = (const T*)c->d_b;
  a.status = c->d_status;
  a.csr_ptr = c->a_mode ? c->csr.row_ptr : nullptr;
  a.csr_col = c->a_mode ? c->csr.col : nullptr;
  a.csr_val = c->a_mode ? c->csr.val : nullptr;
  a.csr_bf16 = c->csr.bf16;
  a.tik_beta = c->tik_lambda * c->tik_lambda / c->n_views;   // M = A_v view blocks
  a.tik_reading = c->tik_reading;
  a.cinv = c->d_cinv;
  a.sg = c->solver == SLIM_SOLVE_SG;
  a.lanes = c->kind == SLIM_BLOCKS_VIEWS ? 32 : c->ray_lanes;
  a.cyclic = c->cyclic;
  a.perm = c->d_perm;
  a.perm_epoch = c->d_perm_epoch;
  return a;
}

RayArgs make_ray_args(slim_ctx* c) {
  RayArgs a;
  a.info = c->d_info;
  a.done = c->d_done;
  a.views = c->d_views;
  a.N = c->N;
  a.Du = c->D;
  a.Dv = c->Dv;
  a.n_views = c->n_views;
  a.dim = c->dim;
  a.n = c->n;
  a.m = c->m;
  a.ell = c->ell;
  a.nslots = c->nslots;
  a.r = c->r;
  a.p = c->p;
  a.taps = c->taps;
  a.magic_n = c->N > 1 ? (unsigned)((0x100000000ull + c->N - 1) / c->N) : 0xFFFFFFFFu;
  a.lanes = c->ray_lanes;
  a.short_window = c->pair_window;
  a.kind = c->kind;
  a.steps_per_view = c->steps_per_view;
  a.seed = c->seed;
  a.lam = c->lam;
  a.ramp = c->ramp;
  a.decay_after = c->decay_after;
  a.ring_ids = c->d_ring_ids;
  a.ring_pix = c->d_ring_pix;
  a.ring_w = c->d_ring_w;
  a.rhs = c->d_rhs;
  a.z = c->d_z;
  a.status = c->d_status;
  a.G = c->d_G;
  a.P = c->P;
  a.S = c->S;
  a.cap = c->cap;
  a.slice_cnt = c->d_slice_cnt;
  a.slice_rows = c->d_slice_rows;
  a.dense = c->dim == 2 || c->general3d;
  a.distinct = c->distinct;
  return a;
}

// Phase boundaries recorded when timing is on (event i closes phase i-1).
enum { kPhSample = 1, kPhForward, kPhGram, kPhFormK, kPhFactor, kPhSolve, kPhScatter };

// External event records stay real event records inside a captured graph, so
// they can be timed with cudaEventElapsedTime after each replay.
cudaError_t mark(slim_ctx* c, int i) {
  if (!c->timing) return cudaSuccess;
  if (c->capturing) return cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal);
  return cudaEventRecord(c->ev[i], c->stream);
}

// Float32 factor with float64-residual refinement (solved through the
// factor, or through its tensor-core inverse).
// CTAs per SM of the plain form's persistent factorisation.  Left to the
// library: one CTA per SM with the whole register file for float32 factors of
// up to 96 tiles a side (latency-bound: the chain of diagonal tiles decides);
// two at 128 registers for float64 factors and larger ones, which are bound by
// their arithmetic and gain from more tasks in flight (measured: p = 2178
// float64 5.6 ms against 6.0; p = 10240 float32 14.8 ms against 18.6; p = 2178
// float32 0.66 ms against 1.02).
inline int plan_ctas_per_sm(const slim_ctx* c) {
  if (!c->cps_auto) return c->ctas_per_sm;
  return (c->solver == SLIM_SOLVE_FP64 || c->P / c->nb > 96) ? 2 : 1;
}

// the pipelined forms whose iterate chain solves through X = L^{-1}
inline bool uses_inverse(const slim_ctx* c) {
  return c->solver == SLIM_SOLVE_MIXED_TC || c->solver == SLIM_SOLVE_MIXED_INV;
}

inline bool is_mixed(const slim_ctx* c) {
  return c->solver == SLIM_SOLVE_MIXED || uses_inverse(c);
}

// Kernels one step launches (sample, forward, Gram, K, factor, the solves:
// one cluster kernel each, else a forward and a backward kernel; 2 per
// refinement round (residual, z += dz), scatter).
int kernels_per_step(const slim_ctx* c) {
  if (c->dim == 3 && !c->general3d) return 6;   // sample, march, collect, slice Gram, slice solve, scatter
  if (c->solver == SLIM_SOLVE_LSQR)   // sample, forward + residual, (slimTik rhs,) LSQR with x update
    return c->tik_lambda > 0.0 ? 4 : 3;
  if (c->solver == SLIM_SOLVE_SG) return 3;     // sample, forward + residual, scatter
  if (c->solver == SLIM_SOLVE_OLBFGS) return 3; // sample, forward + residual, the olbfgs step
  const int solves = is_mixed(c) ? 1 + c->refine_iters : 1;
  const int refine = is_mixed(c) ? 2 * c->refine_iters : 0;
  if (c->lookahead && uses_inverse(c)) {
    // geometry: sample, taps, Gram, map clear, ring map, K; the factor (per
    // panel: diagonal tile, panel product, trailing product; the last panel
    // its diagonal tile only -- or one persistent launch), the inverse
    // (diagonal tiles; per recursion depth and side a split pass of the
    // operands and one product; mirror);
    // iterate: residual, 2 products per solve, a residual per refinement
    // round, scatter -- or all of the iterate chain in one cooperative kernel
    const int factor = c->solver == SLIM_SOLVE_MIXED_TC ? 3 * c->cplan[0].T - 2 : 1;
    const int inv = 2 + 2 * ((int)c->tplan[0].level_first.size() - 1);
    const int tik = c->tik_lambda > 0.0 ? 2 : 0;
    const int iterate = c->coop_grid ? 1 : 1 + 2 * solves + c->refine_iters + 1 + tik;
    return 6 + factor + inv + iterate;
  }
  if (c->lookahead) {
    // geometry: sample, taps, Gram, map clear, ring map, K, factor; iterate:
    // residual, the solves, refinement rounds, scatter
    const int per_solve = c->planb[0].cluster ? 1 : 2;
    const int tik = c->tik_lambda > 0.0 ? 2 : 0;   // window projection, x scale
    return 7 + 1 + per_solve * solves + refine + 1 + tik;
  }
  const int per_solve = c->plan.cluster ? 1 : 2;
  const int tik = c->tik_lambda > 0.0 ? 2 : 0;   // window projection, x scale
  const int mirror = c->general3d ? 1 : 0;       // the Gram's mirrored block
  // bidiagonal L: the Gram is rows W a_i, a transpose and the products (3);
  // the update M^T z, W v and the axpy (3) instead of the scatter
  const int tikl = c->d_tl_d0inv ? 4 : 0;
  return 5 + per_solve * solves + refine + 1 + tik + mirror + tikl;
}

// The damped solve (lambda_k I + G) z = rhs: float64 tiled Cholesky, or a
// float32 factor refined with float64 residuals.
cudaError_t enqueue_solve(slim_ctx* c) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  if (c->stage != 2) {
    e = c->solver == SLIM_SOLVE_FP64
            ? launch_form_k<double>(c->d_info, c->d_G, (double*)c->d_L, c->P, s)
            : launch_form_k<float>(c->d_info, c->d_G, (float*)c->d_L, c->P, s);
    if (e != cudaSuccess) return e;
    if ((e = mark(c, kPhFormK)) != cudaSuccess) return e;
  }
  if (c->stage == 1) return cudaSuccess;   // the batch factors between its stages
  if (c->stage == 0 && (e = chol_factor(c->plan, c->d_L, c->d_status, s)) != cudaSuccess) return e;
  if ((e = mark(c, kPhFactor)) != cudaSuccess) return e;
  if (c->solver == SLIM_SOLVE_FP64)
    return chol_solve(c->plan, c->d_L, c->d_rhs, c->d_z, c->d_status, s);
  if ((e = chol_solve(c->plan, c->d_L, c->d_rhs, c->d_z, c->d_status, s)) != cudaSuccess) return e;
  for (int it = 0; it < c->refine_iters; ++it) {
    if ((e = launch_refine_residual(c->d_info, c->d_G, c->d_z, c->d_rhs, c->d_res, c->P, s)) !=
        cudaSuccess)
      return e;
    if ((e = chol_solve(c->plan, c->d_L, c->d_res, c->d_dz, c->d_status, s)) != cudaSuccess)
      return e;
    if ((e = launch_axpy(c->d_z, c->d_dz, c->P, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// A step with random-ray blocks: 2D forms the dense Gram from pair overlaps
// and uses the tiled solve; 3D solves slice by slice.
template <typename T>
cudaError_t enqueue_ray_step_t(slim_ctx* c) {
  RayArgs ra = make_ray_args(c);
  StepArgs<T> a = make_args<T>(c);
  a.map_ray = nullptr;
  cudaStream_t s = c->stream;
  cudaError_t e;
  if (c->stage == 2) {   // a batch's second stage: the part after the factor
    if (c->dim == 3 && !c->general3d) return cudaSuccess;   // no tiled factor: all in stage 1
    if (c->general3d) a.map_ray = c->d_map_ray;
    if ((e = enqueue_solve(c)) != cudaSuccess) return e;
    if ((e = mark(c, kPhSolve)) != cudaSuccess) return e;
    if ((e = launch_scatter<T>(a, s)) != cudaSuccess) return e;
    return mark(c, kPhScatter);
  }
  if ((e = mark(c, 0)) != cudaSuccess) return e;
  if ((e = launch_sample_rays<T>(ra, s)) != cudaSuccess) return e;
  if ((e = mark(c, kPhSample)) != cudaSuccess) return e;
  if (c->general3d) {
    // random directions: march with voxel lists, Gram through them, tiled
    // solve; the scatter clears the lists' heads
    const FrameArgs fa{c->d_frames, c->d_map_ray, c->d_vnext};
    a.map_ray = c->d_map_ray;
    if ((e = launch_forward_frames<T>(ra, fa, (T*)c->d_x, (const T*)c->d_b, s)) != cudaSuccess)
      return e;
    if ((e = mark(c, kPhForward)) != cudaSuccess) return e;
    if ((e = launch_gram_frames(ra, fa, s)) != cudaSuccess) return e;
    if ((e = mark(c, kPhGram)) != cudaSuccess) return e;
    if ((e = enqueue_solve(c)) != cudaSuccess) return e;
    if (c->stage == 1) return cudaSuccess;
    if ((e = mark(c, kPhSolve)) != cudaSuccess) return e;
    if ((e = launch_scatter<T>(a, s)) != cudaSuccess) return e;
    return mark(c, kPhScatter);
  }
  if ((e = launch_forward_rays<T>(ra, (T*)c->d_x, (const T*)c->d_b, s)) != cudaSuccess) return e;
  if ((e = mark(c, kPhForward)) != cudaSuccess) return e;
  if (c->dim == 2) {
    if ((e = launch_gram_pairs(ra, s)) != cudaSuccess) return e;
    if ((e = mark(c, kPhGram)) != cudaSuccess) return e;
    if ((e = enqueue_solve(c)) != cudaSuccess) return e;
    if (c->stage == 1) return cudaSuccess;
  } else {
    if ((e = launch_slice_collect(ra, s)) != cudaSuccess) return e;
    if ((e = mark(c, kPhGram)) != cudaSuccess) return e;
    if ((e = mark(c, kPhFormK)) != cudaSuccess) return e;
    if ((e = launch_slice_solve(ra, s)) != cudaSuccess) return e;
    if ((e = mark(c, kPhFactor)) != cudaSuccess) return e;
  }
  if ((e = mark(c, kPhSolve)) != cudaSuccess) return e;
  if ((e = launch_scatter<T>(a, s)) != cudaSuccess) return e;
  return mark(c, kPhScatter);
}

template <typename T>
LsqrArgs<T> make_lsqr_args(slim_ctx* c) {
  LsqrArgs<T> l;
  l.info = c->d_info;
  l.p = c->p;
  l.taps = c->taps;
  l.n = c->n;
  l.ring_ids = c->d_ring_ids;
  l.ring_pix = c->d_ring_pix;
  l.ring_w = c->d_ring_w;
  l.c = c->d_rhs;
  l.eta = c->eta;
  l.max_iter = c->lsqr_max_iter;
  l.tol = c->lsqr_tol;
  l.x = (T*)c->d_x;
  l.u = c->d_lsqr;
  l.v = l.u + c->p;
  l.w = l.v + c->n;
  l.s = l.w + c->n;
  l.tmp = l.s + c->n;
  l.part = l.tmp + c->n;
  l.stats = l.part + lsqr_part_count(c->num_sms);
  l.bar = c->d_lsqr_bar;
  l.status = c->d_status;
  l.wh = c->d_cinvh;
  l.vs = l.stats + 3;
  return l;
}

TiklArgs make_tikl_args(const slim_ctx* c) {
  return TiklArgs{c->d_tl_d0inv, c->d_tl_d1, c->d_tl_U, c->d_tl_UT, c->d_tl_v};
}

template <typename T>
cudaError_t enqueue_step_t(slim_ctx* c) {
  if (c->kind != SLIM_BLOCKS_VIEWS) return enqueue_ray_step_t<T>(c);
  StepArgs<T> a = make_args<T>(c);
  cudaError_t e;
  if (c->solver == SLIM_SOLVE_LSQR) {
    // Eq. (slimLSstep) by LSQR over the window's taps: no Gram, no factor
    if ((e = mark(c, 0)) != cudaSuccess) return e;
    if ((e = launch_sample<T>(a, c->stream)) != cudaSuccess) return e;
    if ((e = mark(c, kPhSample)) != cudaSuccess) return e;
    if ((e = launch_forward_residual<T>(a, c->stream)) != cudaSuccess) return e;
    // slimTik: c - (beta/mu_k) M_k x_{k-1}
    if (c->tik_lambda > 0.0 && (e = launch_tik_rhs<T>(a, c->stream)) != cudaSuccess) return e;
    // the residual kernel enters the new block in the pixel map for the Gram
    // update, which LSQR does not run: clear it for the next step
    if ((e = cudaMemsetAsync(c->d_map_ray, 0xFF, 2 * (size_t)c->n * sizeof(int), c->stream)) !=
        cudaSuccess)
      return e;
    for (int ph = kPhForward; ph <= kPhFactor; ++ph)
      if ((e = mark(c, ph)) != cudaSuccess) return e;
    if ((e = launch_lsqr<T>(make_lsqr_args<T>(c), c->num_sms, c->stream)) != cudaSuccess) return e;
    if ((e = mark(c, kPhSolve)) != cudaSuccess) return e;
    return mark(c, kPhScatter);
  }
  if (c->solver == SLIM_SOLVE_SG || c->solver == SLIM_SOLVE_OLBFGS) {
    // the comparators: no Gram matrix, no factor
    if ((e = mark(c, 0)) != cudaSuccess) return e;
    if ((e = launch_sample<T>(a, c->stream)) != cudaSuccess) return e;
    if ((e = mark(c, kPhSample)) != cudaSuccess) return e;
    if ((e = launch_forward_residual<T>(a, c->stream)) != cudaSuccess) return e;
    for (int ph = kPhForward; ph <= kPhSolve; ++ph)
      if ((e = mark(c, ph)) != cudaSuccess) return e;
    if (c->solver == SLIM_SOLVE_SG) {
      if ((e = launch_scatter<T>(a, c->stream)) != cudaSuccess) return e;
    } else {
      OlbfgsArgs<T> o;
      o.info = c->d_info;
      o.ell = c->ell;
      o.taps = c->taps;
      o.tau = c->olbfgs_memory;
      o.n = c->n;
      o.ring_pix = c->d_ring_pix;
      o.ring_w = c->d_ring_w;
      o.rhs = c->d_rhs;
      o.map_ray = c->d_map_ray;
      o.eta = c->eta;
      o.x = (T*)c->d_x;
      o.state = c->d_olb_state;
      o.bar = c->d_lsqr_bar;
      o.status = c->d_status;
      olbfgs_bind(&o, c->d_olb, c->num_sms);
      if ((e = launch_olbfgs<T>(o, c->num_sms, c->stream)) != cudaSuccess) return e;
    }
    return mark(c, kPhScatter);
  }
  const bool tik = c->tik_lambda > 0.0;
  const bool tikl = c->d_tl_d0inv != nullptr;
  if (c->stage == 2) goto solves;   // a batch's second stage: the part after the factor
  if ((e = mark(c, 0)) != cudaSuccess) return e;
  if ((e = launch_sample<T>(a, c->stream)) != cudaSuccess) return e;
  if ((e = mark(c, kPhSample)) != cudaSuccess) return e;
  if ((e = launch_forward_residual<T>(a, c->stream)) != cudaSuccess) return e;
  // slimTik: rhs c - (beta/mu_k) M_k x_{k-1}
  if (tik && (e = launch_tik_rhs<T>(a, c->stream)) != cudaSuccess) return e;
  if ((e = mark(c, kPhForward)) != cudaSuccess) return e;
  if (tikl) {
    // G = M W M^T with W = (L^T L)^{-1}: rows W a_i^T of the new block first
    if ((e = launch_tikl_gram<T>(a, make_tikl_args(c), c->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_map_ray, 0xFF, 2 * (size_t)c->n * sizeof(int), c->stream)) !=
        cudaSuccess)
      return e;
  } else if ((e = launch_gram_update<T>(a, c->stream)) != cudaSuccess) {
    return e;
  }
  if ((e = mark(c, kPhGram)) != cudaSuccess) return e;
solves:
  if ((e = enqueue_solve(c)) != cudaSuccess) return e;
  if (c->stage == 1) return cudaSuccess;
  if ((e = mark(c, kPhSolve)) != cudaSuccess) return e;
  if (tik && (e = launch_tik_scale<T>(a, c->stream)) != cudaSuccess) return e;
  if (tikl)
    e = launch_tikl_update<T>(a, make_tikl_args(c), c->stream);
  else
    e = launch_scatter<T>(a, c->stream);
  if (e != cudaSuccess) return e;
  return mark(c, kPhScatter);
}

cudaError_t enqueue_step(slim_ctx* c) {
  return c->precision == SLIM_PREC_FP32 ? enqueue_step_t<float>(c) : enqueue_step_t<double>(c);
}

// Rebuild the memory for the state after k steps (no change to x).
template <typename T>
cudaError_t rebuild_t(slim_ctx* c, long long k) {
  cudaStream_t s = c->stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->d_ring_ids, 0xFF, (size_t)c->p * sizeof(int), s)) != cudaSuccess)
    return e;
  if (c->d_G && (e = cudaMemsetAsync(c->d_G, 0, (size_t)c->P * c->P * sizeof(double), s)) !=
                    cudaSuccess)
    return e;
  if (c->d_map_ray &&
      (e = cudaMemsetAsync(c->d_map_ray, 0xFF, 2 * (size_t)c->n * sizeof(int), s)) != cudaSuccess)
    return e;
  StepArgs<T> a = make_args<T>(c);
  long long j0 = k - c->r;
  if (j0 < 1) j0 = 1;
  for (long long j = j0; j <= k; ++j) {
    long long done = j - 1;
    if ((e = cudaMemcpyAsync(c->d_done, &done, sizeof(done), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;   // `done` is a host local
    if (c->general3d) {
      RayArgs ra = make_ray_args(c);
      const FrameArgs fa{c->d_frames, c->d_map_ray, c->d_vnext};
      if ((e = launch_sample_rays<T>(ra, s)) != cudaSuccess) return e;
      if ((e = launch_forward_frames<T>(ra, fa, (T*)c->d_x, (const T*)c->d_b, s)) != cudaSuccess)
        return e;
      if ((e = launch_gram_frames(ra, fa, s)) != cudaSuccess) return e;
      if ((e = cudaMemsetAsync(c->d_map_ray, 0xFF, 2 * (size_t)c->n * sizeof(int), s)) !=
          cudaSuccess)
        return e;
      continue;
    }
    if (c->kind != SLIM_BLOCKS_VIEWS) {
      RayArgs ra = make_ray_args(c);
      if ((e = launch_sample_rays<T>(ra, s)) != cudaSuccess) return e;
      if ((e = launch_forward_rays<T>(ra, (T*)c->d_x, (const T*)c->d_b, s)) != cudaSuccess) return e;
      e = c->dim == 2 ? launch_gram_pairs(ra, s) : launch_slice_collect(ra, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    if ((e = launch_sample<T>(a, s)) != cudaSuccess) return e;
    if ((e = launch_forward_residual<T>(a, s)) != cudaSuccess) return e;
    if (c->d_G && c->d_tl_d0inv) {
      if ((e = launch_tikl_gram<T>(a, make_tikl_args(c), s)) != cudaSuccess) return e;
    } else if (c->d_G && (e = launch_gram_update<T>(a, s)) != cudaSuccess) {
      return e;
    }
    if ((e = cudaMemsetAsync(c->d_map_ray, 0xFF, 2 * (size_t)c->n * sizeof(int), s)) !=
        cudaSuccess)
      return e;
  }
  long long done = k;
  if ((e = cudaMemcpyAsync(c->d_done, &done, sizeof(done), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  return cudaStreamSynchronize(s);
}

slim_status read_status(slim_ctx* c) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "status");
  if (st != 0) {
    int zero = 0;
    cudaMemcpy(c->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    switch (st) {
      case SLIM_ENOTPD: return fail(c, SLIM_ENOTPD, "lambda_k I + G is not positive definite");
      case SLIM_ETIMEOUT: return fail(c, SLIM_ETIMEOUT, "a bounded device wait ran out");
      case SLIM_EINVAL:
        return fail(c, SLIM_EINVAL, "a pixel is tapped by more than two rays of one view");
      default: return fail(c, (slim_status)st, "device error");
    }
  }
  return SLIM_OK;
}

void free_all(slim_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  void* ptrs[] = {c->d_slice_cnt, c->d_slice_rows, c->d_views, c->d_info, c->d_done, c->d_status, c->d_x, c->d_b,
                  c->d_ring_ids, c->d_ring_pix, c->d_ring_w, c->d_map_ray, c->d_map_w,
                  c->d_G, c->d_L, c->d_rhs, c->d_z, c->d_dz, c->d_res, c->d_ref, c->d_err,
                  c->d_lsqr, c->d_lsqr_bar, c->d_cinv, c->d_olb, c->d_olb_state,
                  c->d_frames, c->d_vnext, c->d_cinvh, c->d_perm, c->d_perm_epoch,
                  c->d_tl_d0inv, c->d_tl_d1, c->d_tl_U, c->d_tl_UT, c->d_tl_v};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  chol_plan_destroy(&c->plan);
  free_csr(&c->csr);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  // pipelined form
  for (cudaEvent_t e : c->log_f) cudaEventDestroy(e);
  for (cudaEvent_t e : c->log_x) cudaEventDestroy(e);
  for (int b = 0; b < kMaxBuf; ++b) {
    if (c->g1_exec[b]) cudaGraphExecDestroy(c->g1_exec[b]);
    if (c->g2_exec[b]) cudaGraphExecDestroy(c->g2_exec[b]);
    if (c->gx_exec[b]) cudaGraphExecDestroy(c->gx_exec[b]);
    if (c->d_Lb[b]) cudaFree(c->d_Lb[b]);
    chol_plan_destroy(&c->planb[b]);
    if (c->d_Xb[b]) cudaFree(c->d_Xb[b]);
    tri_inverse_plan_destroy(&c->tplan[b]);
    tc_chol_plan_destroy(&c->cplan[b]);
    if (c->ev_g2[b]) cudaEventDestroy(c->ev_g2[b]);
    if (c->ev_x[b]) cudaEventDestroy(c->ev_x[b]);
    if (c->fs[b]) cudaStreamDestroy(c->fs[b]);
  }
  for (cudaEvent_t e : c->la_ev)
    if (e) cudaEventDestroy(e);
  if (c->ev_user) cudaEventDestroy(c->ev_user);
  if (c->ev_g1) cudaEventDestroy(c->ev_g1);
  if (c->xs) cudaStreamDestroy(c->xs);
  if (c->gs) cudaStreamDestroy(c->gs);
  if (c->d_gdone) cudaFree(c->d_gdone);
  if (c->d_ty) cudaFree(c->d_ty);
  if (c->d_coop_bar) cudaFree(c->d_coop_bar);
  if (c->d_info_buf) cudaFree(c->d_info_buf);
  if (c->d_ext) cudaFree(c->d_ext);
}

void drop_graph(slim_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
}

// ---------------------------------------------------------------------------
// Pipelined form: three kinds of graph, replayed on internal streams
//   geometry (one graph, stream gs): draw tau_j, march its taps, Gram rows,
//     clear the pixel map;
//   factor (graph b, stream fs[b]): ring map and K_j into buffer b = j mod (D+1),
//     tiled factorisation;
//   iterate (graph b, high-priority stream xs): residual, solve with buffer b,
//     refinement, scatter.
// Events order them: geometry j waits for the iterate chain j-D-1 (the last
// reader of its tap slot, Gram rows and buffer); factor j waits for geometry
// j; iterate k waits for the caller's stream and for factor k.
// ---------------------------------------------------------------------------
template <typename T>
LaArgs<T> make_la_args(slim_ctx* c) {
  LaArgs<T> a;
  a.views = c->d_views;
  a.N = c->N;
  a.D = c->D;
  a.n_views = c->n_views;
  a.n = c->n;
  a.m = c->m;
  a.ell = c->ell;
  a.r = c->r;
  a.nslots = c->nslots;
  a.eslots = c->eslots;
  a.p = c->p;
  a.P = c->P;
  a.Pe = c->Pe;
  a.taps = c->taps;
  a.seed = c->seed;
  a.lam = c->lam;
  a.eta = c->eta;
  a.ramp = c->ramp;
  a.decay_after = c->decay_after;
  a.gdone = c->d_gdone;
  a.info_buf = c->d_info_buf;
  a.nbuf = c->nbuf;
  a.ring_ids = c->d_ring_ids;
  a.ring_pix = c->d_ring_pix;
  a.ring_w = c->d_ring_w;
  a.map_ray = c->d_map_ray;
  a.map_w = c->d_map_w;
  a.G = c->d_G;
  a.rhs = c->d_rhs;
  a.z = c->d_z;
  a.x = (T*)c->d_x;
  a.b = (const T*)c->d_b;
  a.status = c->d_status;
  a.tik_beta = c->tik_lambda * c->tik_lambda / c->n_views;   // M = A_v view blocks
  a.tik_reading = c->tik_reading;
  a.cinv = c->d_cinv;
  a.cyclic = c->cyclic;
  a.perm = c->d_perm;
  a.perm_epoch = c->d_perm_epoch;
  return a;
}

cudaError_t la_mark(slim_ctx* c, int i, cudaStream_t s) {
  if (!c->timing) return cudaSuccess;
  return cudaEventRecordWithFlags(c->la_ev[i], s, cudaEventRecordExternal);
}

template <typename T>
cudaError_t la_enqueue_geometry(slim_ctx* c, int b, cudaStream_t s) {
  LaArgs<T> a = make_la_args<T>(c);
  int* ext = c->d_ext + (size_t)b * c->P;
  const StepInfo* info = c->d_info_buf + b;
  cudaError_t e;
  if ((e = la_mark(c, 0, s)) != cudaSuccess) return e;
  if ((e = la_launch_sample<T>(a, s)) != cudaSuccess) return e;
  if ((e = la_launch_taps<T>(a, s)) != cudaSuccess) return e;
  if ((e = la_mark(c, 1, s)) != cudaSuccess) return e;
  if ((e = la_launch_gram<T>(a, s)) != cudaSuccess) return e;
  if ((e = la_launch_map_clear<T>(a, s)) != cudaSuccess) return e;
  if ((e = la_mark(c, 2, s)) != cudaSuccess) return e;
  if ((e = la_launch_ext_map(info, c->ell, c->nslots, c->eslots, c->p, c->P, ext, s)) !=
      cudaSuccess)
    return e;
  if (is_mixed(c))
    e = la_launch_form<float>(info, ext, c->d_G, c->Pe, (float*)c->d_Lb[b], c->P, s);
  else
    e = la_launch_form<double>(info, ext, c->d_G, c->Pe, (double*)c->d_Lb[b], c->P, s);
  if (e != cudaSuccess) return e;
  return la_mark(c, 3, s);
}

cudaError_t la_enqueue_factor(slim_ctx* c, int b, cudaStream_t s) {
  cudaError_t e;
  if ((e = la_mark(c, 4, s)) != cudaSuccess) return e;
  if (c->solver == SLIM_SOLVE_MIXED_TC)
    e = tc_cholesky(c->cplan[b], (float*)c->d_Lb[b], (float*)c->planb[b].d_winv, c->d_status, s);
  else
    e = chol_factor(c->planb[b], c->d_Lb[b], c->d_status, s);
  if (e != cudaSuccess) return e;
  if (uses_inverse(c) &&
      (e = tri_inverse(c->tplan[b], (const float*)c->planb[b].d_winv, (float*)c->d_Xb[b],
                       c->d_status, s)) != cudaSuccess)
    return e;
  return la_mark(c, 5, s);
}

template <typename T>
cudaError_t la_enqueue_iterate(slim_ctx* c, int b, cudaStream_t s) {
  LaArgs<T> a = make_la_args<T>(c);
  const int* ext = c->d_ext + (size_t)b * c->P;
  const StepInfo* info = c->d_info_buf + b;
  cudaError_t e;
  if ((e = la_mark(c, 6, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->d_rhs, 0, (size_t)c->P * sizeof(double), s)) != cudaSuccess) return e;
  if ((e = la_launch_residual<T>(a, info, s)) != cudaSuccess) return e;
  const bool tik = c->tik_lambda > 0.0;
  // slimTik: rhs c - (beta/mu_k) M_k x_{k-1}
  if (tik && (e = la_launch_tik_rhs<T>(a, ext, info, s)) != cudaSuccess) return e;
  if ((e = la_mark(c, 7, s)) != cudaSuccess) return e;
  // slimLS: the right-hand side is zero above the newest block (the last one)
  const int first_tile = tik ? 0 : (c->nslots - 1) * c->ell / c->nb;
  if (uses_inverse(c)) {
    // z = X^T X rhs with X = L^{-1}: two matrix-vector products per solve
    const float* X = (const float*)c->d_Xb[b];
    const int lo = tik ? 0 : (c->nslots - 1) * c->ell;
    if ((e = trinv_lower(X, c->P, c->p, lo, c->d_rhs, c->d_ty, s)) != cudaSuccess) return e;
    if ((e = trinv_upper(X, c->P, c->p, lo, c->d_ty, c->d_z, 0, s)) != cudaSuccess) return e;
    for (int it = 0; it < c->refine_iters; ++it) {
      if ((e = la_launch_refine(info, ext, c->d_G, c->Pe, c->d_z, c->d_rhs, c->d_res, c->P, s)) !=
          cudaSuccess)
        return e;
      if ((e = trinv_lower(X, c->P, c->p, 0, c->d_res, c->d_ty, s)) != cudaSuccess) return e;
      if ((e = trinv_upper(X, c->P, c->p, 0, c->d_ty, c->d_z, 1, s)) != cudaSuccess) return e;
    }
  } else if ((e = chol_solve(c->planb[b], c->d_Lb[b], c->d_rhs, c->d_z, c->d_status, s,
                             first_tile)) != cudaSuccess) {
    return e;
  }
  if (c->solver == SLIM_SOLVE_MIXED) {
    for (int it = 0; it < c->refine_iters; ++it) {
      if ((e = la_launch_refine(info, ext, c->d_G, c->Pe, c->d_z, c->d_rhs, c->d_res, c->P, s)) !=
          cudaSuccess)
        return e;
      if ((e = chol_solve(c->planb[b], c->d_Lb[b], c->d_res, c->d_dz, c->d_status, s)) !=
          cudaSuccess)
        return e;
      if ((e = launch_axpy(c->d_z, c->d_dz, c->P, s)) != cudaSuccess) return e;
    }
  }
  if ((e = la_mark(c, 8, s)) != cudaSuccess) return e;
  if (tik && (e = la_launch_tik_scale<T>(a, info, s)) != cudaSuccess) return e;
  if ((e = la_launch_scatter<T>(a, ext, s)) != cudaSuccess) return e;
  return la_mark(c, 9, s);
}

// Capture `body` on stream s into an instantiated graph.
template <typename F>
cudaError_t la_capture(cudaStream_t s, cudaGraphExec_t* exec, F body) {
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t eb = body();
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  if (eb != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return eb != cudaSuccess ? eb : e;
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

void la_drop_graphs(slim_ctx* c) {
  for (int b = 0; b < kMaxBuf; ++b) {
    if (c->g1_exec[b]) cudaGraphExecDestroy(c->g1_exec[b]);
    c->g1_exec[b] = nullptr;
    if (c->g2_exec[b]) cudaGraphExecDestroy(c->g2_exec[b]);
    if (c->gx_exec[b]) cudaGraphExecDestroy(c->gx_exec[b]);
    c->g2_exec[b] = nullptr;
    c->gx_exec[b] = nullptr;
  }
}

cudaError_t la_build_graphs(slim_ctx* c) {
  const bool f32 = c->precision == SLIM_PREC_FP32;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < c->nbuf && e == cudaSuccess; ++b) {
    e = la_capture(c->gs, &c->g1_exec[b], [&] {
      return f32 ? la_enqueue_geometry<float>(c, b, c->gs) : la_enqueue_geometry<double>(c, b, c->gs);
    });
    if (e == cudaSuccess)
      e = la_capture(c->fs[b], &c->g2_exec[b], [&] { return la_enqueue_factor(c, b, c->fs[b]); });
    if (e == cudaSuccess)
      e = la_capture(c->xs, &c->gx_exec[b], [&] {
        return f32 ? la_enqueue_iterate<float>(c, b, c->xs) : la_enqueue_iterate<double>(c, b, c->xs);
      });
  }
  return e;
}

cudaError_t la_sync_all(slim_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->gs);
  for (int b = 0; b < c->nbuf && e == cudaSuccess; ++b) e = cudaStreamSynchronize(c->fs[b]);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->xs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

// Enqueue steps h_k+1 .. h_k+nsteps.
cudaError_t la_step(slim_ctx* c, int nsteps) {
  cudaError_t e = cudaSuccess;
  if (!c->g1_exec[0] && (e = la_build_graphs(c)) != cudaSuccess) return e;
  const bool log = c->timing && !c->log_f.empty();
  for (int t = 0; t < nsteps; ++t) {
    const long long k = c->h_k + 1;
    while (c->h_g < k + c->lookahead) {
      const long long j = ++c->h_g;
      const int b = (int)(j % c->nbuf);
      if ((e = cudaStreamWaitEvent(c->gs, c->ev_x[b], 0)) != cudaSuccess) return e;
      if ((e = cudaGraphLaunch(c->g1_exec[b], c->gs)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(c->ev_g1, c->gs)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(c->fs[b], c->ev_g1, 0)) != cudaSuccess) return e;
      const int li = (int)(c->log_nf % slim_ctx::kLog);
      if (log && (e = cudaEventRecord(c->log_f[2 * li], c->fs[b])) != cudaSuccess) return e;
      if ((e = cudaGraphLaunch(c->g2_exec[b], c->fs[b])) != cudaSuccess) return e;
      if (log) {
        if ((e = cudaEventRecord(c->log_f[2 * li + 1], c->fs[b])) != cudaSuccess) return e;
        ++c->log_nf;
      }
      if ((e = cudaEventRecord(c->ev_g2[b], c->fs[b])) != cudaSuccess) return e;
    }
    const int b = (int)(k % c->nbuf);
    if ((e = cudaEventRecord(c->ev_user, c->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->xs, c->ev_user, 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->xs, c->ev_g2[b], 0)) != cudaSuccess) return e;
    const int lx = (int)(c->log_nx % slim_ctx::kLog);
    if (log && (e = cudaEventRecord(c->log_x[2 * lx], c->xs)) != cudaSuccess) return e;
    if (c->coop_grid) {
      // the tensor-core form's chain as one cooperative launch (its phases
      // are one interval: the timing reports it all as the solve phase)
      if (c->timing && ((e = cudaEventRecord(c->la_ev[6], c->xs)) != cudaSuccess ||
                        (e = cudaEventRecord(c->la_ev[7], c->xs)) != cudaSuccess))
        return e;
      const bool f32 = c->precision == SLIM_PREC_FP32;
      const int* ext = c->d_ext + (size_t)b * c->P;
      const StepInfo* info = c->d_info_buf + b;
      e = f32 ? iterate_tc<float>(make_la_args<float>(c), info, ext, (const float*)c->d_Xb[b],
                                  c->d_ty, c->d_res, c->d_coop_bar, c->refine_iters,
                                  c->coop_grid, c->xs)
              : iterate_tc<double>(make_la_args<double>(c), info, ext, (const float*)c->d_Xb[b],
                                   c->d_ty, c->d_res, c->d_coop_bar, c->refine_iters,
                                   c->coop_grid, c->xs);
      if (e != cudaSuccess) return e;
      if (c->timing && ((e = cudaEventRecord(c->la_ev[8], c->xs)) != cudaSuccess ||
                        (e = cudaEventRecord(c->la_ev[9], c->xs)) != cudaSuccess))
        return e;
    } else if ((e = cudaGraphLaunch(c->gx_exec[b], c->xs)) != cudaSuccess) {
      return e;
    }
    if (log) {
      if ((e = cudaEventRecord(c->log_x[2 * lx + 1], c->xs)) != cudaSuccess) return e;
      ++c->log_nx;
    }
    if ((e = cudaEventRecord(c->ev_x[b], c->xs)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->stream, c->ev_x[b], 0)) != cudaSuccess) return e;
    c->h_k = k;
  }
  return e;
}

// Rebuild the tap ring and the Gram rows of the window of step k (x unchanged).
cudaError_t la_rebuild(slim_ctx* c, long long k) {
  cudaError_t e = la_sync_all(c);
  if (e != cudaSuccess) return e;
  if (!c->g1_exec[0] && (e = la_build_graphs(c)) != cudaSuccess) return e;
  for (long long j = std::max<long long>(1, k - c->r); j <= k; ++j) {
    long long done = j - 1;
    if ((e = cudaMemcpy(c->d_gdone, &done, sizeof(done), cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
    if ((e = cudaGraphLaunch(c->g1_exec[j % c->nbuf], c->gs)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(c->gs)) != cudaSuccess) return e;
  }
  long long done = k;
  if ((e = cudaMemcpy(c->d_gdone, &done, sizeof(done), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  c->h_g = k;
  c->h_k = k;
  return cudaSuccess;
}

// Ring index q of step k -> extended row (host copy of the device map).
int la_ext_host(const slim_ctx* c, long long k, int q) {
  if (q >= c->p) return -1;
  const int s = q / c->ell;
  const long long blk = k - (((k - 1 - s) % c->nslots) + c->nslots) % c->nslots;
  if (blk < 1) return -1;
  return (int)((blk - 1) % c->eslots) * c->ell + q % c->ell;
}

}  // namespace

extern "C" {

slim_status slim_create(const slim_geometry* geom, const slim_blocks* blocks, int r, double lambda,
                        const slim_step_opts* step, slim_ctx** out) {
  if (!out) return SLIM_EINVAL;
  *out = nullptr;
  if (!geom || !blocks) return SLIM_EINVAL;
  if (geom->dim != 2 && geom->dim != 3) return SLIM_EINVAL;
  if (geom->dim == 2 && geom->det_v != 1) return SLIM_EINVAL;
  const bool frames = geom->dim == 3 && geom->frames != nullptr;
  if (geom->dim == 2 && geom->frames) return SLIM_EINVAL;
  if (geom->dim == 3 && !frames && geom->det_v != geom->n_side) return SLIM_ENOTSUP;
  if (frames) {
    // each row (d, u, v) orthonormal
    for (int a = 0; a < geom->n_views; ++a) {
      const double* f = geom->frames + 9 * (size_t)a;
      for (int q = 0; q < 9; ++q)
        if (!std::isfinite(f[q])) return SLIM_EINVAL;
      auto dot = [&](int x, int y) { return f[x] * f[y] + f[x + 1] * f[y + 1] + f[x + 2] * f[y + 2]; };
      if (std::fabs(dot(0, 0) - 1.0) > 1e-9 || std::fabs(dot(3, 3) - 1.0) > 1e-9 ||
          std::fabs(dot(6, 6) - 1.0) > 1e-9 || std::fabs(dot(0, 3)) > 1e-9 ||
          std::fabs(dot(0, 6)) > 1e-9 || std::fabs(dot(3, 6)) > 1e-9)
        return SLIM_EINVAL;
    }
    if (geom->det_v < 1 || (long long)geom->det_v * geom->det_u * geom->n_views > 0x7fffffffLL)
      return SLIM_EINVAL;
  }
  if (geom->a_mode < 0 || geom->a_mode > 2) return SLIM_EINVAL;
  if (geom->n_side < 2 || geom->n_side > 16384 || geom->n_views < 1 || geom->det_u < 1)
    return SLIM_EINVAL;
  if (geom->precision != SLIM_PREC_FP64 && geom->precision != SLIM_PREC_FP32) return SLIM_EINVAL;
  if (blocks->kind < SLIM_BLOCKS_VIEWS || blocks->kind > SLIM_BLOCKS_STREAM) return SLIM_EINVAL;
  if (blocks->kind == SLIM_BLOCKS_VIEWS && (geom->dim != 2 || blocks->ell != geom->det_u))
    return SLIM_EINVAL;
  if (blocks->kind != SLIM_BLOCKS_VIEWS && geom->a_mode != 0) return SLIM_ENOTSUP;
  if (geom->dim == 3 && blocks->kind == SLIM_BLOCKS_VIEWS) return SLIM_ENOTSUP;
  if (blocks->kind == SLIM_BLOCKS_STREAM && blocks->steps_per_view < 1) return SLIM_EINVAL;
  if (blocks->ell < 1) return SLIM_EINVAL;
  if ((blocks->with_replacement != 0 && blocks->with_replacement != 1) ||
      (blocks->cyclic != 0 && blocks->cyclic != 1))
    return SLIM_EINVAL;
  if (blocks->kind == SLIM_BLOCKS_VIEWS) {
    // a view block without replacement within the epoch is the random cyclic order
    if ((blocks->cyclic || !blocks->with_replacement) && geom->n_views > kMaxCyclicViews)
      return SLIM_ENOTSUP;
  } else {
    if (blocks->cyclic) return SLIM_ENOTSUP;   // random-ray blocks have no epoch order
    if (!blocks->with_replacement) {
      const long long first = blocks->kind == SLIM_BLOCKS_STREAM
                                  ? (long long)geom->det_u * (geom->dim == 3 ? geom->det_v : 1)
                                  : (long long)geom->n_views * geom->det_u *
                                        (geom->dim == 3 ? geom->det_v : 1);
      if (blocks->ell > kMaxDistinctRays) return SLIM_ENOTSUP;
      if (blocks->ell > first) return SLIM_EINVAL;   // not enough rays to draw distinct ones
    }
  }
  if (r < 0 || !(lambda > 0.0) || !std::isfinite(lambda)) return SLIM_EINVAL;
  slim_ctx* c = new (std::nothrow) slim_ctx();
  if (!c) return SLIM_ENOMEM;
  c->N = geom->n_side;
  c->n_views = geom->n_views;
  c->D = geom->det_u;
  c->Dv = geom->det_v;
  c->dim = geom->dim;
  c->kind = blocks->kind;
  c->steps_per_view = blocks->kind == SLIM_BLOCKS_STREAM ? blocks->steps_per_view : 1;
  c->cyclic = blocks->kind == SLIM_BLOCKS_VIEWS && (blocks->cyclic || !blocks->with_replacement);
  c->distinct = blocks->kind != SLIM_BLOCKS_VIEWS && !blocks->with_replacement;
  c->n = c->dim == 3 ? (long long)c->N * c->N * c->N : (long long)c->N * c->N;
  c->m = (long long)c->n_views * c->D * c->Dv;
  c->precision = geom->precision;
  c->a_mode = geom->a_mode;
  c->r = r;
  c->nslots = r + 1;
  c->ell = blocks->ell;
  c->seed = blocks->seed;
  c->lam = lambda;
  c->p = c->nslots * c->ell;
  c->taps = 2 * c->N;
  c->general3d = frames;
  if (frames) c->taps = 4 * c->N;   // four bilinear taps per slice
  if (step) {
    c->eta = step->eta;
    c->ramp = step->ramp;
    c->solver = step->solver;
    c->refine_iters = step->refine_iters;
    c->use_graph = step->use_graph;
    c->tile = step->tile;
    c->lookahead = step->lookahead;
    c->cps_auto = step->ctas_per_sm == 0;
    c->ctas_per_sm = step->ctas_per_sm ? step->ctas_per_sm : 1;
    c->lsqr_max_iter = step->lsqr_max_iter;
    c->lsqr_tol = step->lsqr_tol;
    c->tik_lambda = step->tik_lambda;
    c->tik_reading = step->tik_reading;
    c->decay_after = step->decay_after;
    c->olbfgs_memory = step->olbfgs_memory ? step->olbfgs_memory : 10;
    c->ray_lanes = step->ray_lanes ? step->ray_lanes : 32;
    c->pair_window = step->pair_window ? step->pair_window : 32;
    if (c->decay_after < 0 ||
        (c->ray_lanes != 8 && c->ray_lanes != 16 && c->ray_lanes != 32) ||
        c->pair_window < 8 || c->pair_window > 256 ||
        (c->solver == SLIM_SOLVE_OLBFGS &&
         (c->olbfgs_memory < 1 || c->olbfgs_memory > kOlbfgsMaxMem))) {
      delete c;
      return SLIM_EINVAL;
    }
    if (c->solver == SLIM_SOLVE_SG || c->solver == SLIM_SOLVE_OLBFGS) {
      if (c->r != 0) {   // the comparators keep no slimLS memory
        delete c;
        return SLIM_EINVAL;
      }
      if (c->kind != SLIM_BLOCKS_VIEWS || c->dim != 2 || c->lookahead != 0 ||
          c->tik_lambda != 0.0) {
        delete c;
        return SLIM_ENOTSUP;
      }
      if (c->solver == SLIM_SOLVE_OLBFGS) c->use_graph = 0;   // a cooperative launch per step
    }
    if (!(c->tik_lambda >= 0.0) || !std::isfinite(c->tik_lambda) ||
        (c->tik_reading != 0 && c->tik_reading != 1)) {
      delete c;
      return SLIM_EINVAL;
    }
    if (c->tik_lambda > 0.0 && (c->kind != SLIM_BLOCKS_VIEWS || c->dim != 2 ||
                                (c->solver != SLIM_SOLVE_FP64 && !is_mixed(c) &&
                                 c->solver != SLIM_SOLVE_LSQR))) {
      delete c;
      return SLIM_ENOTSUP;
    }
    if (c->solver == SLIM_SOLVE_LSQR) {
      if (c->lsqr_max_iter < 1 || c->lsqr_max_iter > 1000000 || !(c->lsqr_tol >= 0.0) ||
          !std::isfinite(c->lsqr_tol)) {
        delete c;
        return SLIM_EINVAL;
      }
      if (c->kind != SLIM_BLOCKS_VIEWS || c->dim != 2 || c->a_mode != 0 || c->lookahead != 0) {
        delete c;
        return SLIM_ENOTSUP;
      }
      c->use_graph = 0;   // a cooperative launch per step
    }
    if (!(c->eta > 0.0) ||
        (c->solver != SLIM_SOLVE_FP64 && !is_mixed(c) &&
         c->solver != SLIM_SOLVE_LSQR && c->solver != SLIM_SOLVE_SG &&
         c->solver != SLIM_SOLVE_OLBFGS) ||
        c->refine_iters < 0 || c->refine_iters > 16 || (c->tile != 0 && c->tile != 32 && c->tile != 64) ||
        c->ctas_per_sm < 1 || c->ctas_per_sm > 4 || c->lookahead < 0 ||
        c->lookahead > kMaxBuf - 1) {
      delete c;
      return SLIM_EINVAL;
    }
    if (c->lookahead && (c->kind != SLIM_BLOCKS_VIEWS || c->dim != 2 || c->a_mode != 0)) {
      delete c;
      return SLIM_ENOTSUP;
    }
    // the tensor-core inverse runs in the geometry chain of the pipelined
    // form, on the 64-wide tiles of the float32 factor
    if (uses_inverse(c) &&
        (c->lookahead == 0 || (c->tile != 0 && c->tile != 64) || c->p > 8192)) {
      delete c;
      return SLIM_ENOTSUP;
    }
  }
  if (c->lookahead) {
    c->eslots = c->nslots + c->lookahead;
    c->Pe = c->eslots * c->ell;
    c->nbuf = c->lookahead + 1;
  }
  const bool la = c->lookahead > 0;
  if (c->m > 0x7fffffffLL || c->n > 0x7fffffffLL || (long long)c->p * c->p > (1LL << 33) ||
      (long long)c->Pe * c->Pe > (1LL << 33) || c->ell > c->m) {
    delete c;
    return SLIM_EINVAL;
  }
  c->nb = c->tile ? c->tile : (c->solver == SLIM_SOLVE_FP64 ? 32 : 64);
  c->P = (c->p + c->nb - 1) / c->nb * c->nb;
  // tiled Cholesky of the full p x p system (2D, and 3D with random directions)
  const bool dense_solve = c->dim == 2 || c->general3d;
  // pixel -> ray map of the new block (view blocks), or voxel list heads
  const bool use_map = c->kind == SLIM_BLOCKS_VIEWS || c->general3d;
  if (c->general3d && (c->solver != SLIM_SOLVE_FP64 && c->solver != SLIM_SOLVE_MIXED)) {
    delete c;
    return SLIM_ENOTSUP;
  }
  if (c->general3d) {
    c->h_frames.resize(c->n_views);
    for (int a = 0; a < c->n_views; ++a) c->h_frames[a] = make_frame_geom(geom->frames + 9 * (size_t)a);
  }
  if (c->dim == 3 && !c->general3d) {
    c->P = c->p;      // G stored p x p; the solve runs slice by slice
    c->S = c->N;
    c->cap = 96;
  }
  // geometry tables: host libm cos/sin, row-stepping iff |cos| >= |sin|.
  // A component below 1e-15 in magnitude is the rounding residue of an
  // axis-aligned view (cos(pi/2) evaluates to 6.1e-17): it is taken as 0 and
  // the other as +-1.  Kept, it shifts every interpolation position by a
  // fraction of an ulp, and where t + (N - 1) / 2 is an integer two
  // neighbouring rays then round into the same interpolated pixel of a step
  // (one with a weight of 1e-16), which the block's pixel -> ray map cannot hold.
  c->h_views.resize(c->n_views);
  for (int a = 0; a < c->n_views; ++a) {
    double th = geom->angles ? geom->angles[a] : a * M_PI / c->n_views;
    ViewGeom v;
    v.co = std::cos(th);
    v.si = std::sin(th);
    if (std::fabs(v.co) < 1e-15) {
      v.co = 0.0;
      v.si = std::copysign(1.0, v.si);
    } else if (std::fabs(v.si) < 1e-15) {
      v.si = 0.0;
      v.co = std::copysign(1.0, v.co);
    }
    v.row_step = std::fabs(v.co) >= std::fabs(v.si) ? 1 : 0;
    v.rc = 1.0 / (v.row_step ? v.co : v.si);
    v.ia = std::fabs(v.rc);
    v.pad_ = 0;
    c->h_views[a] = v;
  }
  slim_status st = SLIM_OK;
  auto chk = [&](cudaError_t e, const char* w) {
    if (e != cudaSuccess && st == SLIM_OK) st = cuda_fail(c, e, w);
    return e == cudaSuccess;
  };
  int dev = 0;
  chk(cudaGetDevice(&dev), "cudaGetDevice");
  chk(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
  if (st == SLIM_OK && chk(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream"))
    c->own_stream = true;
  if (la && st == SLIM_OK) {
    // the iterate chain outranks the geometry chains running ahead of it
    int least = 0, greatest = 0;
    chk(cudaDeviceGetStreamPriorityRange(&least, &greatest), "priorities");
    chk(cudaStreamCreateWithPriority(&c->xs, cudaStreamNonBlocking, greatest), "stream");
    chk(cudaStreamCreateWithPriority(&c->gs, cudaStreamNonBlocking, least), "stream");
    for (int b = 0; b < c->nbuf; ++b) {
      chk(cudaStreamCreateWithPriority(&c->fs[b], cudaStreamNonBlocking, least), "stream");
      chk(cudaEventCreateWithFlags(&c->ev_g2[b], cudaEventDisableTiming), "event");
      chk(cudaEventCreateWithFlags(&c->ev_x[b], cudaEventDisableTiming), "event");
    }
    chk(cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming), "event");
    chk(cudaEventCreateWithFlags(&c->ev_g1, cudaEventDisableTiming), "event");
  }
  const int ring_rows = la ? c->Pe : c->p;
  // LSQR and the comparators: no Gram matrix, no factor
  const bool lsqr = c->solver == SLIM_SOLVE_LSQR || c->solver == SLIM_SOLVE_SG ||
                    c->solver == SLIM_SOLVE_OLBFGS;
  const size_t g_elems = lsqr ? 0 : la ? (size_t)c->Pe * c->Pe : (size_t)c->P * c->P;
  const size_t es = elem(c->precision);
  const size_t fs = c->solver == SLIM_SOLVE_FP64 ? sizeof(double) : sizeof(float);
  struct { void** p; size_t bytes; } allocs[] = {
      {(void**)&c->d_views, c->h_views.size() * sizeof(ViewGeom)},
      {(void**)&c->d_info, sizeof(StepInfo)},
      {(void**)&c->d_done, sizeof(long long)},
      {(void**)&c->d_status, sizeof(int)},
      {&c->d_x, (size_t)c->n * es},
      {&c->d_b, (size_t)c->m * es},
      {(void**)&c->d_ring_ids, (size_t)ring_rows * sizeof(int)},
      {(void**)&c->d_ring_pix, (size_t)ring_rows * c->taps * sizeof(int)},
      {(void**)&c->d_ring_w, (size_t)ring_rows * c->taps * sizeof(double)},
      {(void**)&c->d_map_ray, use_map ? 2 * (size_t)c->n * sizeof(int) : 0},
      {(void**)&c->d_map_w, c->kind == SLIM_BLOCKS_VIEWS ? 2 * (size_t)c->n * sizeof(double) : 0},
      {(void**)&c->d_frames, c->general3d ? c->h_frames.size() * sizeof(FrameGeom) : 0},
      {(void**)&c->d_vnext, c->general3d ? (size_t)c->ell * c->taps * sizeof(int) : 0},
      {(void**)&c->d_G, g_elems * sizeof(double)},
      {&c->d_L, dense_solve && !la && !lsqr ? (size_t)c->P * c->P * fs : 0},
      {(void**)&c->d_gdone, la ? sizeof(long long) : 0},
      {(void**)&c->d_info_buf, la ? c->nbuf * sizeof(StepInfo) : 0},
      {(void**)&c->d_ext, la ? (size_t)c->nbuf * c->P * sizeof(int) : 0},
      {(void**)&c->d_slice_cnt, (size_t)c->S * sizeof(int)},
      {(void**)&c->d_slice_rows, (size_t)c->S * c->cap * sizeof(int)},
      {(void**)&c->d_rhs, (size_t)c->P * sizeof(double)},
      {(void**)&c->d_z, (size_t)c->P * sizeof(double)},
      {(void**)&c->d_dz, (size_t)c->P * sizeof(double)},
      {(void**)&c->d_res, (size_t)c->P * sizeof(double)},
      {(void**)&c->d_err, 2 * sizeof(double)},
      {(void**)&c->d_perm, c->cyclic ? (size_t)c->n_views * sizeof(int) : 0},
      {(void**)&c->d_perm_epoch, c->cyclic ? sizeof(long long) : 0},
  };
  for (auto& al : allocs)
    if (st == SLIM_OK && al.bytes > 0) chk(cudaMalloc(al.p, al.bytes), "cudaMalloc");
  if (st == SLIM_OK) {
    chk(cudaMemcpy(c->d_views, c->h_views.data(), c->h_views.size() * sizeof(ViewGeom),
                   cudaMemcpyHostToDevice), "views");
    if (c->general3d)
      chk(cudaMemcpy(c->d_frames, c->h_frames.data(), c->h_frames.size() * sizeof(FrameGeom),
                     cudaMemcpyHostToDevice), "frames");
    chk(cudaMemset(c->d_done, 0, sizeof(long long)), "memset");
    chk(cudaMemset(c->d_status, 0, sizeof(int)), "memset");
    chk(cudaMemset(c->d_x, 0, (size_t)c->n * es), "memset");
    chk(cudaMemset(c->d_b, 0, (size_t)c->m * es), "memset");
    chk(cudaMemset(c->d_ring_ids, 0xFF, (size_t)ring_rows * sizeof(int)), "memset");
    chk(cudaMemset(c->d_ring_pix, 0xFF, (size_t)ring_rows * c->taps * sizeof(int)), "memset");
    chk(cudaMemset(c->d_ring_w, 0, (size_t)ring_rows * c->taps * sizeof(double)), "memset");
    if (use_map) chk(cudaMemset(c->d_map_ray, 0xFF, 2 * (size_t)c->n * sizeof(int)), "memset");
    if (g_elems) chk(cudaMemset(c->d_G, 0, g_elems * sizeof(double)), "memset");
    if (dense_solve && !la && !lsqr) chk(cudaMemset(c->d_L, 0, (size_t)c->P * c->P * fs), "memset");
    chk(cudaMemset(c->d_z, 0, (size_t)c->P * sizeof(double)), "memset");
    if (c->cyclic) chk(cudaMemset(c->d_perm_epoch, 0xFF, sizeof(long long)), "memset");   // -1
    if (la) {
      for (int b = 0; b < c->nbuf && st == SLIM_OK; ++b)
        chk(cudaMalloc(&c->d_Lb[b], (size_t)c->P * c->P * fs), "cudaMalloc");
      chk(cudaMemset(c->d_gdone, 0, sizeof(long long)), "memset");
      chk(cudaMemset(c->d_info_buf, 0, c->nbuf * sizeof(StepInfo)), "memset");
      // up to D factorisations run at once next to the iterate chain: together
      // they take ctas_per_sm CTAs per SM, leaving room for the iterate kernels
      const int fgrid = std::max(16, c->num_sms * c->ctas_per_sm / c->lookahead);
      for (int b = 0; b < c->nbuf; ++b) {
        chk(cudaMemset(c->d_Lb[b], 0, (size_t)c->P * c->P * fs), "memset");
        chk(chol_plan_create(&c->planb[b], c->P, c->nb, is_mixed(c) ? 1 : 0,
                             fgrid, 1, 0), "chol plan");
      }
      if (uses_inverse(c) && st == SLIM_OK) {
        chk(tc_prepare(), "tensor-core product");
        if (c->solver == SLIM_SOLVE_MIXED_TC) {
          chk(chol_potrf_tile_prepare(), "diagonal tiles");
          for (int b = 0; b < c->nbuf && st == SLIM_OK; ++b)
            chk(tc_chol_plan(&c->cplan[b], c->P, (float*)c->d_Lb[b],
                             (const float*)c->planb[b].d_winv), "factor plan");
        }
        chk(cudaMalloc(&c->d_ty, (size_t)c->P * sizeof(double)), "cudaMalloc");
        if (c->tik_lambda == 0.0 && st == SLIM_OK) {
          chk(cudaMalloc(&c->d_coop_bar, 2 * sizeof(unsigned)), "cudaMalloc");
          chk(c->precision == SLIM_PREC_FP32
                  ? iterate_tc_prepare<float>(c->P, c->num_sms, &c->coop_grid)
                  : iterate_tc_prepare<double>(c->P, c->num_sms, &c->coop_grid),
              "cooperative iterate chain");
        }
        for (int b = 0; b < c->nbuf && st == SLIM_OK; ++b) {
          chk(cudaMalloc(&c->d_Xb[b], (size_t)c->P * c->P * sizeof(float)), "cudaMalloc");
          chk(cudaMemset(c->d_Xb[b], 0, (size_t)c->P * c->P * sizeof(float)), "memset");
          chk(tri_inverse_plan(&c->tplan[b], c->P, (const float*)c->d_Lb[b],
                               (const float*)c->planb[b].d_winv, (float*)c->d_Xb[b]),
              "inverse plan");
        }
      }
    } else if (c->solver == SLIM_SOLVE_SG) {
      // the scatter alone
    } else if (c->solver == SLIM_SOLVE_OLBFGS) {
      const size_t cnt = olbfgs_scratch_count(c->n, c->ell, c->olbfgs_memory, c->num_sms);
      chk(cudaMalloc(&c->d_olb, cnt * sizeof(double)), "cudaMalloc");
      chk(cudaMalloc(&c->d_olb_state, (2 + kOlbfgsMaxMem) * sizeof(int)), "cudaMalloc");
      chk(cudaMalloc(&c->d_lsqr_bar, 2 * sizeof(unsigned)), "cudaMalloc");
      // g, the spare y and the bookkeeping (no pairs) start at zero
      chk(cudaMemset(c->d_olb, 0, cnt * sizeof(double)), "memset");
      chk(cudaMemset(c->d_olb_state, 0, (2 + kOlbfgsMaxMem) * sizeof(int)), "memset");
    } else if (c->solver == SLIM_SOLVE_LSQR) {
      const size_t cnt = (size_t)c->p + 5 * (size_t)c->n + lsqr_part_count(c->num_sms) + 3;
      chk(cudaMalloc(&c->d_lsqr, cnt * sizeof(double)), "cudaMalloc");
      chk(cudaMalloc(&c->d_lsqr_bar, 2 * sizeof(unsigned)), "cudaMalloc");
      // tmp (and the rest) start at zero: the solve leaves tmp at zero
      chk(cudaMemset(c->d_lsqr, 0, cnt * sizeof(double)), "memset");
    } else if (dense_solve)
      chk(chol_plan_create(&c->plan, c->P, c->nb, is_mixed(c) ? 1 : 0,
                           c->num_sms, plan_ctas_per_sm(c)), "chol plan");
    else
      chk(prepare_slice_solve(c->cap), "slice solve");
    if (st == SLIM_OK && c->a_mode != 0)
      chk(build_csr(c->d_views, c->N, c->D, c->m, c->n, c->a_mode == 2, &c->csr, c->stream),
          "stored matrix");
    size_t gsmem = 8 * (size_t)c->ell * sizeof(double);
    if (gsmem > 200 * 1024) st = fail(c, SLIM_ENOTSUP, "ell too large for the Gram kernel");
  }
  if (st != SLIM_OK) {
    std::string msg = c->err;
    free_all(c);
    delete c;
    fprintf(stderr, "slim_create: %s\n", msg.c_str());
    return st;
  }
  *out = c;
  return SLIM_OK;
}

void slim_destroy(slim_ctx* c) {
  if (!c) return;
  if (c->lookahead && c->xs) la_sync_all(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

const char* slim_last_error(const slim_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

slim_status slim_set_stream(slim_ctx* c, void* stream) {
  if (!c) return SLIM_EINVAL;
  CK(cudaStreamSynchronize(c->stream), "sync");
  if (c->own_stream) cudaStreamDestroy(c->stream);
  c->own_stream = false;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream");
    c->own_stream = true;
  }
  drop_graph(c);
  return SLIM_OK;
}

slim_status slim_set_timing(slim_ctx* c, int on) {
  if (!c) return SLIM_EINVAL;
  if (on && !c->ev[0])
    for (cudaEvent_t& e : c->ev) CK(cudaEventCreate(&e), "event");
  if (on && c->lookahead && !c->la_ev[0]) {
    for (cudaEvent_t& e : c->la_ev) CK(cudaEventCreate(&e), "event");
    c->log_f.assign(2 * slim_ctx::kLog, nullptr);
    c->log_x.assign(2 * slim_ctx::kLog, nullptr);
    for (cudaEvent_t& e : c->log_f) CK(cudaEventCreate(&e), "event");
    for (cudaEvent_t& e : c->log_x) CK(cudaEventCreate(&e), "event");
  }
  if ((on != 0) != c->timing) {
    CK(cudaStreamSynchronize(c->stream), "sync");
    drop_graph(c);   // the captured step changes with the event records
    if (c->lookahead) {
      CK(la_sync_all(c), "sync");
      la_drop_graphs(c);
    }
  }
  c->timing = on != 0;
  return SLIM_OK;
}

slim_status slim_get_timing(slim_ctx* c, double* phase_ms, int nphase, int* kernels) {
  if (!c) return SLIM_EINVAL;
  if (kernels) *kernels = kernels_per_step(c);
  if (!phase_ms) return SLIM_OK;
  if (!c->timing || nphase < 1 || nphase > 7) return fail(c, SLIM_ESTATE, "timing is off");
  if (c->lookahead) {
    // sample+taps, residual, Gram, K, factor, solve, scatter: each from its own
    // pair of events (the geometry phases are those of the latest prepared step)
    CK(la_sync_all(c), "sync");
    const int pairs[7][2] = {{0, 1}, {6, 7}, {1, 2}, {2, 3}, {4, 5}, {7, 8}, {8, 9}};
    for (int i = 0; i < nphase; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c->la_ev[pairs[i][0]], c->la_ev[pairs[i][1]]), "elapsed");
      phase_ms[i] = ms;
    }
    return SLIM_OK;
  }
  CK(cudaStreamSynchronize(c->stream), "sync");
  for (int i = 0; i < nphase; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]), "elapsed");
    phase_ms[i] = ms;
  }
  return SLIM_OK;
}

slim_status slim_get_launch_log(slim_ctx* c, double* factor_ms, double* iterate_ms,
                                long long* count) {
  if (!c) return SLIM_EINVAL;
  if (!c->lookahead || !c->timing || c->log_f.empty())
    return fail(c, SLIM_ESTATE, "launch log: pipelined form with timing on only");
  CK(la_sync_all(c), "sync");
  auto mean = [&](std::vector<cudaEvent_t>& ev, long long n0, long long n1, double* out) {
    const long long first = std::max(n0, n1 - slim_ctx::kLog);
    double sum = 0.0;
    for (long long i = first; i < n1; ++i) {
      const int li = (int)(i % slim_ctx::kLog);
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * li], ev[2 * li + 1]) != cudaSuccess) return false;
      sum += ms;
    }
    if (out) *out = n1 > first ? sum / (double)(n1 - first) : 0.0;
    return true;
  };
  if (!mean(c->log_f, c->log_f0, c->log_nf, factor_ms) ||
      !mean(c->log_x, c->log_x0, c->log_nx, iterate_ms))
    return cuda_fail(c, cudaGetLastError(), "launch log");
  if (count) *count = c->log_nx - c->log_x0;
  c->log_f0 = c->log_nf;
  c->log_x0 = c->log_nx;
  return SLIM_OK;
}

slim_status slim_set_data(slim_ctx* c, const void* b, size_t m, int dtype, int on_device) {
  if (!c || !b || (long long)m != c->m || (dtype != SLIM_F32 && dtype != SLIM_F64))
    return fail(c, SLIM_EINVAL, "set_data: bad arguments");
  CK(copy_in(c->d_b, c->precision == SLIM_PREC_FP32, b, dtype, on_device, c->m, c->stream),
     "set_data");
  CK(cudaStreamSynchronize(c->stream), "set_data");
  c->has_data = true;
  return SLIM_OK;
}

slim_status slim_set_x(slim_ctx* c, const void* x, size_t n, int dtype, int on_device) {
  if (!c || !x || (long long)n != c->n || (dtype != SLIM_F32 && dtype != SLIM_F64))
    return fail(c, SLIM_EINVAL, "set_x: bad arguments");
  CK(copy_in(c->d_x, c->precision == SLIM_PREC_FP32, x, dtype, on_device, c->n, c->stream),
     "set_x");
  CK(cudaStreamSynchronize(c->stream), "set_x");
  return SLIM_OK;
}

slim_status slim_set_tik_bidiag(slim_ctx* c, const double* d0, const double* d1, size_t n,
                                int on_device) {
  if (!c || (d0 && (long long)n != c->n)) return fail(c, SLIM_EINVAL, "set_tik_bidiag: bad arguments");
  if (c->kind != SLIM_BLOCKS_VIEWS || c->dim != 2 || c->lookahead != 0 || c->a_mode != 0 ||
      (c->solver != SLIM_SOLVE_FP64 && c->solver != SLIM_SOLVE_MIXED))
    return fail(c, SLIM_ENOTSUP,
                "set_tik_bidiag: 2D view blocks, rows from the projector, Woodbury form "
                "(FP64 or MIXED solver), lookahead 0");
  CK(cudaStreamSynchronize(c->stream), "set_tik_bidiag");
  const size_t nn = (size_t)c->n;
  std::vector<double> h0, h1;
  if (d0) {   // read and check the new L before anything changes
    h0.resize(nn);
    h1.assign(nn, 0.0);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    CK(cudaMemcpy(h0.data(), d0, nn * sizeof(double), kind), "set_tik_bidiag");
    if (d1) CK(cudaMemcpy(h1.data(), d1, nn * sizeof(double), kind), "set_tik_bidiag");
    for (size_t i = 0; i < nn; ++i) {
      if (!(h0[i] != 0.0) || !std::isfinite(h0[i]) || !std::isfinite(h1[i]))
        return fail(c, SLIM_EINVAL, "set_tik_bidiag: L must be invertible (d0 != 0, finite)");
      h0[i] = 1.0 / h0[i];
    }
    h1[0] = 0.0;
  }
  double** bufs[] = {&c->d_tl_d0inv, &c->d_tl_d1, &c->d_tl_U, &c->d_tl_UT, &c->d_tl_v};
  for (double** b : bufs) {
    if (*b) CK(cudaFree(*b), "set_tik_bidiag");
    *b = nullptr;
  }
  if (d0) {
    // a diagonal C_k set before is replaced
    if (c->d_cinv) CK(cudaFree(c->d_cinv), "set_tik_bidiag");
    if (c->d_cinvh) CK(cudaFree(c->d_cinvh), "set_tik_bidiag");
    c->d_cinv = c->d_cinvh = nullptr;
    CK(cudaMalloc(&c->d_tl_d0inv, nn * sizeof(double)), "cudaMalloc");
    CK(cudaMalloc(&c->d_tl_d1, nn * sizeof(double)), "cudaMalloc");
    CK(cudaMalloc(&c->d_tl_U, (size_t)c->ell * nn * sizeof(double)), "cudaMalloc");
    CK(cudaMalloc(&c->d_tl_UT, (size_t)c->ell * nn * sizeof(double)), "cudaMalloc");
    CK(cudaMalloc(&c->d_tl_v, nn * sizeof(double)), "cudaMalloc");
    CK(cudaMemcpy(c->d_tl_d0inv, h0.data(), nn * sizeof(double), cudaMemcpyHostToDevice),
       "set_tik_bidiag");
    CK(cudaMemcpy(c->d_tl_d1, h1.data(), nn * sizeof(double), cudaMemcpyHostToDevice),
       "set_tik_bidiag");
  }
  // the captured step and the retained Gram entries used the previous C_k
  drop_graph(c);
  if (c->h_k > 0) {
    cudaError_t e = c->precision == SLIM_PREC_FP32 ? rebuild_t<float>(c, c->h_k)
                                                   : rebuild_t<double>(c, c->h_k);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_tik_bidiag");
  }
  return read_status(c);
}

slim_status slim_set_c_diag(slim_ctx* c, const void* cdiag, size_t n, int dtype, int on_device) {
  if (!c || (cdiag && ((long long)n != c->n || (dtype != SLIM_F32 && dtype != SLIM_F64))))
    return fail(c, SLIM_EINVAL, "set_c_diag: bad arguments");
  if (c->kind != SLIM_BLOCKS_VIEWS || c->dim != 2 ||
      (c->solver != SLIM_SOLVE_FP64 && !is_mixed(c) && c->solver != SLIM_SOLVE_LSQR))
    return fail(c, SLIM_ENOTSUP, "set_c_diag: 2D view blocks, Woodbury or LSQR form");
  CK(c->lookahead ? la_sync_all(c) : cudaStreamSynchronize(c->stream), "set_c_diag");
  {   // a bidiagonal L set before is replaced
    double** bufs[] = {&c->d_tl_d0inv, &c->d_tl_d1, &c->d_tl_U, &c->d_tl_UT, &c->d_tl_v};
    for (double** b : bufs) {
      if (*b) CK(cudaFree(*b), "set_c_diag");
      *b = nullptr;
    }
  }
  if (!cdiag) {
    if (c->d_cinv) CK(cudaFree(c->d_cinv), "set_c_diag");
    if (c->d_cinvh) CK(cudaFree(c->d_cinvh), "set_c_diag");
    c->d_cinv = nullptr;
    c->d_cinvh = nullptr;
  } else {
    // read the values to the host (as float64), check C is positive definite
    std::vector<double> h((size_t)c->n);
    if (dtype == SLIM_F64) {
      CK(cudaMemcpy(h.data(), cdiag, h.size() * sizeof(double),
                    on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost), "set_c_diag");
    } else {
      std::vector<float> f((size_t)c->n);
      CK(cudaMemcpy(f.data(), cdiag, f.size() * sizeof(float),
                    on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost), "set_c_diag");
      for (size_t i = 0; i < f.size(); ++i) h[i] = f[i];
    }
    std::vector<double> hh(h.size());
    for (size_t i = 0; i < h.size(); ++i) {
      const double v = h[i];
      if (!(v > 0.0) || !std::isfinite(v))
        return fail(c, SLIM_EINVAL, "set_c_diag: C_k must be positive definite (c > 0, finite)");
      h[i] = 1.0 / v;
      hh[i] = 1.0 / std::sqrt(v);
    }
    if (!c->d_cinv) CK(cudaMalloc(&c->d_cinv, h.size() * sizeof(double)), "cudaMalloc");
    if (!c->d_cinvh) CK(cudaMalloc(&c->d_cinvh, hh.size() * sizeof(double)), "cudaMalloc");
    CK(cudaMemcpy(c->d_cinv, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice),
       "set_c_diag");
    CK(cudaMemcpy(c->d_cinvh, hh.data(), hh.size() * sizeof(double), cudaMemcpyHostToDevice),
       "set_c_diag");
  }
  // the captured step and the retained Gram entries used the previous C_k
  if (c->lookahead) {
    la_drop_graphs(c);
    CK(la_rebuild(c, c->h_k), "set_c_diag");
    return read_status(c);
  }
  drop_graph(c);
  if (c->h_k > 0) {
    cudaError_t e = c->precision == SLIM_PREC_FP32 ? rebuild_t<float>(c, c->h_k)
                                                   : rebuild_t<double>(c, c->h_k);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_c_diag");
  }
  return read_status(c);
}

slim_status slim_get_x(slim_ctx* c, void* x, size_t n, int dtype, int on_device) {
  if (!c || !x || (long long)n != c->n || (dtype != SLIM_F32 && dtype != SLIM_F64))
    return fail(c, SLIM_EINVAL, "get_x: bad arguments");
  CK(copy_out(x, dtype, on_device, c->d_x, c->precision == SLIM_PREC_FP32, c->n, c->stream),
     "get_x");
  return read_status(c);
}

slim_status slim_step(slim_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return fail(c, SLIM_EINVAL, "step: bad arguments");
  if (!c->has_data) return fail(c, SLIM_ESTATE, "step before slim_set_data");
  if (c->lookahead) {
    CK(la_step(c, nsteps), "pipelined step");
    return SLIM_OK;
  }
  if (c->use_graph) {
    if (!c->graph_exec) {
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "capture");
      c->capturing = true;
      cudaError_t e = enqueue_step(c);
      c->capturing = false;
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e, "capture step");
      }
      CK(e2, "end capture");
      c->graph = g;
      CK(cudaGraphInstantiate(&c->graph_exec, g, 0), "instantiate");
    }
    for (int i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(c->graph_exec, c->stream), "graph launch");
  } else {
    for (int i = 0; i < nsteps; ++i) CK(enqueue_step(c), "step");
  }
  c->h_k += nsteps;
  return SLIM_OK;
}

slim_status slim_sync(slim_ctx* c) {
  if (!c) return SLIM_EINVAL;
  if (c->lookahead) CK(la_sync_all(c), "sync");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return read_status(c);
}

slim_status slim_join_stream(slim_ctx* c, void* stream) {
  if (!c) return SLIM_EINVAL;
  cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
  if (c->lookahead && c->gs) {
    // the last record of each event marks the newest work on its stream
    CK(cudaStreamWaitEvent(s, c->ev_g1, 0), "join");
    for (int b = 0; b < c->nbuf; ++b) {
      CK(cudaStreamWaitEvent(s, c->ev_g2[b], 0), "join");
      CK(cudaStreamWaitEvent(s, c->ev_x[b], 0), "join");
    }
  }
  if (s != c->stream) {
    if (!c->ev_user) CK(cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming), "join");
    CK(cudaEventRecord(c->ev_user, c->stream), "join");
    CK(cudaStreamWaitEvent(s, c->ev_user, 0), "join");
  }
  return SLIM_OK;
}

slim_status slim_set_ref(slim_ctx* c, const void* x_ref, size_t n, int dtype, int on_device) {
  if (!c) return SLIM_EINVAL;
  if (!x_ref) {
    if (c->d_ref) cudaFree(c->d_ref);
    c->d_ref = nullptr;
    return SLIM_OK;
  }
  if ((long long)n != c->n || (dtype != SLIM_F32 && dtype != SLIM_F64))
    return fail(c, SLIM_EINVAL, "set_ref: bad arguments");
  if (!c->d_ref) CK(cudaMalloc(&c->d_ref, (size_t)c->n * sizeof(double)), "set_ref");
  CK(copy_in(c->d_ref, 0, x_ref, dtype, on_device, c->n, c->stream), "set_ref");
  CK(cudaStreamSynchronize(c->stream), "set_ref");
  return SLIM_OK;
}

static slim_status eval_err(slim_ctx* c, double* err) {
  CK(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(double), c->stream), "err");
  if (c->precision == SLIM_PREC_FP32)
    CK(launch_rel_err<float>((const float*)c->d_x, c->d_ref, c->n, c->d_err, c->stream), "err");
  else
    CK(launch_rel_err<double>((const double*)c->d_x, c->d_ref, c->n, c->d_err, c->stream), "err");
  double h[2];
  CK(cudaMemcpyAsync(h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "err");
  CK(cudaStreamSynchronize(c->stream), "err");
  *err = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
  return SLIM_OK;
}

slim_status slim_run(slim_ctx* c, long long max_steps, double tol, int eval_every,
                     long long* steps_done, double* seconds, double* final_err) {
  if (!c || max_steps < 0 || eval_every < 1) return fail(c, SLIM_EINVAL, "run: bad arguments");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  long long done = 0;
  double total_ms = 0.0, err = -1.0;
  slim_status st = SLIM_OK;
  while (done < max_steps) {
    int nb = (int)std::min<long long>(eval_every, max_steps - done);
    cudaEventRecord(e0, c->stream);
    if ((st = slim_step(c, nb)) != SLIM_OK) break;
    cudaEventRecord(e1, c->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { st = cuda_fail(c, e, "run"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    total_ms += ms;
    done += nb;
    if ((st = read_status(c)) != SLIM_OK) break;
    if (c->d_ref) {
      if ((st = eval_err(c, &err)) != SLIM_OK) break;
      if (err <= tol) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (steps_done) *steps_done = done;
  if (seconds) *seconds = total_ms * 1e-3;
  if (final_err) *final_err = err;
  return st;
}

slim_status slim_get_iter(const slim_ctx* c, long long* k) {
  if (!c || !k) return SLIM_EINVAL;
  *k = c->h_k;
  return SLIM_OK;
}

slim_status slim_set_iter(slim_ctx* c, long long k) {
  if (!c || k < 0) return fail(c, SLIM_EINVAL, "set_iter: bad arguments");
  if (c->solver == SLIM_SOLVE_OLBFGS) {
    // the pairs depend on the iterates: only a restart from step 0 (no pairs)
    if (k != 0) return fail(c, SLIM_ENOTSUP, "set_iter: olbfgs restarts at 0 only");
    CK(cudaStreamSynchronize(c->stream), "set_iter");
    CK(cudaMemset(c->d_olb_state, 0, (2 + kOlbfgsMaxMem) * sizeof(int)), "set_iter");
  }
  cudaError_t e = c->lookahead ? la_rebuild(c, k)
                 : c->precision == SLIM_PREC_FP32 ? rebuild_t<float>(c, k) : rebuild_t<double>(c, k);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_iter");
  c->h_k = k;
  return read_status(c);
}

namespace {
struct CkptHeader {
  char magic[8];
  long long k, n;
  int precision, version;
};
}  // namespace

slim_status slim_checkpoint(slim_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return SLIM_EINVAL;
  if (c->solver == SLIM_SOLVE_OLBFGS)
    return fail(c, SLIM_ENOTSUP, "checkpoint: the olbfgs pairs are not checkpointed");
  size_t need = sizeof(CkptHeader) + (size_t)c->n * elem(c->precision);
  if (!buf) {
    *len = need;
    return SLIM_OK;
  }
  if (*len < need) return fail(c, SLIM_EINVAL, "checkpoint buffer too small");
  CkptHeader h;
  memcpy(h.magic, "SLIMCKP1", 8);
  h.k = c->h_k;
  h.n = c->n;
  h.precision = c->precision;
  h.version = 1;
  memcpy(buf, &h, sizeof(h));
  CK(cudaMemcpyAsync((char*)buf + sizeof(h), c->d_x, (size_t)c->n * elem(c->precision),
                     cudaMemcpyDeviceToHost, c->stream), "checkpoint");
  CK(cudaStreamSynchronize(c->stream), "checkpoint");
  *len = need;
  return read_status(c);
}

slim_status slim_restore(slim_ctx* c, const void* buf, size_t len) {
  if (!c || !buf || len < sizeof(CkptHeader)) return fail(c, SLIM_EINVAL, "restore: bad buffer");
  if (c->solver == SLIM_SOLVE_OLBFGS)
    return fail(c, SLIM_ENOTSUP, "restore: the olbfgs pairs are not checkpointed");
  CkptHeader h;
  memcpy(&h, buf, sizeof(h));
  if (memcmp(h.magic, "SLIMCKP1", 8) != 0 || h.version != 1 || h.n != c->n ||
      h.precision != c->precision || h.k < 0 ||
      len != sizeof(CkptHeader) + (size_t)c->n * elem(c->precision))
    return fail(c, SLIM_EINVAL, "restore: checkpoint does not match this context");
  CK(cudaMemcpyAsync(c->d_x, (const char*)buf + sizeof(h), (size_t)c->n * elem(c->precision),
                     cudaMemcpyHostToDevice, c->stream), "restore");
  return slim_set_iter(c, h.k);
}

slim_status slim_get_lsqr_info(slim_ctx* c, int* iters, double* normal_res, double* normal_res0) {
  if (!c) return SLIM_EINVAL;
  if (c->solver != SLIM_SOLVE_LSQR) return fail(c, SLIM_ESTATE, "lsqr_info: not an LSQR context");
  CK(cudaStreamSynchronize(c->stream), "lsqr_info");
  double st[3];
  CK(cudaMemcpy(st, c->d_lsqr + (size_t)c->p + 4 * (size_t)c->n + lsqr_part_count(c->num_sms),
                sizeof(st), cudaMemcpyDeviceToHost), "lsqr_info");
  if (iters) *iters = (int)st[0];
  if (normal_res) *normal_res = st[1];
  if (normal_res0) *normal_res0 = st[2];
  return read_status(c);
}

slim_status slim_get_memory(slim_ctx* c, int* ids, double* G, double* z) {
  if (!c) return SLIM_EINVAL;
  if (!c->d_G && (G || z))
    return fail(c, SLIM_ENOTSUP, "get_memory: LSQR keeps no Gram matrix and no z");
  CK(cudaStreamSynchronize(c->stream), "get_memory");
  if (c->lookahead) {
    // gather the window of step h_k from the extended ring into ring order
    CK(la_sync_all(c), "get_memory");
    std::vector<int> ext(c->p);
    for (int q = 0; q < c->p; ++q) ext[q] = la_ext_host(c, c->h_k, q);
    if (ids) {
      std::vector<int> all((size_t)c->Pe);
      CK(cudaMemcpy(all.data(), c->d_ring_ids, all.size() * sizeof(int), cudaMemcpyDeviceToHost),
         "get_memory");
      for (int q = 0; q < c->p; ++q) ids[q] = ext[q] >= 0 ? all[ext[q]] : -1;
    }
    if (G) {
      std::vector<double> row((size_t)c->Pe);
      for (int i = 0; i < c->p; ++i) {
        if (ext[i] < 0) {
          for (int j = 0; j < c->p; ++j) G[(size_t)i * c->p + j] = 0.0;
          continue;
        }
        CK(cudaMemcpy(row.data(), c->d_G + (size_t)ext[i] * c->Pe, row.size() * sizeof(double),
                      cudaMemcpyDeviceToHost), "get_memory");
        for (int j = 0; j < c->p; ++j) G[(size_t)i * c->p + j] = ext[j] >= 0 ? row[ext[j]] : 0.0;
      }
    }
    if (z) {
      // z is in the factored matrix's order (blocks chronological); report it
      // in ring order like ids and G: ring slot s holds block k - d with
      // d = (k-1-s) mod (r+1), at chronological position r - d
      std::vector<double> zf((size_t)c->p);
      CK(cudaMemcpy(zf.data(), c->d_z, zf.size() * sizeof(double), cudaMemcpyDeviceToHost),
         "get_memory");
      for (int q = 0; q < c->p; ++q) {
        const int s = q / c->ell;
        const long long d = ((c->h_k - 1 - s) % c->nslots + c->nslots) % c->nslots;
        z[q] = zf[(size_t)(c->nslots - 1 - d) * c->ell + q % c->ell];
      }
    }
    return read_status(c);
  }
  if (ids) CK(cudaMemcpy(ids, c->d_ring_ids, (size_t)c->p * sizeof(int), cudaMemcpyDeviceToHost),
              "get_memory");
  if (G) CK(cudaMemcpy2D(G, (size_t)c->p * sizeof(double), c->d_G, (size_t)c->P * sizeof(double),
                         (size_t)c->p * sizeof(double), c->p, cudaMemcpyDeviceToHost),
            "get_memory");
  if (z) CK(cudaMemcpy(z, c->d_z, (size_t)c->p * sizeof(double), cudaMemcpyDeviceToHost),
            "get_memory");
  return read_status(c);
}

}  // extern "C"

namespace {
// out[0] += sum (r_i - b_i)^2, out[1] += sum b_i^2
template <typename T>
__global__ void resid_norms_kernel(const T* r, const T* b, long long m, double* out) {
  double e = 0.0, q = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)r[i] - (double)b[i];
    e += d * d;
    q += (double)b[i] * (double)b[i];
  }
  e = warp_sum(e);
  q = warp_sum(q);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], e);
    atomicAdd(&out[1], q);
  }
}

// A^T b of the context's data into a device array of precision T (zeroed first).
template <typename T>
cudaError_t backproject_data_t(slim_ctx* c, T* x) {
  cudaError_t e = cudaMemsetAsync(x, 0, (size_t)c->n * sizeof(T), c->stream);
  if (e != cudaSuccess) return e;
  if (c->a_mode)
    return launch_csr_backproject<T>(c->csr, c->n, nullptr, (int)c->m, (const T*)c->d_b, x, c->stream);
  return launch_backproject<T>(c->d_views, c->N, c->D, nullptr, (int)c->m, (const T*)c->d_b, x,
                               c->stream);
}

template <typename T>
slim_status warm_start_t(slim_ctx* c, slim_unet* net, double s_in, double s_out, int* used,
                         double* ratio) {
  const long long n = c->n, m = c->m;
  T *atb = nullptr, *x0 = nullptr, *r = nullptr;
  float *fin = nullptr, *fout = nullptr;
  double* nrm = nullptr;
  cudaStream_t s = c->stream;
  slim_status st = SLIM_OK;
  auto ck = [&](cudaError_t e, const char* w) {
    if (e != cudaSuccess && st == SLIM_OK) st = cuda_fail(c, e, w);
    return st == SLIM_OK;
  };
  const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
  if (ck(cudaMalloc(&atb, n * sizeof(T)), "warm start") && ck(cudaMalloc(&x0, n * sizeof(T)), "warm start") &&
      ck(cudaMalloc(&r, m * sizeof(T)), "warm start") && ck(cudaMalloc(&fin, n * sizeof(float)), "warm start") &&
      ck(cudaMalloc(&fout, n * sizeof(float)), "warm start") &&
      ck(cudaMalloc(&nrm, 2 * sizeof(double)), "warm start") &&
      ck(backproject_data_t<T>(c, atb), "back-projection")) {
    if (sizeof(T) == 4) {
      ck(unet_scale((const float*)atb, fin, n, (float)s_in, s), "scale");
    } else {
      convert_kernel<T, float><<<grid, 256, 0, s>>>(atb, fin, n);
      ck(cudaGetLastError(), "convert");
      ck(unet_scale(fin, fin, n, (float)s_in, s), "scale");
    }
    if (st == SLIM_OK && slim_unet_forward(net, fin, fout, 1, s) != SLIM_OK)
      st = fail(c, SLIM_ECUDA, "warm start: network forward");
    if (st == SLIM_OK) ck(unet_scale(fout, fout, n, (float)s_out, s), "scale");
    if (st == SLIM_OK) {
      if (sizeof(T) == 4) {
        ck(cudaMemcpyAsync(x0, fout, n * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy");
      } else {
        convert_kernel<float, T><<<grid, 256, 0, s>>>(fout, x0, n);
        ck(cudaGetLastError(), "convert");
      }
    }
    // residual of the guess against the data
    if (st == SLIM_OK) {
      if (c->a_mode)
        ck(launch_csr_project<T>(c->csr, nullptr, (int)m, x0, r, s), "project");
      else
        ck(launch_project<T>(c->d_views, c->N, c->D, nullptr, (int)m, x0, r, s), "project");
    }
    double h[2] = {0.0, 0.0};
    if (st == SLIM_OK && ck(cudaMemsetAsync(nrm, 0, 2 * sizeof(double), s), "norms")) {
      resid_norms_kernel<T><<<(int)std::min<long long>((m + 255) / 256, 4096), 256, 0, s>>>(
          r, (const T*)c->d_b, m, nrm);
      ck(cudaGetLastError(), "norms");
      ck(cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, s), "norms");
      ck(cudaStreamSynchronize(s), "norms");
    }
    if (st == SLIM_OK) {
      const double q = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
      const bool keep = h[1] > 0 && q < 1.0;
      if (ratio) *ratio = q;
      if (used) *used = keep ? 1 : 0;
      if (keep)
        ck(cudaMemcpyAsync(c->d_x, x0, n * sizeof(T), cudaMemcpyDeviceToDevice, s), "set x");
      else
        ck(cudaMemsetAsync(c->d_x, 0, n * sizeof(T), s), "set x");
      ck(cudaStreamSynchronize(s), "warm start");
    }
  }
  cudaFree(atb);
  cudaFree(x0);
  cudaFree(r);
  cudaFree(fin);
  cudaFree(fout);
  cudaFree(nrm);
  return st;
}
}  // namespace

extern "C" {

slim_status slim_warm_start(slim_ctx* c, slim_unet* net, double s_in, double s_out, int* used,
                            double* ratio) {
  if (!c || !net || !(s_in > 0.0) || !(s_out > 0.0)) return fail(c, SLIM_EINVAL, "warm start: bad arguments");
  if (c->dim != 2) return fail(c, SLIM_ENOTSUP, "warm start: 2D only");
  if (unet_height(net) != c->N || unet_width(net) != c->N)
    return fail(c, SLIM_EINVAL, "warm start: network size differs from the image");
  if (!c->has_data) return fail(c, SLIM_ESTATE, "warm start before slim_set_data");
  if (c->lookahead) CK(la_sync_all(c), "sync");
  CK(cudaStreamSynchronize(c->stream), "sync");
  return c->precision == SLIM_PREC_FP32 ? warm_start_t<float>(c, net, s_in, s_out, used, ratio)
                                        : warm_start_t<double>(c, net, s_in, s_out, used, ratio);
}

slim_status slim_backproject_data(slim_ctx* c, float* x) {
  if (!c || !x) return SLIM_EINVAL;
  if (c->dim != 2) return fail(c, SLIM_ENOTSUP, "back-projection of the data: 2D only");
  if (!c->has_data) return fail(c, SLIM_ESTATE, "no data");
  if (c->precision == SLIM_PREC_FP32) {
    CK(backproject_data_t<float>(c, x), "back-projection");
  } else {
    double* tmp = nullptr;
    CK(cudaMalloc(&tmp, (size_t)c->n * sizeof(double)), "back-projection");
    cudaError_t e = backproject_data_t<double>(c, tmp);
    if (e == cudaSuccess) {
      const int grid = (int)std::min<long long>((c->n + 255) / 256, 4096);
      convert_kernel<double, float><<<grid, 256, 0, c->stream>>>(tmp, x, c->n);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    CK(e, "back-projection");
  }
  CK(cudaStreamSynchronize(c->stream), "back-projection");
  return SLIM_OK;
}

slim_status slim_get_csr(slim_ctx* c, long long* nnz, int* row_ptr, int* col, float* val) {
  if (!c || !nnz) return SLIM_EINVAL;
  if (!c->a_mode) return fail(c, SLIM_ESTATE, "the context stores no matrix");
  *nnz = c->csr.nnz;
  CK(cudaStreamSynchronize(c->stream), "get_csr");
  if (row_ptr)
    CK(cudaMemcpy(row_ptr, c->csr.row_ptr, (size_t)(c->m + 1) * sizeof(int), cudaMemcpyDeviceToHost),
       "get_csr");
  if (col)
    CK(cudaMemcpy(col, c->csr.col, (size_t)c->csr.nnz * sizeof(int), cudaMemcpyDeviceToHost),
       "get_csr");
  if (val) {
    if (c->csr.bf16) {
      std::vector<uint16_t> raw((size_t)c->csr.nnz);
      CK(cudaMemcpy(raw.data(), c->csr.val, raw.size() * 2, cudaMemcpyDeviceToHost), "get_csr");
      for (size_t e = 0; e < raw.size(); ++e) {
        uint32_t bits = (uint32_t)raw[e] << 16;
        memcpy(&val[e], &bits, 4);
      }
    } else {
      CK(cudaMemcpy(val, c->csr.val, (size_t)c->csr.nnz * sizeof(float), cudaMemcpyDeviceToHost),
         "get_csr");
    }
  }
  return SLIM_OK;
}

slim_status slim_get_sizes(const slim_ctx* c, long long* n, long long* m, int* p) {
  if (!c) return SLIM_EINVAL;
  if (n) *n = c->n;
  if (m) *m = c->m;
  if (p) *p = c->p;
  return SLIM_OK;
}

slim_status slim_project(slim_ctx* c, const int* ids, int count, const void* x, void* y) {
  if (!c || !x || !y) return fail(c, SLIM_EINVAL, "project: bad arguments");
  if (!ids) count = (int)c->m;
  if (count < 0) return fail(c, SLIM_EINVAL, "project: bad count");
  if (c->general3d) {
    if (c->precision == SLIM_PREC_FP32)
      CK(launch_project_frames<float>(c->d_frames, c->N, c->D, c->Dv, ids, count,
                                      (const float*)x, (float*)y, c->stream), "project");
    else
      CK(launch_project_frames<double>(c->d_frames, c->N, c->D, c->Dv, ids, count,
                                       (const double*)x, (double*)y, c->stream), "project");
    return SLIM_OK;
  }
  if (c->dim == 3) {
    if (c->precision == SLIM_PREC_FP32)
      CK(launch_project_rays<float>(c->d_views, c->N, c->D, c->Dv, ids, count, (const float*)x,
                                    (float*)y, c->stream), "project");
    else
      CK(launch_project_rays<double>(c->d_views, c->N, c->D, c->Dv, ids, count, (const double*)x,
                                     (double*)y, c->stream), "project");
    return SLIM_OK;
  }
  if (c->a_mode) {
    if (c->precision == SLIM_PREC_FP32)
      CK(launch_csr_project<float>(c->csr, ids, count, (const float*)x, (float*)y, c->stream),
         "project");
    else
      CK(launch_csr_project<double>(c->csr, ids, count, (const double*)x, (double*)y, c->stream),
         "project");
    return SLIM_OK;
  }
  if (c->precision == SLIM_PREC_FP32)
    CK(launch_project<float>(c->d_views, c->N, c->D, ids, count, (const float*)x, (float*)y,
                             c->stream), "project");
  else
    CK(launch_project<double>(c->d_views, c->N, c->D, ids, count, (const double*)x, (double*)y,
                              c->stream), "project");
  return SLIM_OK;
}

slim_status slim_backproject(slim_ctx* c, const int* ids, int count, const void* y, void* x) {
  if (!c || !x || !y) return fail(c, SLIM_EINVAL, "backproject: bad arguments");
  if (!ids) count = (int)c->m;
  if (count < 0) return fail(c, SLIM_EINVAL, "backproject: bad count");
  if (c->general3d) {
    if (c->precision == SLIM_PREC_FP32)
      CK(launch_backproject_frames<float>(c->d_frames, c->N, c->D, c->Dv, ids, count,
                                          (const float*)y, (float*)x, c->stream), "backproject");
    else
      CK(launch_backproject_frames<double>(c->d_frames, c->N, c->D, c->Dv, ids, count,
                                           (const double*)y, (double*)x, c->stream), "backproject");
    return SLIM_OK;
  }
  if (c->dim == 3) return fail(c, SLIM_ENOTSUP, "backproject: 2D only");
  if (c->a_mode) {
    if (c->precision == SLIM_PREC_FP32)
      CK(launch_csr_backproject<float>(c->csr, c->n, ids, count, (const float*)y, (float*)x,
                                       c->stream), "backproject");
    else
      CK(launch_csr_backproject<double>(c->csr, c->n, ids, count, (const double*)y, (double*)x,
                                        c->stream), "backproject");
    return SLIM_OK;
  }
  if (c->precision == SLIM_PREC_FP32)
    CK(launch_backproject<float>(c->d_views, c->N, c->D, ids, count, (const float*)y, (float*)x,
                                 c->stream), "backproject");
  else
    CK(launch_backproject<double>(c->d_views, c->N, c->D, ids, count, (const double*)y,
                                  (double*)x, c->stream), "backproject");
  return SLIM_OK;
}

}  // extern "C"

namespace {
__global__ void damped_form_kernel(const double* G, int p, double lam, double* L, int P) {
  long long total = (long long)P * P;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx / P), j = (int)(idx % P);
    double v = 0.0;
    if (i < p && j < p) v = G[(size_t)i * p + j] + (i == j ? lam : 0.0);
    else if (i == j) v = 1.0;
    L[idx] = v;
  }
}
}  // namespace

extern "C" slim_status slim_damped_solve(const double* G, int p, double lambda, const double* rhs,
                                         double* z, void* stream) {
  if (!G || !rhs || !z || p <= 0 || p > 65536 || !(lambda >= 0.0)) return SLIM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = 32;
  const int P = (p + nb - 1) / nb * nb;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SLIM_ECUDA;
  CholPlan plan;
  double *L = nullptr, *v = nullptr, *out = nullptr;
  int* status = nullptr;
  slim_status st = SLIM_OK;
  cudaError_t e = chol_plan_create(&plan, P, nb, 0, sms, 2);
  if (e == cudaSuccess) e = cudaMalloc(&L, (size_t)P * P * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&v, (size_t)P * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)P * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, (size_t)P * sizeof(double), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(v, rhs, (size_t)p * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) {
    int grid = (int)std::min<long long>(((long long)P * P + 255) / 256, 152LL * 16);
    damped_form_kernel<<<grid, 256, 0, s>>>(G, p, lambda, L, P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = chol_factor(plan, L, status, s);
  if (e == cudaSuccess) e = chol_solve(plan, L, v, out, status, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(z, out, (size_t)p * sizeof(double), cudaMemcpyDeviceToDevice, s);
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? SLIM_ENOMEM : SLIM_ECUDA;
  else if (hs != 0) st = (slim_status)hs;
  cudaFree(L);
  cudaFree(v);
  cudaFree(out);
  cudaFree(status);
  chol_plan_destroy(&plan);
  return st;
}

// ---------------------------------------------------------------------------
// Autotuner and batched form
// ---------------------------------------------------------------------------
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

namespace {

// size class: dimension, block kind, precisions and the order p of the Gram
// system rounded up to a multiple of 512 (the choice depends on p alone)
struct TuneKey {
  int dim, kind, precision, solver, pclass;
  bool operator<(const TuneKey& o) const {
    return std::tie(dim, kind, precision, solver, pclass) <
           std::tie(o.dim, o.kind, o.precision, o.solver, o.pclass);
  }
  std::string str() const {
    std::ostringstream os;
    os << dim << ' ' << kind << ' ' << precision << ' ' << solver << ' ' << pclass;
    return os.str();
  }
};
struct TuneVal {
  int tile, ctas;
  double ms;
  int lanes = 0, window = 0;   // random-ray mapping (0: the defaults)
};
std::map<TuneKey, TuneVal> g_tune;
std::mutex g_tune_mu;

// One entry per line: the key's five fields, tile, CTAs per SM, ms, threads
// per ray, pair window (lines of another layout are skipped).
void load_tune_file() {
  const char* path = std::getenv("SLIM_AUTOTUNE_CACHE");
  if (!path) return;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    TuneKey k;
    TuneVal v;
    std::string extra;
    if ((is >> k.dim >> k.kind >> k.precision >> k.solver >> k.pclass >> v.tile >> v.ctas >> v.ms >>
         v.lanes >> v.window) &&
        !(is >> extra))
      g_tune[k] = v;
  }
}

void save_tune_entry(const TuneKey& k, const TuneVal& v) {
  const char* path = std::getenv("SLIM_AUTOTUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << k.str() << ' ' << v.tile << ' ' << v.ctas << ' ' << v.ms << ' ' << v.lanes << ' '
    << v.window << '\n';
}

// Mean step time of a temporary context with options o (1e30 on failure):
// r + 1 untimed steps, then `steps` timed on the context's stream.
double time_options(const slim_geometry* geom, const slim_blocks* blocks, int r, double lambda,
                    const slim_step_opts& o, int steps, const std::vector<double>& b) {
  slim_ctx* c = nullptr;
  if (slim_create(geom, blocks, r, lambda, &o, &c) != SLIM_OK) return 1e30;
  double ms = 1e30;
  if (slim_set_data(c, b.data(), b.size(), SLIM_F64, 0) == SLIM_OK &&
      slim_step(c, r + 1) == SLIM_OK && slim_sync(c) == SLIM_OK) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    slim_step(c, steps);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    if (slim_sync(c) == SLIM_OK) ms = f / steps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  slim_destroy(c);
  return ms;
}

}  // namespace

extern "C" slim_status slim_autotune(const slim_geometry* geom, const slim_blocks* blocks, int r,
                                     double lambda, const slim_step_opts* base, int steps,
                                     slim_step_opts* best, double* best_ms) {
  if (!geom || !blocks || !best || steps < 1) return SLIM_EINVAL;
  slim_step_opts b0 = base ? *base : slim_step_opts{1.0, 0, SLIM_SOLVE_FP64, 2, 0, 0, 0, 0};
  *best = b0;
  if (geom->dim == 3) {   // per-slice solves: nothing to tune here
    if (best_ms) *best_ms = 0.0;
    return SLIM_OK;
  }
  const int p = (r + 1) * blocks->ell;
  TuneKey key{geom->dim, blocks->kind, geom->precision, b0.solver, (p + 511) / 512};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    static bool loaded = false;
    if (!loaded) {
      load_tune_file();
      loaded = true;
    }
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      best->tile = it->second.tile;
      best->ctas_per_sm = it->second.ctas;
      best->ray_lanes = it->second.lanes;
      best->pair_window = it->second.window;
      if (best_ms) *best_ms = it->second.ms;
      return SLIM_OK;
    }
  }
  const int tiles[2] = {32, 64};
  const int ctas[3] = {1, 2, 3};
  TuneVal bestv{0, 0, 1e30};
  std::vector<double> b((size_t)geom->n_views * geom->det_u * geom->det_v, 0.0);
  for (int t : tiles) {
    for (int cps : ctas) {
      slim_step_opts o = b0;
      o.tile = t;
      o.ctas_per_sm = cps;
      o.use_graph = 1;
      const double ms = time_options(geom, blocks, r, lambda, o, steps, b);
      if (ms < bestv.ms)
        bestv = TuneVal{t, cps, ms, b0.ray_lanes ? b0.ray_lanes : 32,
                        b0.pair_window ? b0.pair_window : 32};
    }
  }
  if (bestv.tile == 0) return SLIM_ECUDA;
  // 2D random-ray blocks: threads per ray of the march and scatter, and the
  // pair Gram's cut-off, with the factorisation options just chosen
  if (blocks->kind != SLIM_BLOCKS_VIEWS) {
    for (int lanes : {8, 16, 32}) {
      for (int window : {16, 32, 64}) {
        slim_step_opts o = b0;
        o.tile = bestv.tile;
        o.ctas_per_sm = bestv.ctas;
        o.use_graph = 1;
        o.ray_lanes = lanes;
        o.pair_window = window;
        const double ms = time_options(geom, blocks, r, lambda, o, steps, b);
        if (ms < bestv.ms) {
          bestv.ms = ms;
          bestv.lanes = lanes;
          bestv.window = window;
        }
      }
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = bestv;
    save_tune_entry(key, bestv);
  }
  best->tile = bestv.tile;
  best->ctas_per_sm = bestv.ctas;
  best->ray_lanes = bestv.lanes;
  best->pair_window = bestv.window;
  if (best_ms) *best_ms = bestv.ms;
  return SLIM_OK;
}

struct slim_batch {
  std::vector<slim_ctx*> ctx;
  std::vector<cudaEvent_t> join, join2;
  cudaEvent_t fork = nullptr, fork2 = nullptr;
  // the problems' tiled factorisations, one merged persistent launch per
  // factor precision and tile size
  std::vector<slim::CholBatch> groups;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
void batch_drop_graph(slim_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}
}  // namespace

extern "C" void slim_batch_destroy(slim_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  for (slim_ctx* c : b->ctx) slim_destroy(c);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->join2)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->fork2) cudaEventDestroy(b->fork2);
  for (slim::CholBatch& g : b->groups) slim::chol_batch_destroy(&g);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

extern "C" slim_status slim_batch_create(int count, const slim_geometry* geoms,
                                         const slim_blocks* blocks, const int* r,
                                         const double* lambda, const slim_step_opts* steps,
                                         slim_batch** out) {
  if (!out || count < 1 || !geoms || !blocks || !r || !lambda) return SLIM_EINVAL;
  *out = nullptr;
  slim_batch* b = new (std::nothrow) slim_batch();
  if (!b) return SLIM_ENOMEM;
  for (int i = 0; i < count; ++i) {
    slim_ctx* c = nullptr;
    slim_status st = slim_create(&geoms[i], &blocks[i], r[i], lambda[i], steps ? &steps[i] : nullptr,
                                 &c);
    if (st != SLIM_OK) {
      slim_batch_destroy(b);
      return st;
    }
    if (c->lookahead || c->solver >= SLIM_SOLVE_LSQR) {   // a batch captures one plain chain per problem
      slim_destroy(c);
      slim_batch_destroy(b);
      return SLIM_ENOTSUP;
    }
    c->use_graph = 0;   // the batch captures the steps itself
    b->ctx.push_back(c);
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      slim_batch_destroy(b);
      return SLIM_ECUDA;
    }
    b->join.push_back(e);
    e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      slim_batch_destroy(b);
      return SLIM_ECUDA;
    }
    b->join2.push_back(e);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    slim_batch_destroy(b);
    return SLIM_ECUDA;
  }
  b->own_stream = true;
  // The problems' tiled factorisations run as one persistent launch per
  // factor precision and tile size, their task lists merged into one queue:
  // every CTA of the GPU works on whichever problem has a ready task.
  for (int is_f32 = 0; is_f32 < 2; ++is_f32)
    for (int nb : {32, 64}) {
      std::vector<const CholPlan*> plans;
      std::vector<void*> Ls;
      std::vector<int*> sts;
      for (slim_ctx* c : b->ctx)
        if (c->plan.T > 0 && c->plan.is_f32 == is_f32 && c->plan.nb == nb) {
          plans.push_back(&c->plan);
          Ls.push_back(c->d_L);
          sts.push_back(c->d_status);
        }
      if (plans.empty()) continue;
      slim::CholBatch g;
      // throughput-bound: two CTAs per SM at 128 registers keep more tasks in flight
      if (slim::chol_batch_create(&g, plans, Ls, sts, b->ctx[0]->num_sms, 2) != cudaSuccess) {
        slim::chol_batch_destroy(&g);
        slim_batch_destroy(b);
        return SLIM_ECUDA;
      }
      b->groups.push_back(g);
    }
  *out = b;
  return SLIM_OK;
}

extern "C" slim_status slim_batch_ctx(slim_batch* b, int i, slim_ctx** ctx) {
  if (!b || !ctx || i < 0 || i >= (int)b->ctx.size()) return SLIM_EINVAL;
  *ctx = b->ctx[i];
  return SLIM_OK;
}

extern "C" slim_status slim_batch_set_stream(slim_batch* b, void* stream) {
  if (!b) return SLIM_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SLIM_ECUDA;
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->own_stream = false;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return SLIM_ECUDA;
    b->own_stream = true;
  }
  batch_drop_graph(b);
  return SLIM_OK;
}

extern "C" slim_status slim_batch_step(slim_batch* b, int nsteps) {
  if (!b || nsteps < 0) return SLIM_EINVAL;
  for (slim_ctx* c : b->ctx)
    if (!c->has_data) return SLIM_ESTATE;
  if (!b->exec) {
    // one graph in three parts: a parallel branch per problem up to its
    // K = lambda I + G; the merged factorisation launches; a parallel branch
    // per problem from its solves on
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return SLIM_ECUDA;
    cudaError_t e = cudaSuccess;
    for (int stage = 1; stage <= 2 && e == cudaSuccess; ++stage) {
      cudaEvent_t fork = stage == 1 ? b->fork : b->fork2;
      std::vector<cudaEvent_t>& join = stage == 1 ? b->join : b->join2;
      e = cudaEventRecord(fork, b->stream);
      for (size_t i = 0; i < b->ctx.size() && e == cudaSuccess; ++i) {
        slim_ctx* c = b->ctx[i];
        e = cudaStreamWaitEvent(c->stream, fork, 0);
        if (e == cudaSuccess) {
          c->capturing = true;
          c->stage = stage;
          e = enqueue_step(c);
          c->stage = 0;
          c->capturing = false;
        }
        if (e == cudaSuccess) e = cudaEventRecord(join[i], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, join[i], 0);
      }
      if (stage == 1)
        for (size_t g = 0; g < b->groups.size() && e == cudaSuccess; ++g)
          e = chol_factor_batch(b->groups[g], b->stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return SLIM_ECUDA;
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      batch_drop_graph(b);
      return SLIM_ECUDA;
    }
  }
  // order the graph after work already queued on each problem's own stream
  // (set_data, set_x, ...), and later work there after the graph
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (cudaEventRecord(b->join[i], b->ctx[i]->stream) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->join[i], 0) != cudaSuccess)
      return SLIM_ECUDA;
  }
  for (int i = 0; i < nsteps; ++i)
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return SLIM_ECUDA;
  if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return SLIM_ECUDA;
  for (slim_ctx* c : b->ctx) {
    if (cudaStreamWaitEvent(c->stream, b->fork, 0) != cudaSuccess) return SLIM_ECUDA;
    c->h_k += nsteps;
  }
  return SLIM_OK;
}

extern "C" slim_status slim_batch_sync(slim_batch* b) {
  if (!b) return SLIM_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SLIM_ECUDA;
  slim_status st = SLIM_OK;
  for (slim_ctx* c : b->ctx) {
    slim_status s2 = read_status(c);
    if (st == SLIM_OK) st = s2;
  }
  return st;
}
