/*
 * slim.h -- C ABI of the GB300 slimLS library (libslim.so).
 *
 * The sampled limited-memory row-action method for least squares
 * (Chung, Chung, Slagel, Tenorio, arXiv:1912.07962), Sec. 1, Eq. (ram)/(B_k):
 *
 *     x_k = x_{k-1} - eta * B_k A_k^T (A_k x_{k-1} - b_k),
 *     B_k = (lambda_k I + M_k^T M_k)^{-1},   M_k = [A_{k-r}; ...; A_k],
 *
 * with C_k = I and lambda_k = 1/alpha_k.  A is a parallel-beam tomography
 * forward model (Sec. 4.3) whose rows are generated on the device by a Joseph
 * ray-driven projector; it is never stored (Sec. 4.2: blocks are function
 * evaluations).  A block A_k is one projection view (the tomography blocks of
 * Sec. 4.3), drawn i.i.d. uniformly (Sec. 1, the sampling W_k).
 *
 * Each step runs on the device, in the context's CUDA stream:
 *   1. sample tau_k (counter-based SplitMix64; no host round trip);
 *   2. r_k = A_k x_{k-1} - b_k, storing the block's rows in a ring of r+1 slots;
 *   3. G = M_k M_k^T, updating only the new block's rows and columns;
 *   4. (lambda_k I + G) z = [0;...;r_k;...;0] by a tiled Cholesky factorisation
 *      (Sec. 2's Sherman-Woodbury identity turns the n x n solve of Eq. (B_k)
 *      into this p x p one, p = (r+1) * ell);
 *   5. x -= eta * M_k^T z.
 *
 * Conventions
 *   - Every call returns a slim_status; the library never aborts and never
 *     traps the device.  Device-side failures (a non-positive pivot, a bounded
 *     wait that ran out) are recorded in a device status word and returned
 *     by the next synchronising call (slim_sync, slim_get_x, slim_run, ...).
 *   - Pointers are host pointers unless an `on_device` flag says otherwise or
 *     the argument is documented as a device pointer.  All inputs are copied;
 *     the caller keeps ownership of its buffers.
 *   - dtype: SLIM_F32 = 0 (float), SLIM_F64 = 1 (double).
 *   - Image layout: x[iy*N + ix] (2D).  Data layout: b[view*det_u + bin]
 *     (view-major).  Ray id = view*det_u + bin.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef SLIM_H_
#define SLIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slim_ctx slim_ctx;

typedef enum {
  SLIM_OK = 0,
  SLIM_EINVAL = 1,   /* an argument is out of range or inconsistent */
  SLIM_ENOMEM = 2,   /* a device or host allocation failed */
  SLIM_ECUDA = 3,    /* a CUDA runtime call failed (message in slim_last_error) */
  SLIM_ENOTPD = 4,   /* lambda_k I + G is not positive definite (Cholesky pivot <= 0) */
  SLIM_ETIMEOUT = 5, /* a bounded device-side wait ran out; results are invalid */
  SLIM_ESTATE = 6,   /* call order: e.g. a step before slim_set_data */
  SLIM_ENOTSUP = 7   /* a valid but unsupported combination of options */
} slim_status;

enum { SLIM_F32 = 0, SLIM_F64 = 1 };
enum { SLIM_PREC_FP64 = 0, SLIM_PREC_FP32 = 1 };
enum { SLIM_SOLVE_FP64 = 0, SLIM_SOLVE_MIXED = 1, SLIM_SOLVE_LSQR = 2, SLIM_SOLVE_SG = 3,
       SLIM_SOLVE_OLBFGS = 4, SLIM_SOLVE_MIXED_TC = 5, SLIM_SOLVE_MIXED_INV = 6 };
enum { SLIM_BLOCKS_VIEWS = 0, SLIM_BLOCKS_RAYS = 1, SLIM_BLOCKS_STREAM = 2 };

/* Parallel-beam geometry (Sec. 4.3; Joseph rows defined in the library docs).
 *   dim        2 (image N x N) or 3 (volume N x N x N, x[(iz*N + iy)*N + ix],
 *              views rotating about z)
 *   n_side     N
 *   n_views    A_v projection angles
 *   det_u      D detector bins per view row, unit spacing, centred
 *   det_v      1 in 2D; in 3D (no frames) the detector rows, which must equal N: row v
 *              then lies in z-slice v, rays of different slices share no voxel
 *              and the Gram matrix is block diagonal by slice
 *   angles     host array [n_views] of radians, or NULL for theta_a = a*pi/A_v
 *   a_mode     0: rows generated on the fly by the projector (matrix-free);
 *              1: all of A built once on the device and stored as CSR (plus a
 *                 CSC copy) with float32 values; 2: the same with bfloat16
 *                 values (Sec. 4.2: blocks may be stored when A fits in memory).
 *                 The step then reads its rows from the stored matrix, and the
 *                 method runs on that (rounded) A: residual, Gram and scatter
 *                 all use the stored values.
 *   frames     3D only: NULL (views rotate about z, as above), or a host
 *              array [n_views * 9] of per-view frames (d, u, v) for views from
 *              arbitrary directions (Sec. 4.3: directions uniform on the unit
 *              sphere): d the unit ray direction, (u, v) an orthonormal
 *              detector basis perpendicular to it (SLIM_EINVAL otherwise,
 *              1e-9).  Ray (a, v, uu), id (a*Dv + v)*Du + uu, passes through
 *              t_u u + t_v v (t_u = uu - (Du-1)/2, t_v = v - (Dv-1)/2) from the
 *              volume's centre; Joseph's rows march it along k = argmax |d_c|
 *              with bilinear taps in the other two axes (four per slice,
 *              weights times |1/d_k|).  Any det_v.  Random-ray blocks only
 *              (SLIM_BLOCKS_RAYS / _STREAM); the Gram matrix comes from
 *              voxel lists and the damped solve is the tiled dense one
 *              (FP64 or MIXED solver, lookahead 0)
 *   precision  SLIM_PREC_FP64: x, b, residual and scatter in float64;
 *              SLIM_PREC_FP32: x, b, residual and scatter in float32 with float32
 *              accumulation.  The Gram matrix is float64 in both. */
typedef struct {
  int dim;
  int n_side;
  int n_views;
  int det_u;
  int det_v;
  const double* angles;
  int a_mode;
  int precision;
  const double* frames;
} slim_geometry;

/* Block sampling (Sec. 1: W_k i.i.d. uniform over M selectors).
 *   kind   SLIM_BLOCKS_VIEWS (2D): one view per block, M = n_views, drawn
 *          uniformly with replacement; ell must equal det_u.  Step k draws view
 *          bounded(draw(seed, 2, k-1), A_v) (with `cyclic`, the random cyclic
 *          order below instead).
 *          SLIM_BLOCKS_RAYS: ell rays, each uniform over all m rays.
 *          SLIM_BLOCKS_STREAM (streaming data, Sec. 4.3): views arrive in angle
 *          order, view v from step steps_per_view*v + 1; each of the ell rays is
 *          uniform over the rays of the views that have arrived.  Ray i of step
 *          k is bounded(draw(seed, 3, (k-1)*ell + i), available rays).
 *   ell    rows per block
 *   seed   generator seed
 *   steps_per_view  SLIM_BLOCKS_STREAM only
 *   with_replacement  1 (every configuration here): draws are independent, so
 *          a view may recur within an epoch and a ray within a random-ray
 *          block (Sec. 1's i.i.d. W_k).  0: without replacement -- view
 *          blocks then follow the random cyclic order (as cyclic = 1), and
 *          the ell rays of a random-ray block are distinct: Floyd's algorithm
 *          (Bentley and Floyd 1987) over the available rays, draw i of step k
 *          bounded(draw(seed, 3, (k-1)*ell + i), n_avail - ell + i + 1), the
 *          ids in the algorithm's insertion order (ell <= 2048 and ell <= the
 *          rays of one view for SLIM_BLOCKS_STREAM, of all views for
 *          SLIM_BLOCKS_RAYS; SLIM_ENOTSUP / SLIM_EINVAL otherwise)
 *   cyclic SLIM_BLOCKS_VIEWS only (SLIM_ENOTSUP otherwise): 1 = random cyclic
 *          order (the walnut experiment of Sec. 4.3): epoch e = (k-1) / A_v
 *          visits every view once, in the order of the Fisher-Yates shuffle
 *          of 0..A_v-1 whose swap i (i = A_v-1 down to 1) exchanges entries i
 *          and bounded(draw(seed, 7, e*A_v + A_v-1-i), i+1); step k takes
 *          entry (k-1) mod A_v.  A_v <= 4096 (SLIM_ENOTSUP otherwise). */
typedef struct {
  int kind;
  int ell;
  unsigned long long seed;
  int steps_per_view;
  int with_replacement;
  int cyclic;
} slim_blocks;

/* Step options.
 *   eta           extra step size multiplying s_k (1 = Eq. (ram))
 *   ramp          1: lambda_k = lambda*(r+1)/k for k <= r+1 (the damping ramp of Sec. 4.2)
 *   solver        SLIM_SOLVE_FP64: float64 tiled Cholesky and triangular solves;
 *                 SLIM_SOLVE_MIXED: float32 tiled Cholesky of the same float64
 *                 matrix, then `refine_iters` rounds of iterative refinement whose
 *                 residual (lambda_k I + G) z is computed in float64
 *                 SLIM_SOLVE_MIXED_TC: a float32 factor with the same float64
 *                 refinement, built on the tcgen05 tensor cores with
 *                 float32-accurate split-bfloat16 products (as slim_tc_matmul):
 *                 the geometry chain factors panel by panel (a one-CTA
 *                 diagonal tile, then the panel and the trailing update as
 *                 tensor-core products) and forms X = L^{-1} (recursive
 *                 blocking, X21 = -X22 L21 X11) while it runs ahead; every
 *                 solve of the iterate chain is z = X^T (X v), two
 *                 matrix-vector products instead of two chains of triangular
 *                 sweeps.
 *                 lookahead >= 1 and tile 0 or 64 only (SLIM_ENOTSUP
 *                 otherwise)
 *                 SLIM_SOLVE_MIXED_INV: as SLIM_SOLVE_MIXED_TC, with the
 *                 factor from the persistent tiled factorisation of
 *                 SLIM_SOLVE_MIXED (one launch) and only X = L^{-1} formed by
 *                 tensor-core products; same limits
 *                 SLIM_SOLVE_LSQR: no Gram matrix and no factorisation: s_k of
 *                 Eq. (slimLSstep) by LSQR for damped least squares (Sec. 4.2),
 *                 matrix-free over the window's stored taps, float64 vectors;
 *                 2D view blocks, rows from the projector, lookahead 0 only
 *                 (SLIM_ENOTSUP otherwise), never captured in a graph.  With
 *                 C_k = diag(c) and/or tik_lambda it runs on the columns
 *                 scaled by c^{-1/2} with damping sqrt(mu_k) and right-hand
 *                 side c - (beta/mu_k) M_k x (the same step)
 *                 SLIM_SOLVE_SG: the comparator sg of Sec. 2, B_k = alpha_k I in
 *                 Eq. (ram): x_k = x_{k-1} - eta alpha_k A_k^T r_k with the step
 *                 size alpha_k = 1/lambda_k (lambda_k from the damping schedule)
 *                 SLIM_SOLVE_OLBFGS: the comparator olbfgs of Sec. 4.1 (online
 *                 L-BFGS, memory olbfgs_memory): x_k = x_{k-1} - eta alpha_k H_k g_k,
 *                 g_k = A_k^T r_k, H_k the L-BFGS inverse of the last pairs
 *                 (s_j = x_j - x_{j-1}, y_j = A_j^T A_j s_j) from H^0 = gamma_k I,
 *                 gamma_k the mean of s^T y / y^T y over the stored pairs (I
 *                 before the first); a pair with s^T y <= 0 is not stored.
 *                 SG and OLBFGS keep no slimLS memory: r must be 0
 *                 (SLIM_EINVAL); 2D view blocks, lookahead 0, tik_lambda 0
 *                 (SLIM_ENOTSUP otherwise); OLBFGS is one cooperative launch
 *                 per step, never captured in a graph
 *   refine_iters  refinement rounds for the SLIM_SOLVE_MIXED* solvers (0..16)
 *   use_graph     1: capture one step as a CUDA graph at the first slim_step and
 *                 replay it (one graph launch per step)
 *   tile          tile size of the tiled Cholesky: 32 or 64, 0 = default (64 for
 *                 the float32 factor, 32 for float64)
 *   ctas_per_sm   resident CTAs per SM of the persistent factorisation (1..4,
 *                 0 = chosen by the library: 1 for float32 factors of up to 96
 *                 tiles a side, else 2): 1 gives each CTA the whole register
 *                 file, 2..4 cap it at 128 registers a thread.  With lookahead the D
 *                 factorisations in flight share num_SMs * ctas_per_sm CTAs at
 *                 128 registers a thread (num_SMs * ctas_per_sm / D each), which
 *                 leaves room on the SMs for the iterate chain
 *   lookahead     0: each step runs as one chain.  D = 1..10 (view blocks, 2D,
 *                 rows from the projector): the matrix lambda_k I + M_k M_k^T of
 *                 Eq. (B_k) depends only on the blocks drawn, so the chain that
 *                 draws tau_j, adds its Gram rows and factors K_j runs up to D
 *                 steps ahead of the chain that updates x, on streams of its
 *                 own.  The iterates are the same; slim_step returns with the
 *                 update of x enqueued on the context's stream and the
 *                 geometry of up to D later steps in flight on internal
 *                 streams (slim_sync waits for those too).  Uses graphs
 *                 whatever use_graph says.
 *   lsqr_max_iter SLIM_SOLVE_LSQR: iterations per step at most (1..1000000)
 *   lsqr_tol      SLIM_SOLVE_LSQR: stop once ||M_k^T (c - M_k s) - lambda_k s||
 *                 <= lsqr_tol ||M_k^T c|| (LSQR's estimate; 0: lsqr_max_iter
 *                 iterations exactly)
 *   tik_lambda    slimTik (Sec. 2, Eq. slimTik): slimLS applied to the Tikhonov
 *                 problem min ||A x - b||^2 + tik_lambda^2 ||L x||^2 (Eq. TLS1)
 *                 with C_k = L^T L (set by slim_set_c_diag, default I) and
 *                 M = A_v blocks:
 *                   x_k = x_{k-1} - (mu_k C + M_k^T M_k)^{-1}
 *                         (A_k^T (A_k x_{k-1} - b_k) + beta C x_{k-1}),
 *                   beta = tik_lambda^2 / A_v,  mu_k = lambda_k + c_k beta.
 *                 0 = plain slimLS.  2D view blocks, Woodbury form (FP64 or
 *                 MIXED solver) or LSQR (SLIM_ENOTSUP otherwise), with or without
 *                 lookahead (mu_k I + M_k C^{-1} M_k^T depends only on the
 *                 blocks drawn)
 *   decay_after   0: lambda_k as above.  K > 0: the decaying damping of Sec. 3
 *                 (after a constant one): lambda_k = lambda k / K for k > K
 *                 (alpha_k = alpha K / k), every solver
 *   olbfgs_memory SLIM_SOLVE_OLBFGS: pairs kept (1..20, 0 = 10)
 *   tik_reading   c_k, the Tikhonov rows that the stacked M_k holds: 0 = the
 *                 blocks of M_k, min(k, r+1) (slimLS on the stacked problem,
 *                 whose full-memory iterates reach the Tikhonov solution);
 *                 1 = r, as Eq. (slimTik) prints it
 *   ray_lanes     random-ray blocks: threads per ray of the ray march with
 *                 the residual and of the scatter, 8, 16 or 32 (0 = 32); a
 *                 warp then serves 32 / ray_lanes rays (SLIM_EINVAL otherwise)
 *   pair_window   2D random-ray blocks: the pair-overlap Gram gives each pair
 *                 of rays one thread, and pairs whose overlap window is longer
 *                 than pair_window steps (near-parallel rays) the whole warp;
 *                 8..256 (0 = 32; SLIM_EINVAL otherwise)
 *                 (both change only the order of floating-point sums) */
typedef struct {
  double eta;
  int ramp;
  int solver;
  int refine_iters;
  int use_graph;
  int tile;
  int ctas_per_sm;
  int lookahead;
  int lsqr_max_iter;
  double lsqr_tol;
  double tik_lambda;
  int tik_reading;
  int decay_after;
  int olbfgs_memory;
  int ray_lanes;
  int pair_window;
} slim_step_opts;

/* SLIM_SOLVE_LSQR: the last step's LSQR iterations, its final estimate of
 * ||M_k^T (c - M_k s) - lambda_k s|| and ||M_k^T c|| (synchronises).
 * SLIM_ESTATE for another solver. */
slim_status slim_get_lsqr_info(slim_ctx* ctx, int* iters, double* normal_res,
                               double* normal_res0);

/* Create a context: validates the arguments and allocates all device state
 * (x, b, the ring of r+1 blocks, G and its factor).  r is the memory of
 * Eq. (B_k) (M_k holds r+1 blocks), lambda > 0 the damping 1/alpha.
 * `step` may be NULL (eta 1, no ramp, FP64 solver, no graph).
 * On success *out owns the context; release it with slim_destroy. */
slim_status slim_create(const slim_geometry* geom, const slim_blocks* blocks, int r,
                        double lambda, const slim_step_opts* step, slim_ctx** out);

/* Release every resource of the context (NULL is a no-op). */
void slim_destroy(slim_ctx* ctx);

/* Human-readable text of the last error on this context (never NULL). */
const char* slim_last_error(const slim_ctx* ctx);

/* Run subsequent work on `cuda_stream` (a cudaStream_t; NULL = the context's own). */
slim_status slim_set_stream(slim_ctx* ctx, void* cuda_stream);

/* b (Eq. inverseproblem), m = n_views*det_u values, copied (converted to the
 * context precision).  Must precede slim_step. */
slim_status slim_set_data(slim_ctx* ctx, const void* b, size_t m, int dtype, int on_device);

/* x_0 (default 0), n values, copied.  Does not change the step counter. */
slim_status slim_set_x(slim_ctx* ctx, const void* x, size_t n, int dtype, int on_device);

/* C_k = diag(c) of Eq. (B_k), constant over k (C_k = L^T L with L = diag(sqrt c)
 * in slimTik), n values > 0 and finite (host or device, SLIM_F32/SLIM_F64),
 * copied; NULL restores C_k = I.  The step becomes
 *   x_k = x_{k-1} - (lambda_k C + M_k^T M_k)^{-1} A_k^T r_k  (plus the slimTik
 * terms when tik_lambda > 0), computed as (mu_k I + M_k C^{-1} M_k^T) z = rhs,
 * x_k = (1 - eta beta/mu_k) x_{k-1} - eta C^{-1} M_k^T z.  The memory of the
 * steps taken so far is rebuilt with the new C (with lookahead, the steps
 * prepared ahead are prepared again).  2D view blocks, Woodbury or LSQR form
 * (SLIM_ENOTSUP otherwise); SLIM_EINVAL if a value is not positive.
 * Synchronises. */
slim_status slim_set_c_diag(slim_ctx* ctx, const void* c, size_t n, int dtype, int on_device);

/* slimTik (Eq. slimTik) with C_k = L^T L for a lower-bidiagonal L on the
 * image vector: (L x)_i = d0_i x_i + d1_i x_{i-1} (d1_0 unused), e.g. the
 * first difference along the image rows plus a multiple of the identity.  L
 * must be invertible (every d0_i nonzero and finite; SLIM_EINVAL otherwise).
 * The Woodbury form keeps a p x p system with W = C^{-1} = L^{-1} L^{-T}:
 *   (mu_k I + M_k W M_k^T) z = c - (beta/mu_k) M_k x_{k-1},
 *   x_k = (1 - eta beta/mu_k) x_{k-1} - eta W M_k^T z
 * (with tik_lambda = 0: slimLS with this C_k, beta = 0).  Each step applies W
 * to the new block's ell rows and to M_k^T z; W v is two first-order
 * recurrences (L^T t = v backward, L u = t forward), each a chunked affine
 * scan in one thread block.  d0, d1: n values each (host, or device with
 * on_device = 1), copied; d1 may be NULL (L diagonal); d0 = NULL restores
 * C_k = I.  Replaces a diagonal C_k of slim_set_c_diag (and is replaced by
 * one).  2D view blocks, rows from the projector, FP64 or MIXED solver,
 * lookahead 0 (SLIM_ENOTSUP otherwise).  The memory of the steps taken so far
 * is rebuilt.  Synchronises. */
slim_status slim_set_tik_bidiag(slim_ctx* ctx, const double* d0, const double* d1, size_t n,
                                int on_device);

/* Failure detection self-test: runs a grid barrier (the bounded wait of the
 * cooperative solvers) that one of its two CTAs never reaches, on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream), and
 * returns the status the waiting CTA recorded when its poll limit ran out
 * (about a second): SLIM_ETIMEOUT is the expected outcome.  The kernel ends
 * either way and the device stays usable.  Synchronises the stream. */
slim_status slim_selftest_wait(void* cuda_stream);

/* Copy the current iterate into the caller's buffer (synchronises; returns
 * any device-side error recorded since the last synchronising call). */
slim_status slim_get_x(slim_ctx* ctx, void* x, size_t n, int dtype, int on_device);

/* Enqueue nsteps iterations of Eq. (ram) on the context stream (asynchronous). */
slim_status slim_step(slim_ctx* ctx, int nsteps);

/* Per-phase timing (tracing).  With on = 1 every step records CUDA events at
 * its phase boundaries (also inside a captured graph); slim_get_timing then
 * returns the device milliseconds of the last step's phases, in order:
 * sample, forward+residual, Gram update, K = lambda I + G, factorisation,
 * triangular solves (with refinement), scatter (nphase <= 7).  *kernels
 * receives the number of kernels one step launches.  SLIM_ESTATE if timing
 * is off and phase_ms is not NULL. */
slim_status slim_set_timing(slim_ctx* ctx, int on);
slim_status slim_get_timing(slim_ctx* ctx, double* phase_ms, int nphase, int* kernels);

/* Wait for queued work and return the device status. */
slim_status slim_sync(slim_ctx* ctx);

/* Make `cuda_stream` (a cudaStream_t; NULL = the context's stream) wait,
 * without blocking the host, for all work the context has queued so far on
 * every stream it uses -- with lookahead, the geometry chains and
 * factorisations prepared ahead of the iterate included.  Work queued on
 * cuda_stream afterwards starts once the context is idle.  Used to end a
 * timed region at the point where the steps' whole pipeline has finished. */
slim_status slim_join_stream(slim_ctx* ctx, void* cuda_stream);

/* Reference iterate for slim_run's error metric ||x - x_ref|| / ||x_ref||
 * (host or device array of n values).  NULL clears it. */
slim_status slim_set_ref(slim_ctx* ctx, const void* x_ref, size_t n, int dtype, int on_device);

/* Step until the relative error to the reference is <= tol (checked every
 * eval_every steps) or max_steps steps were taken.  Reports steps taken,
 * device seconds spent stepping (CUDA events; error evaluation excluded) and
 * the last evaluated error (-1 if no reference is set). */
slim_status slim_run(slim_ctx* ctx, long long max_steps, double tol, int eval_every,
                     long long* steps_done, double* seconds, double* final_err);

/* Number of steps taken so far (k). */
slim_status slim_get_iter(const slim_ctx* ctx, long long* k);

/* Jump to the state after k steps: the memory is rebuilt from the sampled
 * blocks tau_{max(1,k-r)}..tau_k and the current x is kept.  Used by
 * slim_restore and to align the device with an externally computed iterate.
 * SLIM_SOLVE_OLBFGS: k = 0 only (the stored pairs are dropped; SLIM_ENOTSUP
 * otherwise, since the pairs depend on the iterates). */
slim_status slim_set_iter(slim_ctx* ctx, long long k);

/* Checkpoint: k and x.  With buf == NULL, *len receives the size needed.
 * SLIM_ENOTSUP for SLIM_SOLVE_OLBFGS (its pairs are not part of it), for
 * both calls. */
slim_status slim_checkpoint(slim_ctx* ctx, void* buf, size_t* len);
slim_status slim_restore(slim_ctx* ctx, const void* buf, size_t len);

/* Memory of the last step, for inspection: ray ids of the ring (p ints, -1
 * for empty slots), the Gram matrix G = M_k M_k^T in ring order (p*p doubles,
 * row-major) and the last solution z (p doubles).  Host pointers; any may be NULL. */
slim_status slim_get_memory(slim_ctx* ctx, int* ray_ids, double* G, double* z);

/* The stored matrix of a context with a_mode 1 or 2: *nnz, and (if not NULL)
 * row_ptr [m+1], col [nnz] and the values as float32 [nnz] (host buffers).
 * SLIM_ESTATE for a matrix-free context. */
slim_status slim_get_csr(slim_ctx* ctx, long long* nnz, int* row_ptr, int* col, float* val);

/* Sizes: n unknowns, m rows, p = (r+1)*ell. */
slim_status slim_get_sizes(const slim_ctx* ctx, long long* n, long long* m, int* p);

/* Forward projection y = A_S x for the rays listed in ray_ids (device array of
 * count ints; NULL = all m rays in order).  x and y are device arrays of the
 * context precision.  Enqueued on the context stream.  With a stored matrix
 * this streams the CSR (the full pass is an HBM-bound SpMV). */
slim_status slim_project(slim_ctx* ctx, const int* ray_ids, int count, const void* x, void* y);

/* Back projection x += A_S^T y for the listed rays (device arrays as above).
 * With a stored matrix and ray_ids == NULL this streams the CSC copy. */
slim_status slim_backproject(slim_ctx* ctx, const int* ray_ids, int count, const void* y,
                             void* x);

/* Damped Gram solve (lambda I + G) z = rhs for a symmetric positive definite
 * G (the inner solve of the Woodbury form of Eq. (B_k)).  G: device array
 * p*p doubles, row-major, lower triangle read; rhs, z: device arrays of p
 * doubles.  Float64 tiled Cholesky and triangular solves.  Allocates its
 * factor storage on each call and synchronises `cuda_stream` before returning.
 * Returns SLIM_ENOTPD on a non-positive pivot. */
slim_status slim_damped_solve(const double* G, int p, double lambda, const double* rhs,
                              double* z, void* cuda_stream);

/* The two building blocks of the mixed-precision solve's triangular inverse,
 * on their own (they serve the damped solve of Eq. (B_k); the paper itself
 * solves with LSQR or a factorisation and names no kernel).
 *
 * slim_tc_matmul: C = alpha op(A) op(B) + beta C on the tcgen05 tensor
 * cores, op(A) M x K, op(B) K x N, float32 device arrays.  Every float32
 * operand enters as three bfloat16 terms (x0 = bf16(x), x1 = bf16(x - x0),
 * x2 = bf16(x - x0 - x1)) and the six term products a_i b_j with i + j <= 2
 * accumulate in float32, so the result has float32 accuracy.  Layout flags:
 * a_km = 0: op(A)[m][k] = A[m*lda + k], 1: A[k*lda + m]; b_kn = 0:
 * op(B)[k][n] = B[n*ldb + k], 1: B[k*ldb + n]; c_nm = 0: C[m*ldc + n], 1:
 * C[n*ldc + m].  a_lower = 1: op(A) is lower triangular (op(A)[m][k] for
 * k > m is read as zero, whatever A holds there); b_lower = 1: op(B) is
 * lower triangular (op(B)[k][n] for k < n read as zero).  K a multiple of 64;
 * K-contiguous operands (a_km = 0, b_kn = 0) 16-byte aligned with lda / ldb
 * multiples of 4 (SLIM_EINVAL otherwise).  beta = 0: C is not read.
 * Each operand is first split into its three bfloat16 terms in a work space
 * of 6 (M + 128) K + 6 (N + 128) K bytes at most, drawn from a stream-ordered
 * memory pool of the library's own that keeps freed memory reserved for later
 * calls (the largest work space so far stays allocated until the process
 * ends).  Synchronises `cuda_stream`.
 *
 * slim_chol_inverse: the float32 tiled Cholesky factor L of lambda I + G
 * (G: p x p float64 device array, lower triangle read) and X = L^{-1},
 * computed by recursive blocking (X21 = -X22 L21 X11) on the tensor-core
 * product above: X (p x p float32 device array, row-major) receives L^{-1} in
 * its lower triangle and diagonal and (L^{-1})^T in its strict upper
 * triangle.  SLIM_ENOTPD on a non-positive pivot.  Allocates its work space
 * and synchronises `cuda_stream`. */
slim_status slim_tc_matmul(int M, int N, int K, const float* A, long long lda, int a_km,
                           const float* B, long long ldb, int b_kn, float* C, long long ldc,
                           int c_nm, float alpha, float beta, int a_lower, int b_lower,
                           void* cuda_stream);
slim_status slim_chol_inverse(const double* G, int p, double lambda, float* X, void* cuda_stream);

/* Launch log of the pipelined form (lookahead > 0, timing on): every
 * factorisation launch and every iterate chain is bracketed by events without
 * any synchronisation, so a pipelined run can be timed as it runs.  Returns
 * their mean durations in ms since the previous call (at most the last 512 of
 * each) and the number of iterate chains.  Synchronises the context. */
slim_status slim_get_launch_log(slim_ctx* ctx, double* factor_ms, double* iterate_ms,
                                long long* count);

/* Autotuner: time the factorisation tile size and CTAs per SM for a problem's
 * size class (geometry, blocks, r, lambda as for slim_create; `base` gives the
 * other step options) over `steps` steps each, then, for 2D random-ray blocks,
 * the threads per ray (ray_lanes 8, 16, 32) and the pair Gram's cut-off
 * (pair_window 16, 32, 64) with the chosen factorisation options, and return
 * the fastest options in *best (and its time per step in *best_ms).  A size class is the
 * dimension, block kind, precisions and the Gram order p = (r+1) ell rounded
 * up to a multiple of 512.  Results are cached per size class for the life of
 * the process; with the environment variable
 * SLIM_AUTOTUNE_CACHE naming a file, also across processes.  Allocates and
 * frees temporary contexts.  For 3D problems (per-slice solves) *best = *base.
 * Neither the tuner nor the batched form below has a counterpart in the
 * paper: they schedule many problems of the kind Sec. 4 solves one at a time. */
slim_status slim_autotune(const slim_geometry* geom, const slim_blocks* blocks, int r,
                          double lambda, const slim_step_opts* base, int steps,
                          slim_step_opts* best, double* best_ms);

/* Batched form: many independent problems of uneven sizes advance together.
 * slim_batch_create makes one context per problem (arrays of `count` entries;
 * `steps` may be NULL for defaults).  slim_batch_step captures, at its first
 * call, every problem's step as a parallel branch of one CUDA graph and then
 * replays that graph: one graph launch advances every problem by one step.
 * slim_batch_ctx returns problem i's context for set_data / get_x / ...
 * (owned by the batch; do not destroy it). */
typedef struct slim_batch slim_batch;
slim_status slim_batch_create(int count, const slim_geometry* geoms, const slim_blocks* blocks,
                              const int* r, const double* lambda, const slim_step_opts* steps,
                              slim_batch** out);
slim_status slim_batch_ctx(slim_batch* batch, int i, slim_ctx** ctx);
slim_status slim_batch_step(slim_batch* batch, int nsteps);
slim_status slim_batch_sync(slim_batch* batch);
slim_status slim_batch_set_stream(slim_batch* batch, void* cuda_stream);
void slim_batch_destroy(slim_batch* batch);

/* ---------------------------------------------------------------------------
 * Learned initial guess (not in the paper, which starts from x_0 = 0, Sec. 4).
 *
 * A U-Net maps the scaled back-projection s_in A^T b (one N x N channel) to
 * x_0 / s_out: three encoder levels of two 3x3 convolutions + ReLU (32, 64,
 * 128 channels) each followed by 2x2 max-pooling, a 256-channel bottom of two
 * 3x3 convolutions + ReLU, three decoder levels of a 2x2 stride-2 transposed
 * convolution, concatenation [upsampled; encoder output of that level] and
 * two 3x3 convolutions + ReLU (128, 64, 32 channels), then a 1x1 convolution
 * to one channel (1,925,025 parameters).  The forward pass uses the float32
 * master weights rounded to bfloat16 (biases unrounded), with float32
 * activations and accumulation; training minimises the mean squared error
 * with Adam (beta 0.9 / 0.999, eps 1e-8) on the float32 master copy.
 *
 * Parameters are one float32 array in layer order, each layer's weights then
 * its bias: convolutions [out][in][3][3], transposed convolutions
 * [in][out][2][2], the final [1][32].  Tensors passed to forward / train are
 * device arrays of n images of H x W float32 (image-major).
 * ------------------------------------------------------------------------- */
typedef struct slim_unet slim_unet;
slim_status slim_unet_param_count(long long* count);
/* H, W multiples of 8; max_batch images per call.  Parameters start at zero. */
slim_status slim_unet_create(int H, int W, int max_batch, slim_unet** out);
void slim_unet_destroy(slim_unet* net);
/* Host float32 parameters in; resets the Adam state. */
slim_status slim_unet_set_params(slim_unet* net, const float* params, long long count);
slim_status slim_unet_get_params(slim_unet* net, float* params, long long count);
/* Gradients of the last slim_unet_train_step (host float32). */
slim_status slim_unet_get_grads(slim_unet* net, float* grads, long long count);
/* y = U-Net(x) for n images; asynchronous on `cuda_stream`. */
slim_status slim_unet_forward(slim_unet* net, const float* x, float* y, int n, void* cuda_stream);
/* One step: forward, loss = mean (y - target)^2, backward, Adam with rate lr.
 * *loss (if not NULL) receives the loss; the call then synchronises. */
slim_status slim_unet_train_step(slim_unet* net, const float* x, const float* target, int n,
                                 float lr, double* loss, void* cuda_stream);
/* The network's layers on their own, as used by forward and train_step.
 * Device float32 arrays in the network's layout: channel c of image i,
 * pixel (y, x) at [c][i][y][x], i.e. c * n*H*W + i * H*W + y * W + x.
 * Asynchronous on `cuda_stream`; no allocation.  Weights are read as
 * bfloat16 (nearest even), which leaves the network's rounded weights
 * unchanged; activations and gradients keep float32 accuracy (they enter the
 * bfloat16 tensor cores as sums of bfloat16 terms) and accumulation is
 * float32.  SLIM_EINVAL for a NULL required pointer, a size < 1, more than
 * 65536 channels or 4 n H W >= 2^31; SLIM_ECUDA if a launch fails.
 *
 * 3x3 convolution, stride 1, zero padding 1: w [c_out][c_in][3][3], b [c_out]
 * (NULL: zero), x [c_in][n][H][W], y [c_out][n][H][W] = conv(x, w) + b, then
 * max(y, 0) when relu != 0. */
slim_status slim_unet_conv3x3(const float* x, int n, int c_in, int H, int W, const float* w,
                              const float* b, int c_out, int relu, float* y, void* cuda_stream);
/* Gradients of that convolution for dy [c_out][n][H][W], the gradient at
 * conv(x, w) + b (before any ReLU): dw [c_out][c_in][3][3] += dL/dw and
 * db [c_out] += dL/db (accumulated; db may be NULL); dx [c_in][n][H][W] =
 * dL/dx, overwritten (skipped when NULL). */
slim_status slim_unet_conv3x3_grad(const float* x, const float* dy, int n, int c_in, int H, int W,
                                   const float* w, int c_out, float* dw, float* db, float* dx,
                                   void* cuda_stream);
/* 2x2 transposed convolution, stride 2: w [c_in][c_out][2][2], b [c_out]
 * (NULL: zero), x [c_in][n][H][W], y [c_out][n][2H][2W] with
 * y[o][i][2r+u][2q+v] = sum_c w[c][o][u][v] x[c][i][r][q] + b[o]. */
slim_status slim_unet_tconv2x2(const float* x, int n, int c_in, int H, int W, const float* w,
                               const float* b, int c_out, float* y, void* cuda_stream);
/* Its gradients for dy [c_out][n][2H][2W]: dw += dL/dw, db += dL/db
 * (accumulated; db may be NULL), dx [c_in][n][H][W] = dL/dx (skipped when
 * NULL). */
slim_status slim_unet_tconv2x2_grad(const float* x, const float* dy, int n, int c_in, int H, int W,
                                    const float* w, int c_out, float* dw, float* db, float* dx,
                                    void* cuda_stream);
/* Warm start of a 2D context: x_0 = s_out * U-Net(s_in * A^T b) with the
 * context's data b (N x N network).  If ||A x_0 - b|| >= ||b|| the network's
 * guess is worse than zero and x is set to 0 instead.  *used = 1 when x_0
 * was kept; *ratio = ||A x_0 - b|| / ||b||.  Synchronises. */
slim_status slim_warm_start(slim_ctx* ctx, slim_unet* net, double s_in, double s_out, int* used,
                            double* ratio);
/* Back-projection A^T b of the context's data into a device float32 array
 * x[n] (the network's input before scaling).  Synchronises. */
slim_status slim_backproject_data(slim_ctx* ctx, float* x);

/* Largest order p accepted by slim_damped_solve_noalloc. */
#define SLIM_NOALLOC_MAX_P 1024

/* The damped Gram solve of slim_damped_solve without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they solve -- an application whose device
 * memory is wholly reserved by its own pool allocator (as under a framework's
 * caching allocator), or a latency-critical loop that must not call
 * cudaMalloc/cudaFree, which synchronise the device.
 *
 * Same arguments as slim_damped_solve and the same computation: the float64
 * tiled Cholesky with the same task list and grid, then the same
 * triangular-solve kernels, so the results agree to rounding (the order of
 * the floating-point sums is the same; only the scheduling of the persistent
 * factorisation's CTAs varies between runs, as it does for the allocating
 * solve).  p <= SLIM_NOALLOC_MAX_P; larger p is rejected with SLIM_EINVAL
 * (use slim_damped_solve).  The caller passes G, rhs and z as device arrays.
 * All scratch lives in one static device array of about 9 MB that every GPU
 * which loads the library keeps until the process exits.  The first call on a
 * device does a one-time set-up with that device current: it resolves the
 * array's address and copies the factorisation's task lists into it with
 * synchronous copies, so make that first call before capturing any stream.
 * Calls share the array and each overwrites what the previous one left
 * there: calls that overlap on the GPU (different streams or host threads at
 * the same time) race and give wrong results.  Each call synchronises
 * `cuda_stream`. */
slim_status slim_damped_solve_noalloc(const double* G, int p, double lambda, const double* rhs,
                                      double* z, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SLIM_H_ */
