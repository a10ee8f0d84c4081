// Tiled Cholesky factorisation and triangular solves of the damped Gram
// matrix K = lambda_k I + M_k M_k^T (the p x p system that the Woodbury form
// of Eq. (B_k) leaves to solve each step).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "slim_chol_tasks.h"

namespace slim {

// One factorisation of a merged launch (chol_factor_batch): its matrix, tile
// grid, task list, tile counters, diagonal-tile inverses and status word.
struct FactorJob {
  void* L;
  int P, T;
  const CholTask* tasks;
  int* cnt;
  void* winv;
  int* status;
};

struct CholPlan {
  int P = 0;          // padded order (multiple of NB)
  int T = 0;          // tiles per side
  int nb = 0;         // tile size
  int is_f32 = 0;     // factor precision
  int ntasks = 0;
  CholTask* d_tasks = nullptr;   // device task list
  int* d_sync = nullptr;         // [T*T tile counters | T fwd flags | T bwd flags | 4 tickets]
  void* d_winv = nullptr;        // T inverse diagonal tiles, NB*NB each (factor precision)
  void* d_y = nullptr;           // forward-solve intermediate, P values (factor precision)
  int grid = 0;                  // persistent CTAs for the factorisation
  int wide = 0;                  // 1: the factorisation CTAs use the whole register file
                                 // (one per SM); 0: 128 registers a thread (SMs shared)
  int cluster = 0;               // CTAs of the cluster that runs both solves (0: chained CTAs)
};

// Words of the plan's synchronisation array (d_sync): tile counters, solve
// flags, tickets and the abort flag.
inline size_t chol_sync_words(int T) { return (size_t)T * T + 2 * (size_t)T + 4; }

// Shape the plan for order P (multiple of nb) without allocating anything:
// tiles, factorisation grid, the solve's cluster size and the factor kernel's
// shared-memory opt-in.  wide = 1: one factorisation CTA per SM with the whole
// register file (grid = num_sms); 0: ctas_per_sm CTAs per SM at 128 registers
// a thread; -1: wide when ctas_per_sm is 1.  The caller then provides d_tasks (the list of
// build_chol_tasks(T, is_f32 && nb == 64)) and ntasks, d_sync
// (chol_sync_words(T) ints), d_winv (T * nb * nb values) and d_y (2P values).
cudaError_t chol_plan_configure(CholPlan* plan, int P, int nb, int is_f32, int num_sms,
                                int ctas_per_sm = 2, int wide = -1);

// Factor diagonal tile (j, j) of the float32 matrix L (P x P row-major, tiles
// of 64, its trailing updates applied) in place, L_jj with zeros above the
// diagonal, and write L_jj^{-1} to winv + j * 64 * 64.  One CTA; non-positive
// pivots record SLIM_ENOTPD in *status.  chol_potrf_tile_prepare opts in to
// its shared memory (once per process).
cudaError_t chol_potrf_tile_prepare();
cudaError_t chol_potrf_tile(float* L, int P, int j, float* winv, int* status, cudaStream_t s);

// Allocate / free the plan for order P (multiple of nb).
cudaError_t chol_plan_create(CholPlan* plan, int P, int nb, int is_f32, int num_sms,
                             int ctas_per_sm = 2, int wide = -1);
void chol_plan_destroy(CholPlan* plan);

// Factor L (P x P row-major, lower triangle holds K on entry, L on exit) in
// the factor precision; then solve L L^T z = v (float64 vectors of length P).
// Errors are recorded in *status (SLIM_ENOTPD, SLIM_ETIMEOUT).
// first_tile: v is zero in rows [0, first_tile * nb), so the forward sweep
// starts at that tile (y is zero above it); 0 for a general v.
cudaError_t chol_factor(const CholPlan& plan, void* L, int* status, cudaStream_t s);
cudaError_t chol_solve(const CholPlan& plan, const void* L, const double* v, double* z,
                       int* status, cudaStream_t s, int first_tile = 0);

// Factorisations of many problems (same factor precision and tile size) in
// one persistent launch: their task lists merged into one queue, each
// problem's order kept (task t of a problem with n tasks is placed by
// (t + 1/2) / n, so the problems advance together).  The CTAs of the launch
// claim (problem, task) pairs by ticket; a wait that runs out stops every
// CTA (SLIM_ETIMEOUT in that problem's status).  ctas_per_sm 1: one CTA per
// SM with the whole register file, as a wide plan.
struct CholBatch {
  int is_f32 = 0, nb = 0, grid = 0, wide = 0;
  int njobs = 0, nqueue = 0;
  FactorJob* d_jobs = nullptr;
  int2* d_queue = nullptr;
  int* d_ticket = nullptr;                 // [ticket, abort flag]
  std::vector<const CholPlan*> plans;      // for the counter resets
};
cudaError_t chol_batch_create(CholBatch* b, const std::vector<const CholPlan*>& plans,
                              const std::vector<void*>& Ls, const std::vector<int*>& statuses,
                              int num_sms, int ctas_per_sm);
void chol_batch_destroy(CholBatch* b);
cudaError_t chol_factor_batch(const CholBatch& b, cudaStream_t s);

}  // namespace slim
