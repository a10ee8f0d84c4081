// Damped Gram solve that allocates nothing: the same float64 tiled Cholesky
// (same task list, same grid) and the same triangular-solve kernels as
// slim_damped_solve, with all scratch memory in one file-scope device array
// of fixed size.
#include <mutex>
#include <vector>

#include "../../include/slim.h"
#include "slim_chol.cuh"

using namespace slim;

namespace {

constexpr int kNb = 32;                                  // tile size of the float64 factor
constexpr int kMaxP = SLIM_NOALLOC_MAX_P;                // largest order accepted
constexpr int kMaxT = kMaxP / kNb;
constexpr int kMaxDevices = 64;
constexpr int kCtasPerSm = 2;                            // as slim_damped_solve's plan

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
// An upper bound on the tasks of the T x T factorisation: one POTRF, TRSM and
// single-tile update task per tile operation (the list the factor runs fuses
// some of them into panel tasks, so it is never longer).
constexpr size_t task_bound(int T) {
  size_t n = 0;
  for (int k = 0; k < T; ++k) n += 1 + (size_t)(T - k - 1) + (size_t)(T - k - 1) * (T - k) / 2;
  return n;
}
// Start of the list for T tiles inside the task region: the lists for
// T = 1 .. kMaxT are stored one after another.
constexpr size_t task_offset(int T) {
  size_t n = 0;
  for (int t = 1; t < T; ++t) n += task_bound(t);
  return n;
}

// Byte offsets of the parts of the scratch array.
constexpr size_t kOffL = 0;
constexpr size_t kOffWinv = kOffL + align256((size_t)kMaxP * kMaxP * sizeof(double));
constexpr size_t kOffY = kOffWinv + align256((size_t)kMaxT * kNb * kNb * sizeof(double));
constexpr size_t kOffV = kOffY + align256(2 * (size_t)kMaxP * sizeof(double));
constexpr size_t kOffZ = kOffV + align256((size_t)kMaxP * sizeof(double));
constexpr size_t kOffTasks = kOffZ + align256((size_t)kMaxP * sizeof(double));
constexpr size_t kOffSync =
    kOffTasks + align256(task_offset(kMaxT + 1) * sizeof(CholTask));
constexpr size_t kOffStatus = kOffSync + align256(((size_t)kMaxT * kMaxT + 2 * kMaxT + 4) * sizeof(int));
constexpr size_t kScratchBytes = kOffStatus + 256;

// The scratch itself (about 9 MB).  Host code must not use this name as an
// address: it takes the device address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch on that device
  int num_sms = 0;
  int ntasks[kMaxT + 1] = {};      // length of the stored list for T tiles
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with that device current: resolve the scratch address and
// store the factorisation's task lists for every T up to kMaxT there (built
// by the same host routine as the allocating solve's, so the order is the
// one its counter protocol was checked on).  The copies are synchronous.
slim_status setup_device(int dev, DeviceSetup* out) {
  if (dev < 0 || dev >= kMaxDevices) return SLIM_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return SLIM_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return SLIM_ECUDA;
    }
    unsigned char* base = static_cast<unsigned char*>(ptr);
    for (int T = 1; T <= kMaxT; ++T) {
      const std::vector<CholTask> tasks = build_chol_tasks(T, false);
      if (tasks.size() > task_bound(T)) return SLIM_EINVAL;   // cannot happen; keeps the bound honest
      if (cudaMemcpy(base + kOffTasks + task_offset(T) * sizeof(CholTask), tasks.data(),
                     tasks.size() * sizeof(CholTask), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return SLIM_ECUDA;
      }
      s.ntasks[T] = (int)tasks.size();
    }
    s.base = base;
    s.num_sms = sms;
    s.ready = true;
  }
  *out = s;
  return SLIM_OK;
}

// L = lambda I + G on the p x p block, identity on the padding.
__global__ void noalloc_form_kernel(const double* G, int p, double lam, double* L, int P) {
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

extern "C" slim_status slim_damped_solve_noalloc(const double* G, int p, double lambda,
                                                  const double* rhs, double* z, void* stream) {
  if (!G || !rhs || !z || p <= 0 || !(lambda >= 0.0)) return SLIM_EINVAL;
  if (p > kMaxP) return SLIM_EINVAL;   // larger systems need slim_damped_solve
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SLIM_ECUDA;
  }
  DeviceSetup ds;
  slim_status st = setup_device(dev, &ds);
  if (st != SLIM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int P = (p + kNb - 1) / kNb * kNb;
  CholPlan plan;
  if (chol_plan_configure(&plan, P, kNb, 0, ds.num_sms, kCtasPerSm) != cudaSuccess) {
    cudaGetLastError();
    return SLIM_ECUDA;
  }
  const int T = plan.T;
  double* L = reinterpret_cast<double*>(ds.base + kOffL);
  double* v = reinterpret_cast<double*>(ds.base + kOffV);
  double* out = reinterpret_cast<double*>(ds.base + kOffZ);
  int* status = reinterpret_cast<int*>(ds.base + kOffStatus);
  plan.ntasks = ds.ntasks[T];
  plan.d_tasks = reinterpret_cast<CholTask*>(ds.base + kOffTasks + task_offset(T) * sizeof(CholTask));
  plan.d_sync = reinterpret_cast<int*>(ds.base + kOffSync);
  plan.d_winv = ds.base + kOffWinv;
  plan.d_y = ds.base + kOffY;

  // the previous call's status, counters and right-hand side are stale: the
  // factorisation and the solves clear their counters and flags themselves
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, (size_t)P * sizeof(double), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(v, rhs, (size_t)p * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) {
    long long total = (long long)P * P;
    int grid = (int)((total + 255) / 256 < 152LL * 16 ? (total + 255) / 256 : 152LL * 16);
    noalloc_form_kernel<<<grid, 256, 0, s>>>(G, p, lambda, L, P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = chol_factor(plan, L, status, s);
  if (e == cudaSuccess) e = chol_solve(plan, L, v, out, status, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(z, out, (size_t)p * sizeof(double), cudaMemcpyDeviceToDevice, s);
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SLIM_ECUDA;
  }
  return hs != 0 ? static_cast<slim_status>(hs) : SLIM_OK;
}
