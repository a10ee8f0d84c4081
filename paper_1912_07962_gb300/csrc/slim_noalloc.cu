// Damped Gram solve that allocates nothing: the same float64 tiled Cholesky
// and triangular solves as slim_damped_solve, with all scratch memory in one
// file-scope device array of fixed size.
#include <mutex>

#include "../../include/slim.h"
#include "slim_chol.cuh"

using namespace slim;

namespace {

constexpr int kNb = 32;                                  // tile size of the float64 factor
constexpr int kMaxP = SLIM_NOALLOC_MAX_P;                // largest order accepted
constexpr int kMaxT = kMaxP / kNb;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t task_count(int T) {
  // POTRF + TRSM + update tasks of the tiled factorisation of T x T tiles
  size_t n = 0;
  for (int k = 0; k < T; ++k) n += 1 + (size_t)(T - k - 1) + (size_t)(T - k - 1) * (T - k) / 2;
  return n;
}

// Byte offsets of the parts of the scratch array.
constexpr size_t kOffL = 0;
constexpr size_t kOffWinv = kOffL + align256((size_t)kMaxP * kMaxP * sizeof(double));
constexpr size_t kOffY = kOffWinv + align256((size_t)kMaxT * kNb * kNb * sizeof(double));
constexpr size_t kOffV = kOffY + align256(2 * (size_t)kMaxP * sizeof(double));
constexpr size_t kOffZ = kOffV + align256((size_t)kMaxP * sizeof(double));
constexpr size_t kOffTasks = kOffZ + align256((size_t)kMaxP * sizeof(double));
constexpr size_t kOffSync = kOffTasks + align256(task_count(kMaxT) * sizeof(CholTask));
constexpr size_t kOffStatus = kOffSync + align256(((size_t)kMaxT * kMaxT + 2 * kMaxT + 4) * sizeof(int));
constexpr size_t kScratchBytes = kOffStatus + 256;

// The scratch itself (about 8.7 MB).  Host code must not use this name as an
// address: it takes the device address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch on that device
  int num_sms = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with that device current: resolve the scratch address.
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
    s.base = static_cast<unsigned char*>(ptr);
    s.num_sms = sms;
    s.ready = true;
  }
  *out = s;
  return SLIM_OK;
}

// The task list of the T x T tiled factorisation, in the dependency-compatible
// order the factor kernel expects (lookahead of one panel).
__global__ void gen_tasks_kernel(CholTask* t, int T) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int n = 0;
  t[n++] = {kPotrf, 0, 0, 0};
  for (int i = 1; i < T; ++i) t[n++] = {kTrsm, (uint16_t)i, 0, 0};
  for (int k = 0; k + 1 < T; ++k) {
    const int n1 = k + 1;
    for (int i = n1; i < T; ++i) t[n++] = {kUpd, (uint16_t)i, (uint16_t)n1, (uint16_t)k};
    t[n++] = {kPotrf, (uint16_t)n1, (uint16_t)n1, (uint16_t)n1};
    for (int i = n1 + 1; i < T; ++i) t[n++] = {kTrsm, (uint16_t)i, (uint16_t)n1, (uint16_t)n1};
    for (int m = k + 2; m < T; ++m)
      for (int i = m; i < T; ++i) t[n++] = {kUpd, (uint16_t)i, (uint16_t)m, (uint16_t)k};
  }
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
  const int T = P / kNb;
  double* L = reinterpret_cast<double*>(ds.base + kOffL);
  double* v = reinterpret_cast<double*>(ds.base + kOffV);
  double* out = reinterpret_cast<double*>(ds.base + kOffZ);
  int* status = reinterpret_cast<int*>(ds.base + kOffStatus);
  CholPlan plan;
  plan.P = P;
  plan.T = T;
  plan.nb = kNb;
  plan.is_f32 = 0;
  plan.ntasks = (int)task_count(T);
  plan.d_tasks = reinterpret_cast<CholTask*>(ds.base + kOffTasks);
  plan.d_sync = reinterpret_cast<int*>(ds.base + kOffSync);
  plan.d_winv = ds.base + kOffWinv;
  plan.d_y = ds.base + kOffY;
  plan.grid = 2 * ds.num_sms;

  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    gen_tasks_kernel<<<1, 1, 0, s>>>(plan.d_tasks, T);
    e = cudaGetLastError();
  }
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
