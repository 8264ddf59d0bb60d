// js_max_dt_noalloc: the CFL time-step reduction for callers that cannot allocate device
// memory -- for example a host application or plugin that owns every device allocation
// itself (a fixed memory pool, a budget enforced by its allocator), so a library call must
// not reach for cudaMalloc.  The caller passes the state and optional cell tags; the
// reduction's scratch is a file-scope device array, so this entry point allocates nothing.
//
// Scratch: g_cfl_scratch holds one (max wave-speed rate, min density) pair per block of
// 2048 cells and a final pair; at most JS_NOALLOC_MAX_CELLS cells per call.  Every GPU that
// loads the library keeps the array (64 KiB) until the process exits.  Each call overwrites
// exactly the partials it reads, so nothing needs clearing; the array keeps the last call's
// values.  Calls whose kernels overlap on the GPU (several streams, several host threads)
// share the array and race: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "jaxshock.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 8;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;  // 2048
constexpr int kMaxBlocks = JS_NOALLOC_MAX_CELLS / kCellsPerBlock;
static_assert(JS_NOALLOC_MAX_CELLS % kCellsPerBlock == 0, "block size must divide the cell limit");

// per-block (rate, rho_min) partials, then the final pair at [2 * kMaxBlocks]
static __device__ __align__(256) double g_cfl_scratch[2 * kMaxBlocks + 2];

// rate = (|u| + a)/dx [+ (|v| + a)/dy] of one cell, IEEE-rounded in the same order as the
// context-based reduction so that both entry points return the same dt.  A non-physical cell
// (rho or p not positive, or not finite) gets the rate +infinity, so the step size is 0 and
// the call returns JS_ERR_NONPHYSICAL, as js_max_dt does.
__device__ __forceinline__ double cell_rate(const double* U, long long n, long long t, double gamma, double dx,
                                            double dy, int two_d, double& r) {
  r = U[t];
  const double u = __ddiv_rn(U[n + t], r), v = __ddiv_rn(U[2 * n + t], r);
  const double ke = __dmul_rn(__dmul_rn(0.5, r), __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)));
  const double p = __dmul_rn(gamma - 1.0, __dsub_rn(U[3 * n + t], ke));
  if (!(r > 0.0) || !(r < INFINITY) || !(p > 0.0) || !(p < INFINITY)) return INFINITY;
  const double a = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), r));
  double s = __ddiv_rn(__dadd_rn(fabs(u), a), dx);
  if (two_d) s = __dadd_rn(s, __ddiv_rn(__dadd_rn(fabs(v), a), dy));
  return s;
}

__device__ __forceinline__ void block_reduce(double& rate, double& rmin) {
  for (int o = 16; o > 0; o >>= 1) {
    rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
  }
  __shared__ double sr[kThreads / 32], sm[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sr[wid] = rate;
    sm[wid] = rmin;
  }
  __syncthreads();
  if (wid == 0) {
    rate = (lane < kThreads / 32) ? sr[lane] : 0.0;
    rmin = (lane < kThreads / 32) ? sm[lane] : INFINITY;
    for (int o = 16; o > 0; o >>= 1) {
      rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
      rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    }
  }
}

// pass 1: block b reduces cells [b * 2048, (b + 1) * 2048) into partial pair b
__global__ void __launch_bounds__(kThreads) cfl_partials(const double* __restrict__ U, long long n,
                                                         const unsigned char* __restrict__ tag, double gamma,
                                                         double dx, double dy, int two_d, double* scratch) {
  double rate = 0.0, rmin = INFINITY;
  const long long b0 = (long long)blockIdx.x * kCellsPerBlock;
  for (int k = 0; k < kCellsPerThread; ++k) {
    const long long t = b0 + (long long)k * kThreads + threadIdx.x;
    if (t >= n || (tag && tag[t] != 0)) continue;
    double r;
    const double s = cell_rate(U, n, t, gamma, dx, dy, two_d, r);
    rate = fmax(rate, s);
    rmin = fmin(rmin, r);
  }
  block_reduce(rate, rmin);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = rate;
    scratch[2 * blockIdx.x + 1] = rmin;
  }
}

// pass 2: one block reduces the nb partials into the final pair
__global__ void __launch_bounds__(kThreads) cfl_final(double* scratch, int nb) {
  double rate = 0.0, rmin = INFINITY;
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    rate = fmax(rate, scratch[2 * b]);
    rmin = fmin(rmin, scratch[2 * b + 1]);
  }
  block_reduce(rate, rmin);
  if (threadIdx.x == 0) {
    scratch[2 * kMaxBlocks] = rate;
    scratch[2 * kMaxBlocks + 1] = rmin;
  }
}

// Device address of g_cfl_scratch on the current device, looked up once per device.  In
// host code the symbol itself is only a host-side stand-in; kernels need this address.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return JS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return JS_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cfl_scratch) != cudaSuccess || !p) return JS_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return JS_OK;
}

}  // namespace

extern "C" int js_max_dt_noalloc(const js_grid* grid, const js_params* params, const double* U,
                                 const unsigned char* tag, double cfl, void* stream, double* dt_out) {
  if (!grid || !params || !U || !dt_out || !(cfl > 0.0)) return JS_ERR_ARG;
  if (grid->nx < 1 || grid->ny < 1 || !(grid->dx > 0.0) || !(grid->dy > 0.0)) return JS_ERR_ARG;
  if (!(params->gamma > 1.0) || !(params->mu >= 0.0) || (params->mu > 0.0 && !(params->Pr > 0.0)))
    return JS_ERR_ARG;
  const long long n = (long long)grid->nx * grid->ny;
  if (n > JS_NOALLOC_MAX_CELLS) return JS_ERR_ARG;  // beyond the static scratch
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != JS_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
  cfl_partials<<<nb, kThreads, 0, s>>>(U, n, tag, params->gamma, grid->dx, grid->dy, grid->ny > 1 ? 1 : 0,
                                       scratch);
  cfl_final<<<1, kThreads, 0, s>>>(scratch, nb);
  if (cudaGetLastError() != cudaSuccess) return JS_ERR_CUDA;
  double h[2];
  if (cudaMemcpyAsync(h, scratch + 2 * kMaxBlocks, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return JS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return JS_ERR_CUDA;
  const double rate = h[0], rmin = h[1];
  double dt = cfl / rate;
  if (params->mu > 0.0) {
    const double hmin = (grid->ny > 1) ? (grid->dx < grid->dy ? grid->dx : grid->dy) : grid->dx;
    const double lim = (4.0 / 3.0 < params->gamma / params->Pr) ? params->gamma / params->Pr : 4.0 / 3.0;
    const double dtv = cfl * hmin * hmin * rmin / (2.0 * params->mu * lim);
    dt = (dtv < dt) ? dtv : dt;
  }
  *dt_out = dt;
  if (!std::isfinite(dt) || !(dt > 0.0)) return JS_ERR_NONPHYSICAL;
  return JS_OK;
}
