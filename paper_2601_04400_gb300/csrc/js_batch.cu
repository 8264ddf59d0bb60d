// Batched path: many independent flow instances (uneven grids, parameters, bodies) advanced
// together in ONE persistent cooperative kernel launch -- the GB300 counterpart of mapping the
// solver step over a batch of problems (the paper's vmap, Sec. 1).
//
// The kernel runs every phase of every step for all instances, separated by grid barriers:
//   pack       user states -> padded buffers
//   per step:  CFL        per-instance max wave-speed rate and min density (atomics)
//              per stage: IB fill | halo fill | fused stage tiles (the per-grid kernel's
//                         device function, so trajectories equal js_step's bit for bit)
//   unpack     padded buffers -> user states
// Each instance's dt is computed on the device from its reduction (same arithmetic as
// js_max_dt).  Work items (tiles, ghosts, halo cells) of all instances are distributed
// round-robin over the resident blocks.  Every barrier wait is bounded: a block that waits
// longer than the budget sets JS_ERR_TIMEOUT in the error flag and returns, and the others
// leave at their next wait.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "jaxshock.h"
#include "js_fill.cuh"
#include "js_internal.h"
#include "js_stage.cuh"

namespace js {

// the per-grid default tile (variant 0): 32x32 cells, concurrent x/y sweeps
constexpr int BTX = 32, BTY = 32, BLX = 16, BLY = 16;
using BStageV = Stage2DC<BTX, BTY, BLX, BLY, true>;
using BStageE = Stage2DC<BTX, BTY, BLX, BLY, false>;
constexpr int BNT = BStageV::NT;
static_assert(BStageV::NT == BStageE::NT && BNT % 32 == 0, "one block shape for both physics");

struct BatchArgs {
  const InstDesc* inst;
  int count;
  const int* tile0;           // prefix sums (count + 1) of tiles, ghosts and halo cells
  const long long* ghost0;
  const long long* halo0;
  unsigned long long* red;    // [2][count][2]: rate bits, rho_min bits
  unsigned* bar;              // [0] arrivals, [1] generation
  int* err;
  double* t;                  // accumulated time per instance or nullptr
  double* dt_log;             // [n_steps][count] step sizes used, or nullptr
  double cfl;
  int n_steps;
  int extra_arrivals;         // > 0 only to exercise the barrier timeout
  long long budget;           // barrier wait budget in clock cycles
};

// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int find_inst(const int* pre, int count, int item) {
  int lo = 0, hi = count;  // pre[lo] <= item < pre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int find_inst64(const long long* pre, int count, long long item) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// grid barrier with a bounded wait; returns false when the launch must stop
__device__ bool grid_sync(const BatchArgs& b) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = b.bar + 1;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned target = gridDim.x + (unsigned)b.extra_arrivals;
    const unsigned arrived = atomicAdd(b.bar, 1u) + 1u;
    if (arrived == target) {
      b.bar[0] = 0u;
      __threadfence();
      atomicAdd(b.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*(volatile int*)b.err & ERR_TIMEOUT_BIT) { ok = 0; break; }
        if (clock64() - t0 > b.budget) {
          atomicOr(b.err, ERR_TIMEOUT_BIT);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ double inst_dt(const InstDesc& d, const unsigned long long* red, double cfl) {
  const double rate = __longlong_as_double((long long)red[0]);
  const double rmin = __longlong_as_double((long long)red[1]);
  double dt = __ddiv_rn(cfl, rate);
  if (d.visc) {
    const double dtv = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(cfl, d.hmin), d.hmin), rmin),
                                 __dmul_rn(__dmul_rn(2.0, d.mu), d.lim));
    dt = (dtv < dt) ? dtv : dt;
  }
  return dt;
}

__global__ void __launch_bounds__(BNT) batch_kernel(BatchArgs b) {
  extern __shared__ double smem[];
  const int ntiles = b.tile0[b.count];
  const long long nghost = b.ghost0[b.count], nhalo = b.halo0[b.count];
  const int tid = threadIdx.x, lane = threadIdx.x & 31;
  // ---- pack user states; reset both reduction buffers
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int k = find_inst(b.tile0, b.count, it);
    const InstDesc& d = b.inst[k];
    const int t = it - b.tile0[k];
    const int i0 = (t % d.ntx) * BTX, j0 = (t / d.ntx) * BTY;
    const long long n = (long long)d.lay.nx * d.lay.ny;
    for (int e = tid; e < BTX * BTY; e += BNT) {
      const int i = i0 + (e % BTX), j = j0 + (e / BTX);
      if (i >= d.lay.nx || j >= d.lay.ny) continue;
      const long long o = (long long)j * d.lay.nx + i, p = d.lay.idx(i, j);
#pragma unroll
      for (int c = 0; c < 4; ++c) d.N[c * d.lay.plane + p] = d.U[c * n + o];
    }
  }
  if (blockIdx.x == 0)
    for (int k = tid; k < 2 * b.count; k += BNT) {
      b.red[2 * k] = 0ULL;
      b.red[2 * k + 1] = 0x7ff0000000000000ULL;
    }
  if (!grid_sync(b)) return;
  for (int step = 0; step < b.n_steps; ++step) {
    const int par = step & 1;
    unsigned long long* red = b.red + 2 * (long long)b.count * par;
    // ---- CFL reduction over fluid cells, per instance
    for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
      const int k = find_inst(b.tile0, b.count, it);
      const InstDesc& d = b.inst[k];
      const int t = it - b.tile0[k];
      const int i0 = (t % d.ntx) * BTX, j0 = (t / d.ntx) * BTY;
      double rate = 0.0, rmin = __longlong_as_double(0x7ff0000000000000LL);
      for (int e = tid; e < BTX * BTY; e += BNT) {
        const int i = i0 + (e % BTX), j = j0 + (e / BTX);
        if (i >= d.lay.nx || j >= d.lay.ny) continue;
        if (d.tag && d.tag[(long long)j * d.lay.nx + i] != 0) continue;
        const long long p = d.lay.idx(i, j);
        const double r = d.N[p];
        rate = fmax(rate, cfl_rate(r, d.N[d.lay.plane + p], d.N[2 * d.lay.plane + p], d.N[3 * d.lay.plane + p],
                                   d.gamma, d.dx, d.dy, d.lay.ny > 1));
        rmin = fmin(rmin, r);
      }
      for (int o = 16; o > 0; o >>= 1) {
        rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
        rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
      }
      if (lane == 0) {
        atomicMax(red + 2 * k, (unsigned long long)__double_as_longlong(rate));
        atomicMin(red + 2 * k + 1, (unsigned long long)__double_as_longlong(rmin));
      }
    }
    if (!grid_sync(b)) return;
    if (blockIdx.x == 0) {
      // the other parity was last read in the previous step: reset it for the next one
      unsigned long long* nxt = b.red + 2 * (long long)b.count * (par ^ 1);
      for (int k = tid; k < b.count; k += BNT) {
        nxt[2 * k] = 0ULL;
        nxt[2 * k + 1] = 0x7ff0000000000000ULL;
        const double dtk = inst_dt(b.inst[k], red + 2 * k, b.cfl);
        // a non-physical fluid cell has an infinite rate (cfl_rate): dt = 0
        if (!(dtk > 0.0) || !(dtk < CUDART_INF)) atomicOr(b.err, ERR_NONPHYSICAL_BIT);
        if (b.t) b.t[k] += dtk;
        if (b.dt_log) b.dt_log[(long long)step * b.count + k] = dtk;
      }
    }
    for (int s = 0; s < 3; ++s) {
      // ---- immersed-boundary ghosts of the stage input
      for (long long g = (long long)blockIdx.x * BNT + tid; g < nghost; g += (long long)gridDim.x * BNT) {
        const int k = find_inst64(b.ghost0, b.count, g);
        const InstDesc& d = b.inst[k];
        double* X = (s == 0) ? d.N : ((s == 1) ? d.A : d.B);
        ib_fill_one(X, d.lay, d.ib, d.gamma, d.wall, (int)(g - b.ghost0[k]));
      }
      if (!grid_sync(b)) return;
      // ---- domain halos
      for (long long h = (long long)blockIdx.x * BNT + tid; h < nhalo; h += (long long)gridDim.x * BNT) {
        const int k = find_inst64(b.halo0, b.count, h);
        const InstDesc& d = b.inst[k];
        double* X = (s == 0) ? d.N : ((s == 1) ? d.A : d.B);
        bc_fill_one(X, d.lay, d.bc, h - b.halo0[k]);
      }
      if (!grid_sync(b)) return;
      // ---- stage tiles
      for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
        const int k = find_inst(b.tile0, b.count, it);
        const InstDesc& d = b.inst[k];
        const int t = it - b.tile0[k];
        const double dt = inst_dt(d, red + 2 * k, b.cfl);
        StageArgs a;
        a.Uin = (s == 0) ? d.N : ((s == 1) ? d.A : d.B);
        a.Un = d.N;
        a.Uout = (s == 0) ? d.A : ((s == 1) ? d.B : d.N);
        a.tag = d.tag;
        a.acc = d.acc;
        a.acc2 = d.acc2;
        a.dtc = nullptr;
        a.err = b.err;
        a.lay = d.lay;
        a.gamma = d.gamma;
        a.gm1 = d.gamma - 1.0;
        a.g1 = 1.0 / (d.gamma - 1.0);
        a.cx = dt / d.dx;
        a.cy = dt / d.dy;
        a.rk_a = (s == 0) ? 0.0 : ((s == 1) ? 0.75 : 1.0 / 3.0);
        a.rk_b = (s == 0) ? 1.0 : ((s == 1) ? 0.25 : 2.0 / 3.0);
        a.avx = dt * d.nu / (d.dx * d.dx);
        a.avy = dt * d.nu / (d.dy * d.dy);
        a.vx = d.vx;
        a.vy = d.vy;
        a.use_un = (s > 0) ? 1 : 0;
        a.has_av = d.has_av;
        if (d.visc) stage_tile_c<BTX, BTY, BLX, BLY, true, false>(a, t % d.ntx, t / d.ntx, smem);
        else stage_tile_c<BTX, BTY, BLX, BLY, false, false>(a, t % d.ntx, t / d.ntx, smem);
        __syncthreads();  // the next tile reuses shared memory
      }
      if (!grid_sync(b)) return;
    }
  }
  // ---- unpack
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int k = find_inst(b.tile0, b.count, it);
    const InstDesc& d = b.inst[k];
    const int t = it - b.tile0[k];
    const int i0 = (t % d.ntx) * BTX, j0 = (t / d.ntx) * BTY;
    const long long n = (long long)d.lay.nx * d.lay.ny;
    for (int e = tid; e < BTX * BTY; e += BNT) {
      const int i = i0 + (e % BTX), j = j0 + (e / BTX);
      if (i >= d.lay.nx || j >= d.lay.ny) continue;
      const long long o = (long long)j * d.lay.nx + i, p = d.lay.idx(i, j);
#pragma unroll
      for (int c = 0; c < 4; ++c) d.U[c * n + o] = d.N[c * d.lay.plane + p];
    }
  }
}

}  // namespace js

// =======================================================================================
// host side
// =======================================================================================
using js::InstDesc;

struct js_batch {
  int count = 0;
  cudaStream_t stream = nullptr;
  std::vector<js_ctx*> ctx;      // one context per instance (buffers, IB tables, tags)
  std::vector<InstDesc> desc;    // host copy
  InstDesc* d_desc = nullptr;
  int* d_tile0 = nullptr;
  long long* d_ghost0 = nullptr;
  long long* d_halo0 = nullptr;
  unsigned long long* d_red = nullptr;
  unsigned* d_bar = nullptr;
  int* d_err = nullptr;
  int blocks = 0;
  int ntiles = 0;
  long long cells = 0;
  bool states_set = false;
  // reverse: instances spread over a few streams (each has its own workspace)
  std::vector<cudaStream_t> rstreams;
  std::vector<cudaEvent_t> revents;  // [0]: fork from the batch stream, [1..]: joins
};

// accessors of a context's internals (defined in js_host.cu)
void js_internal_desc(js_ctx* c, js::InstDesc* d);

namespace {
size_t batch_smem() { return js::BStageV::SMEM > js::BStageE::SMEM ? js::BStageV::SMEM : js::BStageE::SMEM; }
}  // namespace

extern "C" {

void js_batch_destroy(js_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
  for (cudaStream_t r : b->rstreams) cudaStreamDestroy(r);
  for (cudaEvent_t e : b->revents) cudaEventDestroy(e);
  for (js_ctx* c : b->ctx) js_destroy(c);
  cudaFree(b->d_desc); cudaFree(b->d_tile0); cudaFree(b->d_ghost0); cudaFree(b->d_halo0);
  cudaFree(b->d_red); cudaFree(b->d_bar); cudaFree(b->d_err);
  delete b;
}

int js_batch_create(int count, const js_grid* grids, const js_params* params, const js_boundary* bcs,
                    const double* const* sdf_host, void* stream, js_batch** out) {
  if (!out || count < 1 || !grids || !params || !bcs) return JS_ERR_ARG;
  *out = nullptr;
  js_batch* b = new (std::nothrow) js_batch();
  if (!b) return JS_ERR_NOMEM;
  b->count = count;
  b->stream = (cudaStream_t)stream;
  std::vector<int> tile0(count + 1, 0);
  std::vector<long long> ghost0(count + 1, 0), halo0(count + 1, 0);
  for (int k = 0; k < count; ++k) {
    if (grids[k].ny < 2) { js_batch_destroy(b); return JS_ERR_ARG; }  // 2D instances only
    js_ctx* c = nullptr;
    const int rc = js_create(&grids[k], &params[k], &bcs[k], sdf_host ? sdf_host[k] : nullptr, stream, &c);
    if (rc != JS_OK) { js_batch_destroy(b); return rc; }
    b->ctx.push_back(c);
    InstDesc d;
    js_internal_desc(c, &d);
    d.ntx = (grids[k].nx + js::BTX - 1) / js::BTX;
    d.nty = (grids[k].ny + js::BTY - 1) / js::BTY;
    b->desc.push_back(d);
    tile0[k + 1] = tile0[k] + d.ntx * d.nty;
    ghost0[k + 1] = ghost0[k] + d.ib.n;
    halo0[k + 1] = halo0[k] + js::halo_count(d.lay);
    b->cells += (long long)grids[k].nx * grids[k].ny;
  }
  b->ntiles = tile0[count];
  const size_t smem = batch_smem();
  if (cudaFuncSetAttribute(js::batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    js_batch_destroy(b);
    return JS_ERR_CUDA;
  }
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, js::batch_kernel, js::BNT, smem);
  if (!coop || per_sm < 1) { js_batch_destroy(b); return JS_ERR_CUDA; }
  b->blocks = sms * per_sm;
  if (cudaMalloc(&b->d_desc, sizeof(InstDesc) * count) != cudaSuccess ||
      cudaMalloc(&b->d_tile0, sizeof(int) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_ghost0, sizeof(long long) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_halo0, sizeof(long long) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_red, sizeof(unsigned long long) * 4 * count) != cudaSuccess ||
      cudaMalloc(&b->d_bar, 2 * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&b->d_err, sizeof(int)) != cudaSuccess) {
    js_batch_destroy(b);
    return JS_ERR_NOMEM;
  }
  if (cudaMemcpy(b->d_tile0, tile0.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_ghost0, ghost0.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_halo0, halo0.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {  // the batch stream may be non-blocking
    js_batch_destroy(b);
    return JS_ERR_CUDA;
  }
  *out = b;
  return JS_OK;
}

int js_batch_set_states(js_batch* b, double* const* U) {
  if (!b || !U) return JS_ERR_ARG;
  for (int k = 0; k < b->count; ++k) {
    if (!U[k]) return JS_ERR_ARG;
    b->desc[k].U = U[k];
  }
  if (cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(InstDesc) * b->count, cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return JS_ERR_CUDA;
  b->states_set = true;
  return JS_OK;
}

static int batch_launch(js_batch* b, double cfl, int n_steps, double* t_dev, double* dt_log, int extra,
                        double budget_s) {
  js::BatchArgs a;
  a.inst = b->d_desc;
  a.count = b->count;
  a.tile0 = b->d_tile0;
  a.ghost0 = b->d_ghost0;
  a.halo0 = b->d_halo0;
  a.red = b->d_red;
  a.bar = b->d_bar;
  a.err = b->d_err;
  a.t = t_dev;
  a.dt_log = dt_log;
  a.cfl = cfl;
  a.n_steps = n_steps;
  a.extra_arrivals = extra;
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  a.budget = (long long)(budget_s * 1e3 * (khz > 0 ? khz : 2000000));
  void* args[] = {&a};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)js::batch_kernel, dim3(b->blocks), dim3(js::BNT), args,
                                                    batch_smem(), b->stream);
  return e == cudaSuccess ? JS_OK : JS_ERR_CUDA;
}

int js_batch_step(js_batch* b, double cfl, int n_steps, double* t_dev, double* dt_log) {
  if (!b || !b->states_set || !(cfl > 0.0) || n_steps < 0) return JS_ERR_ARG;
  return batch_launch(b, cfl, n_steps, t_dev, dt_log, 0, 2.0);
}

int js_batch_step_vjp(js_batch* b, double* const* U_n, const double* dt, double* const* lam_np1,
                      double* const* lam_n, double* const* p_bar) {
  if (!b || !U_n || !dt || !lam_np1 || !lam_n) return JS_ERR_ARG;
  // the instances are independent: up to kRevStreams of them run at once, each on its own
  // stream forked from and joined back to the batch stream
  constexpr int kRevStreams = 8;
  const int ns = b->count < kRevStreams ? b->count : kRevStreams;
  while ((int)b->rstreams.size() < ns) {
    cudaStream_t r;
    if (cudaStreamCreateWithFlags(&r, cudaStreamNonBlocking) != cudaSuccess) return JS_ERR_CUDA;
    b->rstreams.push_back(r);
  }
  while ((int)b->revents.size() < ns + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return JS_ERR_CUDA;
    b->revents.push_back(e);
  }
  if (cudaEventRecord(b->revents[0], b->stream) != cudaSuccess) return JS_ERR_CUDA;
  for (int r = 0; r < ns; ++r)
    if (cudaStreamWaitEvent(b->rstreams[r], b->revents[0], 0) != cudaSuccess) return JS_ERR_CUDA;
  int rc = JS_OK;
  for (int k = 0; k < b->count && rc == JS_OK; ++k) {
    js_ctx* c = b->ctx[k];
    js_set_stream(c, b->rstreams[k % ns]);
    rc = js_step_vjp(c, U_n[k], dt[k], lam_np1[k], lam_n[k], p_bar ? p_bar[k] : nullptr);
  }
  for (int r = 0; r < ns; ++r) {
    if (cudaEventRecord(b->revents[r + 1], b->rstreams[r]) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->revents[r + 1], 0) != cudaSuccess)
      return JS_ERR_CUDA;
  }
  for (int k = 0; k < b->count; ++k) js_set_stream(b->ctx[k], b->stream);
  return rc;
}

int js_batch_test_timeout(js_batch* b, double budget_s) {
  if (!b || !b->states_set || !(budget_s > 0.0) || budget_s > 2.0) return JS_ERR_ARG;
  return batch_launch(b, 0.5, 0, nullptr, nullptr, 1, budget_s);
}

int js_batch_sync_status(js_batch* b) {
  if (!b) return JS_ERR_ARG;
  int h = 0;
  if (cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return JS_ERR_CUDA;
  if (cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return JS_ERR_CUDA;
  if (h & js::ERR_TIMEOUT_BIT) return JS_ERR_TIMEOUT;
  if (h & js::ERR_NONPHYSICAL_BIT) return JS_ERR_NONPHYSICAL;
  return JS_OK;
}

int js_batch_info(js_batch* b, int* blocks, int* tiles, long long* cells) {
  if (!b) return JS_ERR_ARG;
  if (blocks) *blocks = b->blocks;
  if (tiles) *tiles = b->ntiles;
  if (cells) *cells = b->cells;
  return JS_OK;
}

js_ctx* js_batch_instance(js_batch* b, int k) {
  if (!b || k < 0 || k >= b->count) return nullptr;
  return b->ctx[k];
}

}  // extern "C"
