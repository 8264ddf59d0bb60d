// Forward kernels of the FP64 finite-volume step (arXiv 2601.04400, Sec. 2):
//   bc_fill      domain halos (transmissive / reflective / periodic / inflow), 3 deep
//   ib_fill      ghost-cell immersed boundary: slip-wall mirror of the bilinear image-point
//                interpolation of fluid cells (Sec. 2, Fig. 1(c))
//   stage2d      one fused kernel per Runge-Kutta stage: conserved tile + halo -> primitives
//                in shared memory -> x sweep (WENO5, HLLC, viscous flux, divergence) into a
//                shared accumulator -> y sweep, RK stage combination, store
//   stage1d      the same along a single line (ny == 1)
//   cfl_reduce   maximum wave speed and minimum density (bit-exact IEEE arithmetic)
#include <cuda_runtime.h>
#include <math_constants.h>

#include "js_device.cuh"
#include "js_internal.h"
#include "js_fill.cuh"
#include "js_stage.cuh"

namespace js {

// =======================================================================================
// domain halo
// =======================================================================================
__global__ void bc_fill_kernel(double* __restrict__ U, Lay lay, BcArgs bc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < halo_count(lay)) bc_fill_one(U, lay, bc, t);
}

// =======================================================================================
// immersed-boundary ghost states
// =======================================================================================
__global__ void ib_fill_kernel(double* __restrict__ U, Lay lay, IbArgs ib, double gamma, int wall) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < ib.n) ib_fill_one(U, lay, ib, gamma, wall, k);
}

// =======================================================================================
// layout conversion
// =======================================================================================
__global__ void pack_kernel(const double* __restrict__ U, double* __restrict__ P, Lay lay) {
  const long long n = (long long)lay.nx * lay.ny;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * n) return;
  const int c = (int)(t / n);
  const long long o = t % n;
  const int i = (int)(o % lay.nx), j = (int)(o / lay.nx);
  P[c * lay.plane + lay.idx(i, j)] = U[t];
}

__global__ void unpack_kernel(const double* __restrict__ P, double* __restrict__ U, Lay lay) {
  const long long n = (long long)lay.nx * lay.ny;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * n) return;
  const int c = (int)(t / n);
  const long long o = t % n;
  const int i = (int)(o % lay.nx), j = (int)(o / lay.nx);
  U[t] = P[c * lay.plane + lay.idx(i, j)];
}

// row blocks of a [4][ny][nx] state for the halo exchange of a y-decomposed grid
__global__ void rows_pack_kernel(double* __restrict__ U, long long plane, long long off, long long m,
                                 double* __restrict__ buf, int zero) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * m) return;
  const long long k = (t / m) * plane + off + t % m;
  buf[t] = U[k];
  if (zero) U[k] = 0.0;
}

__global__ void rows_unpack_kernel(double* __restrict__ U, long long plane, long long off, long long m,
                                   const double* __restrict__ buf, int add) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * m) return;
  const long long k = (t / m) * plane + off + t % m;
  U[k] = add ? U[k] + buf[t] : buf[t];
}

__global__ void prim_to_cons_kernel(const double* W, double* U, long long n, double g1) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double r = W[t], u = W[n + t], v = W[2 * n + t], p = W[3 * n + t];
  U[t] = r;
  U[n + t] = r * u;
  U[2 * n + t] = r * v;
  U[3 * n + t] = fma(0.5 * r, fma(u, u, v * v), p * g1);
}

// =======================================================================================
// CFL reduction: rate = (|u| + a)/dx [+ (|v| + a)/dy] and rho over fluid cells, the rate in
// IEEE-rounded intrinsics in the oracle's operation order, so equal states give equal dt.
// Two passes keep that result while taking the IEEE rate of few cells: pass 1 takes every
// fluid cell's rate with the fast reciprocal and reciprocal square root, the exact minimum
// density, the maximum of these approximate rates and each block's maximum; pass 2 takes the
// IEEE rate only in blocks, and of cells, whose approximate rate reaches (1 - CFL_MARGIN) of
// that maximum (once per run of cells with identical states along a row).
// The approximation's relative error is a few ulp plus the pressure's cancellation error,
// about (E/p) ulp.  Pass 1 therefore uses it only where p > 1e-8 E (error below 1e-7) and takes
// the IEEE rate itself elsewhere (near-vacuum or hypersonic cells, non-physical ones), so every
// pass-1 rate is within CFL_MARGIN/2 of the IEEE rate, the cell of the largest IEEE rate is
// always a pass-2 candidate, and the result is the one-pass IEEE maximum for every state.
// A non-physical fluid cell has the rate +infinity in both passes (cfl_rate).
// =======================================================================================
constexpr double CFL_MARGIN = 4e-6;

__device__ __forceinline__ double cfl_rate_fast(double r, double mx, double my, double E, double gamma, double dx,
                                                double dy, double idx, double idy, bool two_d) {
  if (!(r > 1e-290) || !(r < 1e290)) return cfl_rate(r, mx, my, E, gamma, dx, dy, two_d);
  const double rr = recip(r);
  const double u = mx * rr, v = my * rr;
  const double ke = (0.5 * r) * fma(u, u, v * v);
  const double p = (gamma - 1.0) * (E - ke);
  // p <= 1e-8 E, p <= 0 or NaN: the approximation's error bound does not hold
  if (!(p > 1e-8 * E) || !(E < 1e290)) return cfl_rate(r, mx, my, E, gamma, dx, dy, two_d);
  const double c2 = (gamma * p) * rr;
  const double a = (c2 > 1e-290) ? c2 * rsqrt_nr(c2) : sqrt(c2);
  double s = (fabs(u) + a) * idx;
  if (two_d) s = fma(fabs(v) + a, idy, s);
  return s;
}

// block maximum (thread 0 holds it) and, when rmin != nullptr, block minimum
__device__ __forceinline__ void cfl_block_reduce(double& rate, double* rmin) {
  for (int o = 16; o > 0; o >>= 1) {
    rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    if (rmin) *rmin = fmin(*rmin, __shfl_xor_sync(0xffffffffu, *rmin, o));
  }
  __shared__ double sr[32], sm[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sr[wid] = rate;
    if (rmin) sm[wid] = *rmin;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    rate = (lane < nw) ? sr[lane] : 0.0;
    if (rmin) *rmin = (lane < nw) ? sm[lane] : __longlong_as_double(0x7ff0000000000000LL);
    for (int o = 16; o > 0; o >>= 1) {
      rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
      if (rmin) *rmin = fmin(*rmin, __shfl_xor_sync(0xffffffffu, *rmin, o));
    }
  }
}

// the state the reduction reads: the user layout [4][ny][nx] (PADDED false: cell t at t, planes
// n apart) or a context's padded buffer (cell t = (i, j) at off + j pitch + i, planes `plane` apart)
struct CflSrc {
  const double* U;
  long long plane, off;
  int nx, pitch;
};
template <bool PADDED>
__device__ __forceinline__ long long cfl_at(const CflSrc& q, long long t) {
  return PADDED ? q.off + (t / q.nx) * q.pitch + t % q.nx : t;
}

template <bool PADDED>
__global__ void cfl_pass1_kernel(CflSrc q, long long n, int two_d,
                                 const unsigned char* __restrict__ tag, double gamma, double dx, double dy,
                                 double idx, double idy, unsigned long long* __restrict__ red,
                                 double* __restrict__ bmax) {
  double rate = 0.0, rmin = __longlong_as_double(0x7ff0000000000000LL);
  const double* __restrict__ U = q.U;
  const long long P = q.plane;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    if (tag && tag[t] != 0) continue;
    const long long e = cfl_at<PADDED>(q, t);
    const double r = U[e];
    rate = fmax(rate, cfl_rate_fast(r, U[P + e], U[2 * P + e], U[3 * P + e], gamma, dx, dy, idx, idy, two_d != 0));
    rmin = fmin(rmin, r);
  }
  cfl_block_reduce(rate, &rmin);
  if (threadIdx.x == 0) {
    // non-negative doubles order like their bit patterns (a negative density is a non-physical
    // cell, whose infinite rate makes the step size 0 whatever the minimum holds)
    bmax[blockIdx.x] = rate;
    atomicMax(&red[2], (unsigned long long)__double_as_longlong(rate));
    atomicMin(&red[1], (unsigned long long)__double_as_longlong(rmin));
  }
}

// bitwise equality of two states (identical states have identical IEEE rates)
__device__ __forceinline__ bool same_bits(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}

// A candidate cell whose left neighbour in its row is a fluid cell with the identical state
// leaves the IEEE rate to that neighbour (also a candidate, in a block that passes the test):
// of a uniform run of cells, only the first takes it.  The threads of a warp hold consecutive
// cells, so the neighbour's state comes from the next lower lane.
template <bool PADDED>
__global__ void cfl_pass2_kernel(CflSrc q, long long n, int nx, int two_d,
                                 const unsigned char* __restrict__ tag, double gamma, double dx, double dy,
                                 double idx, double idy, unsigned long long* __restrict__ red,
                                 const double* __restrict__ bmax) {
  const double thr = __longlong_as_double((long long)red[2]) * (1.0 - CFL_MARGIN);
  if (!(bmax[blockIdx.x] >= thr)) return;  // the same for the whole block
  const int lane = threadIdx.x & 31;
  const double* __restrict__ U = q.U;
  const long long P = q.plane;
  const long long stride = (long long)gridDim.x * blockDim.x;
  double rate = 0.0;
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x - lane); base < n; base += stride) {
    const long long t = base + lane;
    const bool in = t < n;
    bool fl = false;
    double r = 0.0, mx = 0.0, my = 0.0, E = 0.0;
    if (in) {
      fl = !(tag && tag[t] != 0);
      const long long e = cfl_at<PADDED>(q, t);
      r = U[e];
      mx = U[P + e];
      my = U[2 * P + e];
      E = U[3 * P + e];
    }
    double rl = __shfl_up_sync(0xffffffffu, r, 1), mxl = __shfl_up_sync(0xffffffffu, mx, 1);
    double myl = __shfl_up_sync(0xffffffffu, my, 1), El = __shfl_up_sync(0xffffffffu, E, 1);
    bool fll = __shfl_up_sync(0xffffffffu, fl ? 1 : 0, 1) != 0;
    if (lane == 0 && in && t > 0) {
      fll = !(tag && tag[t - 1] != 0);
      const long long e = cfl_at<PADDED>(q, t - 1);
      rl = U[e];
      mxl = U[P + e];
      myl = U[2 * P + e];
      El = U[3 * P + e];
    }
    if (in && fl && cfl_rate_fast(r, mx, my, E, gamma, dx, dy, idx, idy, two_d != 0) >= thr) {
      const bool same = (t % nx != 0) && fll && same_bits(r, rl) && same_bits(mx, mxl) && same_bits(my, myl) &&
                        same_bits(E, El);
      if (!same) rate = fmax(rate, cfl_rate(r, mx, my, E, gamma, dx, dy, two_d != 0));
    }
  }
  cfl_block_reduce(rate, nullptr);
  if (threadIdx.x == 0) atomicMax(&red[0], (unsigned long long)__double_as_longlong(rate));
}

// Device step size from the CFL reduction in red, with js_max_dt's arithmetic (the same IEEE
// operations in the same order): dt = cfl / rate, capped by the viscous limit
// cfl hmin^2 rho_min / (2 mu lim); clipped to t_end - t when t + dt > t_end (t: running time,
// or nullptr), the step inactive once t reaches t_end or when dt is not a positive number
// (a non-physical state: the error flag is set).  Writes the stage constants dtc and dt_log[k].
__global__ void cfl_dt_kernel(const unsigned long long* __restrict__ red, double cfl, double dx, double dy,
                              double nu, int visc, double mu, double lim, double hmin, double* t, double t_end,
                              double* __restrict__ dtc, double* __restrict__ dt_log, int k, int* err) {
  const double rate = __longlong_as_double((long long)red[0]);
  const double rmin = __longlong_as_double((long long)red[1]);
  double dt = __ddiv_rn(cfl, rate);
  if (visc) {
    const double dtv = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(cfl, hmin), hmin), rmin),
                                 __dmul_rn(__dmul_rn(2.0, mu), lim));
    dt = (dtv < dt) ? dtv : dt;
  }
  bool active = true;
  if (!(dt > 0.0) || !(dt < CUDART_INF)) {
    atomicOr(err, ERR_NONPHYSICAL_BIT);
    active = false;
  }
  if (active && t != nullptr && t_end > 0.0) {
    const double tc = *t;
    if (!(tc < t_end)) active = false;
    else if (__dadd_rn(tc, dt) > t_end) dt = __dsub_rn(t_end, tc);
  }
  if (!active) dt = 0.0;
  if (active && t != nullptr) *t = __dadd_rn(*t, dt);
  dtc[0] = __ddiv_rn(dt, dx);
  dtc[1] = __ddiv_rn(dt, dy);
  dtc[2] = __ddiv_rn(__dmul_rn(dt, nu), __dmul_rn(dx, dx));
  dtc[3] = __ddiv_rn(__dmul_rn(dt, nu), __dmul_rn(dy, dy));
  dtc[4] = active ? 1.0 : 0.0;
  dtc[5] = dt;
  if (dt_log) dt_log[k] = dt;
}

__global__ void cfl_init_kernel(unsigned long long* red) {
  red[0] = 0ULL;                    // IEEE rate maximum
  red[1] = 0x7ff0000000000000ULL;   // density minimum
  red[2] = 0ULL;                    // approximate rate maximum
}

// the stage constants of a launch: the arguments, or those of the device step size
__device__ __forceinline__ bool stage_constants(const StageArgs& a0, StageArgs& a) {
  a = a0;
  if (a0.dtc == nullptr) return true;
  a.cx = a0.dtc[0];
  a.cy = a0.dtc[1];
  a.avx = a0.dtc[2];
  a.avy = a0.dtc[3];
  return a0.dtc[4] != 0.0;
}

template <int TX, int TY, int LX, int LY, bool VISC, bool RHS>
__global__ void __launch_bounds__(Stage2D<TX, TY, LX, LY, VISC, RHS>::NT)
stage2d_kernel(StageArgs a0) {
  StageArgs a;
  if (!stage_constants(a0, a)) return;
  extern __shared__ double smem[];
  stage_tile<TX, TY, LX, LY, VISC, RHS>(a, blockIdx.x, blockIdx.y, smem);
}

// persistent concurrent-sweep stage kernel: blocks stride over the tiles; with SAVE the
// WENO5 internals of the stage go to a.wsave for the reverse pass
template <int TX, int TY, int LX, int LY, bool VISC, bool RHS, bool SAVE, bool IMG = false>
__global__ void __launch_bounds__(Stage2DC<TX, TY, LX, LY, VISC>::NT, SAVE ? 3 : 1)
stage2dc_kernel(StageArgs a0, int ntx, int ntiles) {
  StageArgs a;
  if (!stage_constants(a0, a)) return;
  extern __shared__ double smem[];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    stage_tile_c<TX, TY, LX, LY, VISC, RHS, false, SAVE, IMG>(a, t % ntx, t / ntx, smem);
    __syncthreads();
  }
}

// the same with the tile staged by TMA (tensor map of the stage input as a grid constant)
template <int TX, int TY, int LX, int LY, bool VISC, bool RHS, bool SAVE, bool IMG = false>
__global__ void __launch_bounds__(Stage2DC<TX, TY, LX, LY, VISC, true>::NT, SAVE ? 3 : 1)
stage2dc_tma_kernel(StageArgs a0, int ntx, int ntiles, const __grid_constant__ TensorMap128 tmap) {
  StageArgs a;
  if (!stage_constants(a0, a)) return;
  extern __shared__ __align__(128) double smem[];
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  unsigned phase = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    stage_tile_c<TX, TY, LX, LY, VISC, RHS, true, SAVE, IMG>(a, t % ntx, t / ntx, smem, &tmap, &bar, &phase);
    __syncthreads();
  }
}

template <int TX, int LX, bool VISC, bool RHS>
__global__ void __launch_bounds__(TX / LX) stage1d_kernel(StageArgs a0) {
  StageArgs a;
  if (!stage_constants(a0, a)) return;
  constexpr int NPL = VISC ? 5 : 4;
  constexpr int PS = TX + 6;
  constexpr int NT = TX / LX;
  __shared__ double sq[NPL * PS];
  const Gas g{a.gamma, a.gm1, a.g1};
  const int tx0 = blockIdx.x * TX;
  const int W = a.lay.nx + 6;
  for (int col = threadIdx.x; col < PS; col += NT) {
    int gx = tx0 + col;
    gx = (gx < W) ? gx : W - 1;
    const double r = a.Uin[gx], mx = a.Uin[a.lay.plane + gx], my = a.Uin[2 * a.lay.plane + gx],
                 E = a.Uin[3 * a.lay.plane + gx];
    double u, v, p, T;
    cons_to_prim(r, mx, my, E, g, u, v, p, T);
    sq[col] = r;
    sq[PS + col] = u;
    sq[2 * PS + col] = v;
    sq[3 * PS + col] = p;
    if (NPL == 5) sq[4 * PS + col] = T;
  }
  __syncthreads();
  const int xs = threadIdx.x * LX;
  const double zero[4] = {0.0, 0.0, 0.0, 0.0};
  sweep_line<0, VISC, false, LX>(sq, PS, xs + 3, 1, 0, g, a.vx, [&](int k, const double dF[4]) {
    const int gi = tx0 + xs + k;
    if (gi < a.lay.nx) {
      double ax[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) ax[c] = a.cx * dF[c];
      finish_cell<RHS, true>(a, gi, 0, ax, zero, sq[xs + k + 3], sq[3 * PS + xs + k + 3]);
    }
  });
}

// =======================================================================================
// launchers
// =======================================================================================
namespace {
// 1D grids are small (a few hundred cells): short segments, so that more threads share the
// latency-bound sweep
constexpr int TX1 = 32, LX1 = 4;

template <int TX, int TY, int LX, int LY, bool VISC, bool RHS>
cudaError_t launch_stage2d(const StageArgs& a, cudaStream_t s) {
  using S = Stage2D<TX, TY, LX, LY, VISC, RHS>;
  auto k = stage2d_kernel<TX, TY, LX, LY, VISC, RHS>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((a.lay.nx + TX - 1) / TX, (a.lay.ny + TY - 1) / TY);
  k<<<grid, S::NT, S::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int TX, int TY, int LX, int LY, bool VISC, bool RHS, bool SAVE = false, bool IMG = false>
cudaError_t launch_stage2dc(const StageArgs& a, cudaStream_t s) {
  using S = Stage2DC<TX, TY, LX, LY, VISC>;
  auto k = stage2dc_kernel<TX, TY, LX, LY, VISC, RHS, SAVE, IMG>;
  constexpr size_t SM = S::SMEM;
  static int resident = 0;  // blocks resident on the whole GPU
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, S::NT, SM);
    if (e != cudaSuccess) return e;
    resident = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int ntx = (a.lay.nx + TX - 1) / TX, nty = (a.lay.ny + TY - 1) / TY;
  const int ntiles = ntx * nty;
  k<<<ntiles < resident ? ntiles : resident, S::NT, SM, s>>>(a, ntx, ntiles);
  return cudaGetLastError();
}

template <int TX, int TY, int LX, int LY, bool VISC, bool RHS, bool SAVE = false, bool IMG = false>
cudaError_t launch_stage2dc_tma(const StageArgs& a, const TensorMap128* tmap, cudaStream_t s) {
  using S = Stage2DC<TX, TY, LX, LY, VISC, true>;
  auto k = stage2dc_tma_kernel<TX, TY, LX, LY, VISC, RHS, SAVE, IMG>;
  constexpr size_t SM = S::SMEM;
  static int resident = 0;
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, S::NT, SM);
    if (e != cudaSuccess) return e;
    resident = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int ntx = (a.lay.nx + TX - 1) / TX, nty = (a.lay.ny + TY - 1) / TY;
  const int ntiles = ntx * nty;
  k<<<ntiles < resident ? ntiles : resident, S::NT, SM, s>>>(a, ntx, ntiles, *tmap);
  return cudaGetLastError();
}

// tile shapes (TX x TY cells, x / y segment lengths LX / LY) the tuner chooses from:
// 0 concurrent sweeps with TMA staging, 1-3 concurrent sweeps with plain loads in
// persistent blocks, 4 sequential sweeps in one warp per tile
template <bool VISC, bool RHS>
cudaError_t launch_stage2d_variant(const StageArgs& a, int variant, const TensorMap128* tmap, cudaStream_t s) {
  switch (variant) {
    case 1: return launch_stage2dc<32, 32, 16, 16, VISC, RHS>(a, s);
    case 2: return launch_stage2dc<32, 16, 16, 16, VISC, RHS>(a, s);
    case 3: return launch_stage2dc<64, 16, 16, 16, VISC, RHS>(a, s);
    case 4: return launch_stage2d<32, 16, 16, 16, VISC, RHS>(a, s);
    default:
      if (tmap == nullptr) return launch_stage2dc<32, 32, 16, 16, VISC, RHS>(a, s);
      return launch_stage2dc_tma<32, 32, 16, 16, VISC, RHS>(a, tmap, s);
  }
}

template <bool VISC, bool RHS>
cudaError_t launch_stage1d(const StageArgs& a, cudaStream_t s) {
  dim3 grid((a.lay.nx + TX1 - 1) / TX1);
  stage1d_kernel<TX1, LX1, VISC, RHS><<<grid, TX1 / LX1, 0, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_stage_save(const StageArgs& a, bool visc, const TensorMap128* tmap, cudaStream_t s) {
  if (a.lay.ny == 1 || a.wsave == nullptr) return cudaErrorInvalidValue;
  if (tmap != nullptr)
    return visc ? launch_stage2dc_tma<32, 32, 16, 16, true, false, true>(a, tmap, s)
                : launch_stage2dc_tma<32, 32, 16, 16, false, false, true>(a, tmap, s);
  return visc ? launch_stage2dc<32, 32, 16, 16, true, false, true>(a, s)
              : launch_stage2dc<32, 32, 16, 16, false, false, true>(a, s);
}

cudaError_t launch_stage_img(const StageArgs& a, bool visc, const TensorMap128* tmap, cudaStream_t s) {
  if (a.lay.ny == 1 || a.img == nullptr) return cudaErrorInvalidValue;
  if (tmap != nullptr)
    return visc ? launch_stage2dc_tma<32, 32, 16, 16, true, false, false, true>(a, tmap, s)
                : launch_stage2dc_tma<32, 32, 16, 16, false, false, false, true>(a, tmap, s);
  return visc ? launch_stage2dc<32, 32, 16, 16, true, false, false, true>(a, s)
              : launch_stage2dc<32, 32, 16, 16, false, false, false, true>(a, s);
}

cudaError_t launch_stage(const StageArgs& a, bool visc, bool rhs, int variant, const TensorMap128* tmap,
                         cudaStream_t s) {
  if (a.lay.ny == 1) {
    if (visc) return rhs ? launch_stage1d<true, true>(a, s) : launch_stage1d<true, false>(a, s);
    return rhs ? launch_stage1d<false, true>(a, s) : launch_stage1d<false, false>(a, s);
  }
  if (visc)
    return rhs ? launch_stage2d_variant<true, true>(a, variant, tmap, s)
               : launch_stage2d_variant<true, false>(a, variant, tmap, s);
  return rhs ? launch_stage2d_variant<false, true>(a, variant, tmap, s)
             : launch_stage2d_variant<false, false>(a, variant, tmap, s);
}

cudaError_t launch_bc_fill(double* U, const Lay& lay, const BcArgs& bc, cudaStream_t s) {
  const long long n = halo_count(lay);
  const int bs = 256;
  bc_fill_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(U, lay, bc);
  return cudaGetLastError();
}

cudaError_t launch_ib_fill(double* U, const Lay& lay, const IbArgs& ib, double gamma, int wall, cudaStream_t s) {
  if (ib.n == 0) return cudaSuccess;
  const int bs = 128;
  ib_fill_kernel<<<(ib.n + bs - 1) / bs, bs, 0, s>>>(U, lay, ib, gamma, wall);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double* U, double* P, const Lay& lay, cudaStream_t s) {
  const long long n = 4LL * lay.nx * lay.ny;
  const int bs = 256;
  pack_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(U, P, lay);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const double* P, double* U, const Lay& lay, cudaStream_t s) {
  const long long n = 4LL * lay.nx * lay.ny;
  const int bs = 256;
  unpack_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(P, U, lay);
  return cudaGetLastError();
}

cudaError_t launch_rows_pack(double* U, int nx, int ny, int row0, int nrows, double* buf, int zero, cudaStream_t s) {
  const long long m = (long long)nrows * nx;
  if (m == 0) return cudaSuccess;
  rows_pack_kernel<<<(unsigned)((4 * m + 255) / 256), 256, 0, s>>>(U, (long long)nx * ny, (long long)row0 * nx, m,
                                                                   buf, zero);
  return cudaGetLastError();
}

cudaError_t launch_rows_unpack(double* U, int nx, int ny, int row0, int nrows, const double* buf, int add,
                               cudaStream_t s) {
  const long long m = (long long)nrows * nx;
  if (m == 0) return cudaSuccess;
  rows_unpack_kernel<<<(unsigned)((4 * m + 255) / 256), 256, 0, s>>>(U, (long long)nx * ny, (long long)row0 * nx,
                                                                     m, buf, add);
  return cudaGetLastError();
}

cudaError_t launch_prim_to_cons(const double* W, double* U, long long n, double gamma, cudaStream_t s) {
  const int bs = 256;
  prim_to_cons_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(W, U, n, 1.0 / (gamma - 1.0));
  return cudaGetLastError();
}

cudaError_t launch_cfl_dt(const unsigned long long* red, double cfl, double dx, double dy, double nu, double mu,
                          double lim, double hmin, double* t, double t_end, double* dtc, double* dt_log, int k,
                          int* err, cudaStream_t s) {
  cfl_dt_kernel<<<1, 1, 0, s>>>(red, cfl, dx, dy, nu, mu > 0.0 ? 1 : 0, mu, lim, hmin, t, t_end, dtc, dt_log, k,
                                err);
  return cudaGetLastError();
}

cudaError_t launch_cfl(const double* U, const Lay& lay, const unsigned char* tag, double gamma, double dx,
                       double dy, unsigned long long* red, double* bmax, cudaStream_t s, bool padded) {
  cfl_init_kernel<<<1, 1, 0, s>>>(red);
  const long long n = (long long)lay.nx * lay.ny;
  const int bs = 256;
  long long blocks = (n + bs - 1) / bs;
  if (blocks > CFL_MAX_BLOCKS) blocks = CFL_MAX_BLOCKS;
  const int two_d = lay.ny > 1 ? 1 : 0;
  const CflSrc q{U, padded ? lay.plane : n, padded ? lay.idx(0, 0) : 0, lay.nx, padded ? lay.pitch : lay.nx};
  // both passes on the same grid: a block of pass 2 visits the cells its pass-1 maximum covers
  if (padded) {
    cfl_pass1_kernel<true><<<(unsigned)blocks, bs, 0, s>>>(q, n, two_d, tag, gamma, dx, dy, 1.0 / dx, 1.0 / dy, red,
                                                            bmax);
    cfl_pass2_kernel<true><<<(unsigned)blocks, bs, 0, s>>>(q, n, lay.nx, two_d, tag, gamma, dx, dy, 1.0 / dx,
                                                            1.0 / dy, red, bmax);
  } else {
    cfl_pass1_kernel<false><<<(unsigned)blocks, bs, 0, s>>>(q, n, two_d, tag, gamma, dx, dy, 1.0 / dx, 1.0 / dy, red,
                                                             bmax);
    cfl_pass2_kernel<false><<<(unsigned)blocks, bs, 0, s>>>(q, n, lay.nx, two_d, tag, gamma, dx, dy, 1.0 / dx,
                                                             1.0 / dy, red, bmax);
  }
  return cudaGetLastError();
}

}  // namespace js
