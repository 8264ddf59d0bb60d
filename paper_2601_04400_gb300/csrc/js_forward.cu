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

#include "js_device.cuh"
#include "js_internal.h"

namespace js {

// =======================================================================================
// domain halo
// =======================================================================================
__global__ void bc_fill_kernel(double* __restrict__ U, Lay lay, BcArgs bc) {
  const int nx = lay.nx, ny = lay.ny;
  const long long nxg = 6LL * ny;                       // x ghosts on interior rows
  const long long nyg = (ny > 1) ? 6LL * (nx + 6) : 0;  // y ghosts on the full padded width
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nxg + nyg) return;
  int i, j;
  if (t < nxg) {
    j = (int)(t / 6);
    const int r = (int)(t % 6);
    i = (r < 3) ? -(r + 1) : nx + (r - 3);
  } else {
    const long long u = t - nxg;
    i = (int)(u / 6) - 3;
    const int r = (int)(u % 6);
    j = (r < 3) ? -(r + 1) : ny + (r - 3);
  }
  // Resolve the source of ghost (i, j): the y rule first (it reads x-ghost columns, which
  // the x rule defines from interior cells), then the x rule; reflective sides flip the
  // normal momentum, inflow sides return a fixed state.
  bool flipx = false, flipy = false;
  int side_inflow = -1;
  if (j < 0 || j >= ny) {
    const int side = (j < 0) ? 2 : 3;
    const int k = (j < 0) ? -j : j - ny + 1;
    switch (bc.kind[side]) {
      case 0: j = (side == 2) ? 0 : ny - 1; break;
      case 1: j = (side == 2) ? k - 1 : ny - k; flipy = true; break;
      case 2: j = (side == 2) ? ny - k : k - 1; break;
      default: side_inflow = side; break;
    }
  }
  if (side_inflow < 0 && (i < 0 || i >= nx)) {
    const int side = (i < 0) ? 0 : 1;
    const int k = (i < 0) ? -i : i - nx + 1;
    switch (bc.kind[side]) {
      case 0: i = (side == 0) ? 0 : nx - 1; break;
      case 1: i = (side == 0) ? k - 1 : nx - k; flipx = true; break;
      case 2: i = (side == 0) ? nx - k : k - 1; break;
      default: side_inflow = side; break;
    }
  }
  double v[4];
  if (side_inflow >= 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = bc.inflow_cons[side_inflow][c];
  } else {
    const long long s = lay.idx(i, j);
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = U[c * lay.plane + s];
  }
  if (flipx) v[1] = -v[1];
  if (flipy) v[2] = -v[2];
  // destination: recompute from t
  int di, dj;
  if (t < nxg) {
    dj = (int)(t / 6);
    const int r = (int)(t % 6);
    di = (r < 3) ? -(r + 1) : nx + (r - 3);
  } else {
    const long long u = t - nxg;
    di = (int)(u / 6) - 3;
    const int r = (int)(u % 6);
    dj = (r < 3) ? -(r + 1) : ny + (r - 3);
  }
  const long long d = lay.idx(di, dj);
#pragma unroll
  for (int c = 0; c < 4; ++c) U[c * lay.plane + d] = v[c];
}

// =======================================================================================
// immersed-boundary ghost states
// =======================================================================================
__global__ void ib_fill_kernel(double* __restrict__ U, Lay lay, IbArgs ib, double gamma, int wall) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ib.n) return;
  double q[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const double w = ib.w[4 * k + m];
    if (w == 0.0) continue;
    const long long s = ib.src[4 * k + m];
    const double r = U[s], u = U[lay.plane + s] / r, v = U[2 * lay.plane + s] / r;
    const double p = (gamma - 1.0) * (U[3 * lay.plane + s] - 0.5 * r * (u * u + v * v));
    q[0] += w * r;
    q[1] += w * u;
    q[2] += w * v;
    q[3] += w * p;
  }
  const double nx = ib.nrm[2 * k], ny = ib.nrm[2 * k + 1];
  double ug, vg;
  if (wall == 0) {
    const double vn = q[1] * nx + q[2] * ny;
    ug = q[1] - 2.0 * vn * nx;
    vg = q[2] - 2.0 * vn * ny;
  } else {
    ug = -q[1];
    vg = -q[2];
  }
  const long long d = ib.dst[k];
  U[d] = q[0];
  U[lay.plane + d] = q[0] * ug;
  U[2 * lay.plane + d] = q[0] * vg;
  U[3 * lay.plane + d] = q[3] / (gamma - 1.0) + 0.5 * q[0] * (ug * ug + vg * vg);
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
// CFL reduction: rate = (|u| + a)/dx [+ (|v| + a)/dy] and rho over fluid cells.
// IEEE-rounded intrinsics in the oracle's operation order, so equal states give equal dt.
// =======================================================================================
__global__ void cfl_kernel(const double* __restrict__ U, long long n, int nx, int two_d,
                           const unsigned char* __restrict__ tag, double gamma, double dx, double dy,
                           unsigned long long* __restrict__ red) {
  double rate = 0.0, rmin = __longlong_as_double(0x7ff0000000000000LL);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    if (tag && tag[t] != 0) continue;
    const double r = U[t];
    const double u = __ddiv_rn(U[n + t], r), v = __ddiv_rn(U[2 * n + t], r);
    const double ke = __dmul_rn(__dmul_rn(0.5, r), __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)));
    const double p = __dmul_rn(gamma - 1.0, __dsub_rn(U[3 * n + t], ke));
    const double a = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), r));
    double s = __ddiv_rn(__dadd_rn(fabs(u), a), dx);
    if (two_d) s = __dadd_rn(s, __ddiv_rn(__dadd_rn(fabs(v), a), dy));
    rate = fmax(rate, s);
    rmin = fmin(rmin, r);
    (void)nx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
  }
  __shared__ double sr[32], sm[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sr[wid] = rate; sm[wid] = rmin; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    rate = (lane < nw) ? sr[lane] : 0.0;
    rmin = (lane < nw) ? sm[lane] : __longlong_as_double(0x7ff0000000000000LL);
    for (int o = 16; o > 0; o >>= 1) {
      rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
      rmin = fmin(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    }
    if (lane == 0) {
      // non-negative doubles order like their bit patterns
      atomicMax(&red[0], (unsigned long long)__double_as_longlong(rate));
      atomicMin(&red[1], (unsigned long long)__double_as_longlong(rmin));
    }
  }
}

__global__ void cfl_init_kernel(unsigned long long* red) {
  red[0] = 0ULL;
  red[1] = 0x7ff0000000000000ULL;
}

// =======================================================================================
// line sweep: WENO5 -> HLLC (+ viscous) -> flux differences, on primitives in shared memory
// =======================================================================================
// sq: shared planes rho, u, v, p (and T when VISC), plane stride ps; `base` = index of the
// first output cell of the segment, `st` = stride along the line, `ts` = stride across it.
// emit(k, dF) receives F_{k+1/2} - F_{k-1/2} (conserved order) for output cells k = 0..L-1.
template <int DIR, bool VISC, bool HAS_T, int L, class Emit>
__device__ __forceinline__ void sweep_line(const double* __restrict__ sq, int ps, int base, int st, int ts,
                                           const Gas& g, const ViscC& vc, Emit&& emit) {
  constexpr int PN = (DIR == 0) ? 1 : 2;  // plane of the face-normal velocity
  constexpr int PT = (DIR == 0) ? 2 : 1;  // plane of the tangential velocity
  Win w[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double* q = sq + c * ps;
    w[c].init(q[base - 3 * st], q[base - 2 * st], q[base - st], q[base]);
  }
  double prevL[4], prevF[4];
#pragma unroll 1
  for (int k = -1; k <= L; ++k) {
    const int cell = base + k * st;
    double Lf[4], Rf[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) w[c].step(sq[c * ps + cell + 2 * st], Lf[c], Rf[c]);
    if (k >= 0) {
      // face k - 1/2 between cells k-1 (left state prevL) and k (right state Rf)
      double ql[4], qr[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) { ql[c] = prevL[c]; qr[c] = Rf[c]; }
      if (!(ql[0] > 0.0 && ql[3] > 0.0 && qr[0] > 0.0 && qr[3] > 0.0)) {
        // positivity fallback: first-order (cell) states at this face
#pragma unroll
        for (int c = 0; c < 4; ++c) { ql[c] = sq[c * ps + cell - st]; qr[c] = sq[c * ps + cell]; }
      }
      double Fn[4];
      hllc(ql[0], ql[PN], ql[PT], ql[3], qr[0], qr[PN], qr[PT], qr[3], g, Fn);
      double F[4];
      F[0] = Fn[0];
      F[PN] = Fn[1];
      F[PT] = Fn[2];
      F[3] = Fn[3];
      if (VISC) {
        const int a = cell - st, b = cell;
        const double* un = sq + PN * ps;
        const double* ut = sq + PT * ps;
        const double* Tq = sq + 4 * ps;
        const double dun = un[b] - un[a], dut = ut[b] - ut[a], dT = Tq[b] - Tq[a];
        double tnn, tnt;
        if (HAS_T) {
          const double sun = (un[a + ts] - un[a - ts]) + (un[b + ts] - un[b - ts]);
          const double sut = (ut[a + ts] - ut[a - ts]) + (ut[b + ts] - ut[b - ts]);
          tnn = fma(vc.c43n, dun, -vc.c23t * sut);
          tnt = fma(vc.cn, dut, vc.ct * sun);
        } else {
          tnn = vc.c43n * dun;
          tnt = vc.cn * dut;
        }
        const double sbn = un[a] + un[b], sbt = ut[a] + ut[b];
        const double e = fma(0.5, fma(sbn, tnn, sbt * tnt), vc.ck * dT);
        F[PN] -= tnn;
        F[PT] -= tnt;
        F[3] -= e;
      }
      if (k >= 1) {
        double dF[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) dF[c] = F[c] - prevF[c];
        emit(k - 1, dF);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) prevF[c] = F[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) prevL[c] = Lf[c];
  }
}

// final combination for one interior cell; returns the value stored in the output
template <bool RHS>
__device__ __forceinline__ void finish_cell(const StageArgs& a, int gi, int gj, const double acc[4],
                                            const double dG[4], double rho, double p) {
  const long long pid = a.lay.idx(gi, gj);
  const bool fluid = (a.tag == nullptr) || (a.tag[(long long)gj * a.lay.nx + gi] == 0);
  double out[4];
  if (fluid) {
    if (!(rho > 0.0 && p > 0.0)) atomicOr(a.err, ERR_NONPHYSICAL_BIT);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double* Uc = a.Uin + c * a.lay.plane;
      const double us = RHS ? 0.0 : Uc[pid];
      double v = fma(-a.cy, dG[c], us - acc[c]);
      if (a.has_av) {
        v = fma(a.avx, (Uc[pid + 1] - 2.0 * Uc[pid]) + Uc[pid - 1], v);
        if (a.lay.ny > 1) v = fma(a.avy, (Uc[pid + a.lay.pitch] - 2.0 * Uc[pid]) + Uc[pid - a.lay.pitch], v);
      }
      if (!RHS && a.use_un) v = fma(a.rk_a, a.Un[c * a.lay.plane + pid], a.rk_b * v);
      out[c] = v;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = RHS ? 0.0 : a.Uin[c * a.lay.plane + pid];
  }
  if (RHS) {
    const long long n = (long long)a.lay.nx * a.lay.ny;
    const long long o = (long long)gj * a.lay.nx + gi;
#pragma unroll
    for (int c = 0; c < 4; ++c) a.Uout[c * n + o] = out[c];
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) a.Uout[c * a.lay.plane + pid] = out[c];
  }
}

// load the conserved tile with halo and convert to primitives in shared memory
template <int TX, int TY, int NPL, int NT>
__device__ __forceinline__ void load_tile(const StageArgs& a, double* sq, int ps, int sp, int ox, int oy,
                                          const Gas& g) {
  constexpr int CW = TX + 6, CH = TY + 6;
  const int W = a.lay.nx + 6;
  for (int e = threadIdx.x; e < CW * CH; e += NT) {
    const int row = e / CW, col = e - row * CW;
    int gx = ox + col, gy = oy + row;  // padded coordinates
    gx = (gx < W) ? gx : W - 1;
    gy = (gy < a.lay.H) ? gy : a.lay.H - 1;
    const long long s = (long long)gy * a.lay.pitch + gx;
    const double r = a.Uin[s], mx = a.Uin[a.lay.plane + s], my = a.Uin[2 * a.lay.plane + s],
                 E = a.Uin[3 * a.lay.plane + s];
    double u, v, p, T;
    cons_to_prim(r, mx, my, E, g, u, v, p, T);
    const int d = row * sp + col;
    sq[d] = r;
    sq[ps + d] = u;
    sq[2 * ps + d] = v;
    sq[3 * ps + d] = p;
    if (NPL == 5) sq[4 * ps + d] = T;
  }
}

template <int TX, int TY, int LX, int LY, bool VISC, bool RHS>
struct Stage2D {
  static constexpr int NPL = VISC ? 5 : 4;
  static constexpr int SP = TX + 7;  // odd row pitch (in doubles) of the shared tile
  static constexpr int PS = (TY + 6) * SP;
  static constexpr int NX_ITEMS = TY * (TX / LX);
  static constexpr int NY_ITEMS = TX * (TY / LY);
  static constexpr int NT = (NX_ITEMS > NY_ITEMS) ? NX_ITEMS : NY_ITEMS;
  static constexpr size_t SMEM = sizeof(double) * ((size_t)NPL * PS + 4 * TX * TY);
};

template <int TX, int TY, int LX, int LY, bool VISC, bool RHS>
__global__ void __launch_bounds__(Stage2D<TX, TY, LX, LY, VISC, RHS>::NT)
stage2d_kernel(StageArgs a) {
  using S = Stage2D<TX, TY, LX, LY, VISC, RHS>;
  extern __shared__ double smem[];
  double* sq = smem;
  double* acc = smem + S::NPL * S::PS;
  const Gas g{a.gamma, a.gm1, a.g1};
  const int tx0 = blockIdx.x * TX, ty0 = blockIdx.y * TY;  // interior origin of the tile
  load_tile<TX, TY, S::NPL, S::NT>(a, sq, S::PS, S::SP, tx0, ty0, g);
  __syncthreads();
  // x sweep: one thread per (row, segment)
  for (int it = threadIdx.x; it < S::NX_ITEMS; it += S::NT) {
    const int ty = it % TY, xs = (it / TY) * LX;
    const int base = (ty + 3) * S::SP + xs + 3;
    sweep_line<0, VISC, true, LX>(sq, S::PS, base, 1, S::SP, g, a.vx, [&](int k, const double dF[4]) {
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c * TX * TY + ty * TX + xs + k] = a.cx * dF[c];
    });
  }
  __syncthreads();
  // y sweep + stage combination: one thread per (column, segment)
  for (int it = threadIdx.x; it < S::NY_ITEMS; it += S::NT) {
    const int tx = it % TX, ys = (it / TX) * LY;
    const int base = (ys + 3) * S::SP + tx + 3;
    const int gi = tx0 + tx;
    sweep_line<1, VISC, true, LY>(sq, S::PS, base, S::SP, 1, g, a.vy, [&](int k, const double dG[4]) {
      const int ty = ys + k, gj = ty0 + ty;
      if (gi < a.lay.nx && gj < a.lay.ny) {
        double ax[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) ax[c] = acc[c * TX * TY + ty * TX + tx];
        const int sc = (ty + 3) * S::SP + tx + 3;
        finish_cell<RHS>(a, gi, gj, ax, dG, sq[sc], sq[3 * S::PS + sc]);
      }
    });
  }
}

template <int TX, int LX, bool VISC, bool RHS>
__global__ void __launch_bounds__(TX / LX) stage1d_kernel(StageArgs a) {
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
      finish_cell<RHS>(a, gi, 0, ax, zero, sq[xs + k + 3], sq[3 * PS + xs + k + 3]);
    }
  });
}

// =======================================================================================
// launchers
// =======================================================================================
namespace {
constexpr int TX2 = 32, TY2 = 16, LX2 = 16, LY2 = 16;
constexpr int TX1 = 64, LX1 = 16;

template <bool VISC, bool RHS>
cudaError_t launch_stage2d(const StageArgs& a, cudaStream_t s) {
  using S = Stage2D<TX2, TY2, LX2, LY2, VISC, RHS>;
  auto k = stage2d_kernel<TX2, TY2, LX2, LY2, VISC, RHS>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((a.lay.nx + TX2 - 1) / TX2, (a.lay.ny + TY2 - 1) / TY2);
  k<<<grid, S::NT, S::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <bool VISC, bool RHS>
cudaError_t launch_stage1d(const StageArgs& a, cudaStream_t s) {
  dim3 grid((a.lay.nx + TX1 - 1) / TX1);
  stage1d_kernel<TX1, LX1, VISC, RHS><<<grid, TX1 / LX1, 0, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_stage(const StageArgs& a, bool visc, bool rhs, cudaStream_t s) {
  if (a.lay.ny == 1) {
    if (visc) return rhs ? launch_stage1d<true, true>(a, s) : launch_stage1d<true, false>(a, s);
    return rhs ? launch_stage1d<false, true>(a, s) : launch_stage1d<false, false>(a, s);
  }
  if (visc) return rhs ? launch_stage2d<true, true>(a, s) : launch_stage2d<true, false>(a, s);
  return rhs ? launch_stage2d<false, true>(a, s) : launch_stage2d<false, false>(a, s);
}

cudaError_t launch_bc_fill(double* U, const Lay& lay, const BcArgs& bc, cudaStream_t s) {
  const long long n = 6LL * lay.ny + ((lay.ny > 1) ? 6LL * (lay.nx + 6) : 0);
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

cudaError_t launch_prim_to_cons(const double* W, double* U, long long n, double gamma, cudaStream_t s) {
  const int bs = 256;
  prim_to_cons_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(W, U, n, 1.0 / (gamma - 1.0));
  return cudaGetLastError();
}

cudaError_t launch_cfl(const double* U, const Lay& lay, const unsigned char* tag, double gamma, double dx,
                       double dy, unsigned long long* red, cudaStream_t s) {
  cfl_init_kernel<<<1, 1, 0, s>>>(red);
  const long long n = (long long)lay.nx * lay.ny;
  const int bs = 256;
  long long blocks = (n + bs - 1) / bs;
  if (blocks > 152 * 8) blocks = 152 * 8;
  cfl_kernel<<<(unsigned)blocks, bs, 0, s>>>(U, n, lay.nx, lay.ny > 1 ? 1 : 0, tag, gamma, dx, dy, red);
  return cudaGetLastError();
}

}  // namespace js
