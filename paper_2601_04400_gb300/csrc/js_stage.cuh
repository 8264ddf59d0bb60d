// Fused stage of the FP64 finite-volume step on one 2D tile (arXiv 2601.04400, Sec. 2):
// conserved tile + 3-cell halo -> primitives in shared memory -> x sweep (WENO5, HLLC,
// viscous flux) into a global accumulator (it stays in L2; keeping it out of shared memory
// lets more blocks share an SM's FP64 pipe) -> y sweep, divergence, artificial viscosity and
// the SSP-RK3 stage combination.  Used by the per-grid stage kernel and by the persistent
// batched kernel.
#pragma once
#include <type_traits>

#include "js_device.cuh"
#include "js_internal.h"

namespace js {

// =======================================================================================
// line sweep: WENO5 -> HLLC (+ viscous) -> flux differences, on primitives in shared memory
// =======================================================================================
// sq: shared planes rho, u, v, p (and T when VISC), plane stride ps; `base` = index of the
// first output cell of the segment, `st` = stride along the line, `ts` = stride across it.
// emit(k, dF) receives F_{k+1/2} - F_{k-1/2} (conserved order) for output cells k = 0..L-1.
// keep(k, c, sv), when given, receives the WENO5 internals of variable c at cell k for
// k = -1 (left-biased side only), 0..L-1 (both sides) and L (right-biased side only).
// face(k, ql, qr), when given, receives the two WENO5 states (before any positivity fallback)
// of face k - 1/2 for k = 0..L.
struct NoKeep {
  __device__ __forceinline__ void operator()(int, int, const double*) const {}
};
struct NoFace {
  __device__ __forceinline__ void operator()(int, const double*, const double*) const {}
};

template <int DIR, bool VISC, bool HAS_T, int L, class Emit, class Keep = NoKeep, class Face = NoFace>
__device__ __forceinline__ void sweep_line(const double* __restrict__ sq, int ps, int base, int st, int ts,
                                           const Gas& g, const ViscC& vc, Emit&& emit, Keep keep = Keep{},
                                           Face face = Face{}) {
  constexpr bool SV = !std::is_same<Keep, NoKeep>::value;
  constexpr bool FI = !std::is_same<Face, NoFace>::value;
  constexpr int PN = (DIR == 0) ? 1 : 2;  // plane of the face-normal velocity
  constexpr int PT = (DIR == 0) ? 2 : 1;  // plane of the tangential velocity
  Win w[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double* q = sq + c * ps;
    w[c].init(q[base - 3 * st], q[base - 2 * st], q[base - st], q[base]);
  }
  double prevL[4], prevF[4];
  {
    // cell -1 of the segment: only its right-face (left-biased) state is needed
    double Rf[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double sv[SV ? 7 : 1];
      w[c].template step<true, false, SV>(sq[c * ps + base - st + 2 * st], prevL[c], Rf[c], sv);
      if (SV) keep(-1, c, sv);
    }
  }
#pragma unroll 1
  for (int k = 0; k <= L; ++k) {
    const int cell = base + k * st;
    double Lf[4], Rf[4];
    if (k < L) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        double sv[SV ? 7 : 1];
        w[c].template step<true, true, SV>(sq[c * ps + cell + 2 * st], Lf[c], Rf[c], sv);
        if (SV) keep(k, c, sv);
      }
    } else {
      // cell L (first cell of the next segment): only its left-face state is needed
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        double sv[SV ? 7 : 1];
        w[c].template step<false, true, SV>(sq[c * ps + cell + 2 * st], Lf[c], Rf[c], sv);
        if (SV) keep(L, c, sv);
        Lf[c] = 0.0;  // unused
      }
    }
    {
      // face k - 1/2 between cells k-1 (left state prevL) and k (right state Rf)
      double ql[4], qr[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) { ql[c] = prevL[c]; qr[c] = Rf[c]; }
      if (FI) face(k, ql, qr);
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
// dG: raw y-flux differences (scaled here by cy), or already scaled when YSCALED
template <bool RHS, bool YSCALED = false>
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
      double v = YSCALED ? (us - acc[c]) - dG[c] : fma(-a.cy, dG[c], us - acc[c]);
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
  static constexpr size_t SMEM = sizeof(double) * (size_t)NPL * PS;
};

// one tile (bx, by) of one stage; smem holds Stage2D::SMEM bytes; all NT threads take part
template <int TX, int TY, int LX, int LY, bool VISC, bool RHS>
__device__ __forceinline__ void stage_tile(const StageArgs& a, int bx, int by, double* smem) {
  using S = Stage2D<TX, TY, LX, LY, VISC, RHS>;
  double* sq = smem;
  const long long ncell = (long long)a.lay.nx * a.lay.ny;
  const Gas g{a.gamma, a.gm1, a.g1};
  const int tx0 = bx * TX, ty0 = by * TY;  // interior origin of the tile
  load_tile<TX, TY, S::NPL, S::NT>(a, sq, S::PS, S::SP, tx0, ty0, g);
  __syncthreads();
  // x sweep: one thread per (row, segment)
  for (int it = threadIdx.x; it < S::NX_ITEMS; it += S::NT) {
    const int ty = it % TY, xs = (it / TY) * LX;
    const int base = (ty + 3) * S::SP + xs + 3;
    const int gj = ty0 + ty;
    sweep_line<0, VISC, true, LX>(sq, S::PS, base, 1, S::SP, g, a.vx, [&](int k, const double dF[4]) {
      const int gi = tx0 + xs + k;
      if (gi < a.lay.nx && gj < a.lay.ny) {
        const long long o = (long long)gj * a.lay.nx + gi;
#pragma unroll
        for (int c = 0; c < 4; ++c) a.acc[c * ncell + o] = __dmul_rn(a.cx, dF[c]);
      }
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
        const long long o = (long long)gj * a.lay.nx + gi;
#pragma unroll
        for (int c = 0; c < 4; ++c) ax[c] = a.acc[c * ncell + o];
        double ay[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) ay[c] = __dmul_rn(a.cy, dG[c]);  // rounded as when stored
        const int sc = (ty + 3) * S::SP + tx + 3;
        finish_cell<RHS, true>(a, gi, gj, ax, ay, sq[sc], sq[3 * S::PS + sc]);
      }
    });
  }
}


// ---------------------------------------------------------------------------------------
// Concurrent-sweep tile: the x sweep (first NX_ITEMS threads) and the y sweep (next
// NY_ITEMS threads, warp-aligned) run at the same time on the shared primitive tile and
// write their scaled flux differences to two global accumulators (L2-resident); after a
// barrier every thread combines cells of the tile.  Twice the warps per block at the same
// shared memory: more warps hide the FP64 pipe's latency.
// ---------------------------------------------------------------------------------------
template <int TX, int TY, int LX, int LY, bool VISC, bool TMA = false>
struct Stage2DC {
  static constexpr int NPL = VISC ? 5 : 4;
  static constexpr int SP = TMA ? TX + 6 : TX + 7;  // TMA writes dense box rows
  static constexpr int PS = (TY + 6) * SP;
  static constexpr int NX_ITEMS = TY * (TX / LX);
  static constexpr int NY_ITEMS = TX * (TY / LY);
  static_assert(NX_ITEMS % 32 == 0 && NY_ITEMS % 32 == 0, "sweep roles must be whole warps");
  static constexpr int NT = NX_ITEMS + NY_ITEMS;
  static constexpr size_t SMEM = sizeof(double) * (size_t)NPL * PS;
};

// ---------------------------------------------------------------------------------------
// TMA staging: one cp.async.bulk.tensor brings the conserved (TX+6) x (TY+6) x 4 box of the
// padded state into shared memory ([plane][row][col], row pitch TX+6); an mbarrier tracks
// completion.  Waits are bounded: on timeout the block records JS_ERR_TIMEOUT, drains its copy
// (bounded again) and skips the tile.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// wait for the mbarrier phase `parity` to complete, for at most `budget` SM clock cycles
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long budget) {
  const long long t0 = clock64();
  while (true) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > budget) return false;
  }
}
__device__ __forceinline__ void tma_box3d(void* dst, const void* map, int x, int y, int z,
                                          unsigned long long* bar, unsigned bytes) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Stage the tile with TMA and convert it to primitives in place (T in plane 4 when VISC).
// Returns false when the copy did not complete in time (the tile must be skipped).
template <int TX, int TY, int NPL, int NT>
__device__ __forceinline__ bool load_tile_tma(const StageArgs& a, const void* tmap, double* sq, int ps, int ox,
                                              int oy, const Gas& g, unsigned long long* bar, unsigned& phase) {
  constexpr int CW = TX + 6, CH = TY + 6;
  constexpr unsigned BYTES = 4u * CW * CH * sizeof(double);
  static_assert(CW * CH * sizeof(double) % 16 == 0 && CW * sizeof(double) % 16 == 0, "TMA box rows");
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    // the box origin is the tile origin in padded coordinates: x = ox is a multiple of 32
    tma_box3d(sq, tmap, ox, oy, 0, bar, BYTES);
    constexpr long long kBudget = 2000000000LL;  // about one second of SM clock
    bool ok = mbar_wait(bar, phase, kBudget);
    if (!ok) {
      atomicOr(a.err, ERR_TIMEOUT_BIT);
      mbar_wait(bar, phase, kBudget);  // drain the copy in flight before the block moves on
    }
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  phase ^= 1u;
  if (!s_ok) return false;
  for (int e = threadIdx.x; e < CW * CH; e += NT) {
    const double r = sq[e], mx = sq[ps + e], my = sq[2 * ps + e], E = sq[3 * ps + e];
    double u, v, p, T;
    cons_to_prim(r, mx, my, E, g, u, v, p, T);
    sq[ps + e] = u;
    sq[2 * ps + e] = v;
    sq[3 * ps + e] = p;
    if (NPL == 5) sq[4 * ps + e] = T;
  }
  return true;
}

// Store the WENO5 internals of variable c at cell `k` of line `line` (DIR 0: row, stored
// transposed; DIR 1: column, padded layout), for the cells -1 .. n the reverse pass reads
// (n = cells along the line).  `part` is -1 / 0 / +1 for a cell whose left-biased side only /
// both sides / right-biased side only were formed.  Cell n keeps only its right-biased side,
// so that every writer of a cell stores the same values.
template <int DIR>
__device__ __forceinline__ void keep_internals(const StageArgs& a, int k, int line, int c, const double* sv,
                                               int part) {
  const int n = (DIR == 0) ? a.lay.nx : a.lay.ny;
  const bool store = (part < 0) ? (k == -1) : (part > 0) ? (k == n) : (k >= 0 && k <= n);
  if (!store) return;
  const long long si = (DIR == 0) ? (long long)(k + 3) * a.tpitch + (line + a.lay.gy) : a.lay.idx(line, k);
  double* dst = a.wsave + (long long)(DIR * 28 + c * 7) * a.splane + si;
  const bool left = k < n;
#pragma unroll
  for (int m = 0; m < 7; ++m) dst[m * a.splane] = (m == 3 || m == 4) && !left ? 0.0 : sv[m];
}

// face image of the neural flux (IMG: a.img, FP32 [4][ny][nx+1] for x faces then [4][nx][ny+1]
// for y faces): face f of a line is written by the segment that holds cell f, the line's last
// face by the segment that ends there
template <int DIR>
__device__ __forceinline__ void put_image(const StageArgs& a, int line, int f, const double* ql, const double* qr) {
  const int nx = a.lay.nx, ny = a.lay.ny;
  const long long pix0 = (long long)ny * (nx + 1);
  const long long pix = (DIR == 0) ? pix0 : (long long)nx * (ny + 1);
  float* X = a.img + (DIR == 0 ? 0LL : 4 * pix0) + (long long)line * ((DIR == 0 ? nx : ny) + 1) + f;
  float m[4];
  face_image<float>(ql, qr, DIR == 0 ? 1 : 2, DIR == 0 ? 2 : 1, a.img_g1, a.img_mean, a.img_isd, m);
#pragma unroll
  for (int k = 0; k < 4; ++k) X[k * pix] = m[k];
}

template <int TX, int TY, int LX, int LY, bool VISC, bool RHS, bool TMA = false, bool SAVE = false, bool IMG = false>
__device__ __forceinline__ void stage_tile_c(const StageArgs& a, int bx, int by, double* smem,
                                             const void* tmap = nullptr, unsigned long long* bar = nullptr,
                                             unsigned* phase = nullptr) {
  using S = Stage2DC<TX, TY, LX, LY, VISC, TMA>;
  double* sq = smem;
  const long long ncell = (long long)a.lay.nx * a.lay.ny;
  const Gas g{a.gamma, a.gm1, a.g1};
  const int tx0 = bx * TX, ty0 = by * TY;
  if (TMA) {
    if (!load_tile_tma<TX, TY, S::NPL, S::NT>(a, tmap, sq, S::PS, tx0, ty0, g, bar, *phase)) return;
  } else {
    load_tile<TX, TY, S::NPL, S::NT>(a, sq, S::PS, S::SP, tx0, ty0, g);
  }
  __syncthreads();
  if (threadIdx.x < S::NX_ITEMS) {
    const int it = threadIdx.x;
    const int ty = it % TY, xs = (it / TY) * LX;
    const int gj = ty0 + ty;
    auto emit = [&](int k, const double dF[4]) {
      const int gi = tx0 + xs + k;
      if (gi < a.lay.nx && gj < a.lay.ny) {
        const long long o = (long long)gj * a.lay.nx + gi;
#pragma unroll
        for (int c = 0; c < 4; ++c) a.acc[c * ncell + o] = __dmul_rn(a.cx, dF[c]);
      }
    };
    if constexpr (SAVE) {
      sweep_line<0, VISC, true, LX>(sq, S::PS, (ty + 3) * S::SP + xs + 3, 1, S::SP, g, a.vx, emit,
                                    [&](int k, int c, const double* sv) {
        if (gj < a.lay.ny) keep_internals<0>(a, tx0 + xs + k, gj, c, sv, k < 0 ? -1 : (k == LX ? 1 : 0));
      });
    } else if constexpr (IMG) {
      sweep_line<0, VISC, true, LX>(sq, S::PS, (ty + 3) * S::SP + xs + 3, 1, S::SP, g, a.vx, emit, NoKeep{},
                                    [&](int k, const double* ql, const double* qr) {
        const int f = tx0 + xs + k;
        if (gj < a.lay.ny && f <= a.lay.nx && (k < LX || f == a.lay.nx)) put_image<0>(a, gj, f, ql, qr);
      });
    } else {
      sweep_line<0, VISC, true, LX>(sq, S::PS, (ty + 3) * S::SP + xs + 3, 1, S::SP, g, a.vx, emit);
    }
  } else {
    const int it = threadIdx.x - S::NX_ITEMS;
    const int tx = it % TX, ys = (it / TX) * LY;
    const int gi = tx0 + tx;
    auto emit = [&](int k, const double dG[4]) {
      const int gj = ty0 + ys + k;
      if (gi < a.lay.nx && gj < a.lay.ny) {
        const long long o = (long long)gj * a.lay.nx + gi;
#pragma unroll
        for (int c = 0; c < 4; ++c) a.acc2[c * ncell + o] = __dmul_rn(a.cy, dG[c]);
      }
    };
    if constexpr (SAVE) {
      sweep_line<1, VISC, true, LY>(sq, S::PS, (ys + 3) * S::SP + tx + 3, S::SP, 1, g, a.vy, emit,
                                    [&](int k, int c, const double* sv) {
        if (gi < a.lay.nx) keep_internals<1>(a, ty0 + ys + k, gi, c, sv, k < 0 ? -1 : (k == LY ? 1 : 0));
      });
    } else if constexpr (IMG) {
      sweep_line<1, VISC, true, LY>(sq, S::PS, (ys + 3) * S::SP + tx + 3, S::SP, 1, g, a.vy, emit, NoKeep{},
                                    [&](int k, const double* ql, const double* qr) {
        const int f = ty0 + ys + k;
        if (gi < a.lay.nx && f <= a.lay.ny && (k < LY || f == a.lay.ny)) put_image<1>(a, gi, f, ql, qr);
      });
    } else {
      sweep_line<1, VISC, true, LY>(sq, S::PS, (ys + 3) * S::SP + tx + 3, S::SP, 1, g, a.vy, emit);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TX * TY; e += S::NT) {
    const int tx = e % TX, ty = e / TX;
    const int gi = tx0 + tx, gj = ty0 + ty;
    if (gi >= a.lay.nx || gj >= a.lay.ny) continue;
    const long long o = (long long)gj * a.lay.nx + gi;
    double ax[4], ay[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      ax[c] = a.acc[c * ncell + o];
      ay[c] = a.acc2[c * ncell + o];
    }
    const int sc = (ty + 3) * S::SP + tx + 3;
    finish_cell<RHS, true>(a, gi, gj, ax, ay, sq[sc], sq[3 * S::PS + sc]);
  }
}

}  // namespace js
