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
#include "js_adjoint_body.cuh"
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
  const double* dt_in;        // [n_steps][count] given step sizes (no CFL reduction), or nullptr
  double* const* ustate;      // [count] states advanced instead of the registered ones, or nullptr
  double* const* save;        // [n_steps][count] states after each step, or nullptr
  double* const* save1;       // [n_steps][count] stage states U1, U2 of each step (after stages
  double* const* save2;       //   1 and 2), or nullptr
  const int* order;           // schedule: queue position -> tile number (ntiles), or nullptr
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
__device__ bool grid_sync_on(unsigned* bar, int* err, int extra_arrivals, long long budget) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned target = gridDim.x + (unsigned)extra_arrivals;
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == target) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*(volatile int*)err & ERR_TIMEOUT_BIT) { ok = 0; break; }
        if (clock64() - t0 > budget) {
          atomicOr(err, ERR_TIMEOUT_BIT);
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
__device__ __forceinline__ bool grid_sync(const BatchArgs& b) {
  return grid_sync_on(b.bar, b.err, b.extra_arrivals, b.budget);
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
    const int q = b.order ? b.order[it] : it;
    const int k = find_inst(b.tile0, b.count, q);
    const InstDesc& d = b.inst[k];
    const double* Uk = b.ustate ? b.ustate[k] : d.U;
    const int t = q - b.tile0[k];
    const int i0 = (t % d.ntx) * BTX, j0 = (t / d.ntx) * BTY;
    const long long n = (long long)d.lay.nx * d.lay.ny;
    for (int e = tid; e < BTX * BTY; e += BNT) {
      const int i = i0 + (e % BTX), j = j0 + (e / BTX);
      if (i >= d.lay.nx || j >= d.lay.ny) continue;
      const long long o = (long long)j * d.lay.nx + i, p = d.lay.idx(i, j);
#pragma unroll
      for (int c = 0; c < 4; ++c) d.N[c * d.lay.plane + p] = Uk[c * n + o];
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
    // ---- CFL reduction over fluid cells, per instance (skipped with given step sizes)
    for (int it = blockIdx.x; it < (b.dt_in ? 0 : ntiles); it += gridDim.x) {
      const int q = b.order ? b.order[it] : it;
    const int k = find_inst(b.tile0, b.count, q);
      const InstDesc& d = b.inst[k];
      const int t = q - b.tile0[k];
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
    if (!b.dt_in && !grid_sync(b)) return;
    if (blockIdx.x == 0) {
      // the other parity was last read in the previous step: reset it for the next one
      unsigned long long* nxt = b.red + 2 * (long long)b.count * (par ^ 1);
      for (int k = tid; k < b.count; k += BNT) {
        nxt[2 * k] = 0ULL;
        nxt[2 * k + 1] = 0x7ff0000000000000ULL;
        const double dtk = b.dt_in ? b.dt_in[(long long)step * b.count + k] : inst_dt(b.inst[k], red + 2 * k, b.cfl);
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
        const int q = b.order ? b.order[it] : it;
    const int k = find_inst(b.tile0, b.count, q);
        const InstDesc& d = b.inst[k];
        const int t = q - b.tile0[k];
        const double dt = b.dt_in ? b.dt_in[(long long)step * b.count + k] : inst_dt(d, red + 2 * k, b.cfl);
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
    if (b.save || b.save1) {
      // the state after this step (ghost cells included), before the next step refills them,
      // and the stage states A, B of this step (their ghost cells were refilled from fluid
      // cells, which a reverse pass that fills them again reproduces)
      for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
        const int q = b.order ? b.order[it] : it;
        const int k = find_inst(b.tile0, b.count, q);
        const InstDesc& d = b.inst[k];
        const long long row = (long long)step * b.count + k;
        double* S = b.save ? b.save[row] : nullptr;
        double* S1 = b.save1 ? b.save1[row] : nullptr;
        double* S2 = b.save1 ? b.save2[row] : nullptr;
        const int t = q - b.tile0[k];
        const int i0 = (t % d.ntx) * BTX, j0 = (t / d.ntx) * BTY;
        const long long n = (long long)d.lay.nx * d.lay.ny;
        for (int e = tid; e < BTX * BTY; e += BNT) {
          const int i = i0 + (e % BTX), j = j0 + (e / BTX);
          if (i >= d.lay.nx || j >= d.lay.ny) continue;
          const long long o = (long long)j * d.lay.nx + i, p = d.lay.idx(i, j);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (S) S[c * n + o] = d.N[c * d.lay.plane + p];
            if (S1) {
              S1[c * n + o] = d.A[c * d.lay.plane + p];
              S2[c * n + o] = d.B[c * d.lay.plane + p];
            }
          }
        }
      }
      if (!grid_sync(b)) return;
    }
  }
  // ---- unpack
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int q = b.order ? b.order[it] : it;
    const int k = find_inst(b.tile0, b.count, q);
    const InstDesc& d = b.inst[k];
    double* Uk = b.ustate ? b.ustate[k] : d.U;
    const int t = q - b.tile0[k];
    const int i0 = (t % d.ntx) * BTX, j0 = (t / d.ntx) * BTY;
    const long long n = (long long)d.lay.nx * d.lay.ny;
    for (int e = tid; e < BTX * BTY; e += BNT) {
      const int i = i0 + (e % BTX), j = j0 + (e / BTX);
      if (i >= d.lay.nx || j >= d.lay.ny) continue;
      const long long o = (long long)j * d.lay.nx + i, p = d.lay.idx(i, j);
#pragma unroll
      for (int c = 0; c < 4; ++c) Uk[c * n + o] = d.N[c * d.lay.plane + p];
    }
  }
}

// =======================================================================================
// persistent batched reverse: one launch reverses one SSP-RK3 step of every instance (the
// gradient chain rule of Sec. 2 per instance) -- the per-grid js_step_vjp's phases, each run
// over the work items of all instances, separated by grid barriers:
//   pack U_n, lambda_{n+1}; zero Uacc
//   forward recompute, stages 0 and 1: IB fill | halo fill | stage tiles (storing their WENO5
//   internals); IB and halo fill of the stage-2 input
//   reverse, stages 2, 1, 0: seed + primitives (+ the previous stage's parameter-gradient
//   reduction) | pass 1 | pass 2 | primitive reverse | transposed y halos | transposed x halos |
//   inflow gradient + transposed IB ghosts | transposed IB sources
//   unpack lambda_n (+ the last reduction)
// The device bodies are those of the per-grid launches (js_adjoint_body.cuh, js_stage.cuh,
// js_fill.cuh) on the same elements in the same order, so lambda_n equals js_step_vjp's bit for
// bit; the parameter gradient is reduced in a fixed order too (its partial sums are grouped
// by 128-thread blocks here, so it agrees with js_step_vjp's to rounding).
// Work items of every instance are padded to whole warps, so a warp never spans two instances.
// =======================================================================================
enum RevKind { RK_PLANE = 0, RK_USER4, RK_GHOST, RK_HALO, RK_P1RE, RK_P1SV, RK_P2, RK_BCTY, RK_BCTX, RK_SRC, RK_N };

struct RevCall {
  const double* const* Un;    // [count] user states U_n
  const double* const* lam1;  // [count] lambda_{n+1}
  double* const* lam0;        // [count] lambda_n (may alias lam1)
  double* const* pbar;        // [count] parameter gradients (entries may be null) or null
  const double* dt;           // [count] step sizes
  // [count] the step's stage states U1, U2 (user layout, e.g. kept by a rollout's forward), or
  // null: the reverse recomputes them (storing their WENO5 internals for pass 1 of stages 1, 0)
  const double* const* U1;
  const double* const* U2;
};

struct BatchRevArgs {
  const InstDesc* inst;
  const InstRev* rev;
  int count;
  const long long* pre;       // [RK_N][count + 1] prefix sums of the padded item counts
  const int* tile0;
  RevCall call;
  unsigned* bar;
  int* err;
  long long budget;
};

// every item g of kind K over all instances: f(k, local) with k = -1 past the end (whole
// warps, so warp-collective bodies see all 32 lanes)
template <class F>
__device__ __forceinline__ void rev_items(const BatchRevArgs& b, int kind, F f) {
  const long long* pre = b.pre + (long long)kind * (b.count + 1);
  const long long total = pre[b.count];
  for (long long base = (long long)blockIdx.x * BNT; base < total; base += (long long)gridDim.x * BNT) {
    const long long g = base + threadIdx.x;
    int k = -1;
    long long local = 0;
    if (g < total) {
      k = find_inst64(pre, b.count, g);
      local = g - pre[k];
    }
    f(k, local);
  }
}

// pass 1 of reverse stage s reads the WENO5 internals stored by the forward recompute (stages
// 1, 0 when the reverse recomputes the stage states) or recomputes them
__device__ __forceinline__ bool rev_saved(const RevCall& call, int s) { return s < 2 && call.U1 == nullptr; }

__device__ __forceinline__ AdjArgs rev_adj(const InstRev& r, const InstDesc& d, int s, const RevCall& call, int k,
                                           double* dst, bool with_pbar) {
  AdjArgs a = r.a;
  a.X = (s == 0) ? d.N : ((s == 1) ? d.A : d.B);
  a.Ub = dst;
  a.pbar = with_pbar && call.pbar ? call.pbar[k] : nullptr;
  a.pp = a.pbar ? r.ppart : nullptr;
  if (rev_saved(call, s)) {
    a.wsave = r.wfwd + (long long)56 * s * r.a.splane;
    a.weno_saved = 1;
  } else {
    a.wsave = r.wsave_own;
    a.weno_saved = 0;
  }
  return a;
}

// the parameter-gradient slot ranges of reverse stage s of one instance, summed into its pbar
__device__ __forceinline__ void rev_reduce(const InstRev& r, bool saved, double* pbar) {
  const long long off[4] = {0, r.off_prim, r.off_g, r.off_s};
  const long long cnt[4] = {saved ? r.w1_sv : r.w1_re, r.w_prim, r.w_g, r.w_s};
  adj_pbar_reduce_block(r.ppart, off, cnt, 4, pbar);
}

// The phases of one batched reverse step.  Each runs over the work items of all instances with
// grid-stride loops, so it is correct for any grid; the persistent kernel runs them in order
// with grid barriers between them, the split launch as one kernel per phase (each with its own
// register allocation and occupancy).
enum RevPhase {
  RP_PACK = 0,      // pack U_n, lambda_{n+1} (and given stage states); Uacc = 0
  RP_GHOST,         // IB fill of stage input s
  RP_HALO,          // halo fill of stage input s
  RP_STAGE,         // forward recompute of stage s (0, 1), storing its WENO5 internals
  RP_SEED,          // reverse stage s: seed + primitives (+ reduction of stage s+1's partials)
  RP_PASS1,         // pass 1 (x lines, then y lines)
  RP_PASS2,         // pass 2
  RP_PRIMVJP,       // primitive reverse
  RP_BCTY,          // transposed y halos
  RP_BCTX,          // transposed x halos
  RP_INFLOW_GHOST,  // inflow-state gradient + transposed IB ghosts
  RP_SRC,           // transposed IB sources
  RP_UNPACK,        // lambda_n = P1 + Uacc; the last stage's parameter gradient
  RP_N
};

// pass 1 of reverse stage s (x lines, then y lines from the 32-aligned offset xpad).  SVM 0:
// WENO5 internals stored or recomputed as the call decides (rev_saved), 1: stored, 2:
// recomputed; VM 0: every instance, 1: the viscous instances only, 2: the inviscid ones only --
// the split launch fixes both on the host, so that each kernel holds only the pass-1 variant it
// runs (and its register allocation is that variant's).
template <int SVM, int VM = 0>
__device__ __forceinline__ void rev_pass1(const BatchRevArgs& b, int s) {
  const RevCall& call = b.call;
  const bool even = (s == 2) || (s == 0);
  const bool sv = (SVM == 0) ? rev_saved(call, s) : (SVM == 1);
  rev_items(b, sv ? RK_P1SV : RK_P1RE, [&](int k, long long item) {
    if (k < 0) return;  // whole warps past the end: nothing to do, no partials
    const InstDesc& d = b.inst[k];
    if ((VM == 1 && !d.visc) || (VM == 2 && d.visc)) return;  // the other kernel's instance
    const InstRev& r = b.rev[k];
    const AdjArgs a = rev_adj(r, d, s, call, k, even ? r.P1 : r.P0, true);
    const long long xpad = sv ? r.xpad_sv : r.xpad_re;
    const int seg = sv ? r.seg1_sv : r.seg1_re;
    const int dir = item < xpad ? 0 : 1;
    const long long it = dir == 0 ? item : item - xpad;
    const long long wofs = dir == 0 ? 0 : (xpad >> 5);
    const bool visc = (VM == 0) ? d.visc : (VM == 1);
    if (SVM != 2 && sv) {
      if (VM != 2 && visc) {
        if (dir == 0) pass1_body<0, true, true, true>(a, seg, it, wofs);
        else pass1_body<1, true, true, true>(a, seg, it, wofs);
      } else if (VM != 1) {
        if (dir == 0) pass1_body<0, false, false, true>(a, seg, it, wofs);
        else pass1_body<1, false, false, true>(a, seg, it, wofs);
      }
    } else if (SVM != 1) {
      if (VM != 2 && visc) {
        if (dir == 0) pass1_body<0, true, true, false>(a, seg, it, wofs);
        else pass1_body<1, true, true, false>(a, seg, it, wofs);
      } else if (VM != 1) {
        if (dir == 0) pass1_body<0, false, false, false>(a, seg, it, wofs);
        else pass1_body<1, false, false, false>(a, seg, it, wofs);
      }
    }
  });
}

template <int PH>
__device__ __forceinline__ void rev_phase(const BatchRevArgs& b, int s, double* smem) {
  const RevCall& call = b.call;
  const bool even = (s == 2) || (s == 0);  // reverse stages 2 and 0 read P0, write P1
  if constexpr (PH == RP_PACK) {
    rev_items(b, RK_USER4, [&](int k, long long t) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      const long long n = (long long)d.lay.nx * d.lay.ny;
      if (t >= 4 * n) return;
      const int c = (int)(t / n);
      const long long o = t % n;
      const long long p = c * d.lay.plane + d.lay.idx((int)(o % d.lay.nx), (int)(o / d.lay.nx));
      d.N[p] = call.Un[k][t];
      b.rev[k].P0[p] = call.lam1[k][t];
      if (call.U1) {
        d.A[p] = call.U1[k][t];
        d.B[p] = call.U2[k][t];
      }
    });
    rev_items(b, RK_PLANE, [&](int k, long long t) {
      if (k < 0 || t >= b.inst[k].lay.plane) return;
      const InstDesc& d = b.inst[k];
#pragma unroll
      for (int c = 0; c < 4; ++c) b.rev[k].Uacc[c * d.lay.plane + t] = 0.0;
    });
  } else if constexpr (PH == RP_GHOST) {
    rev_items(b, RK_GHOST, [&](int k, long long g) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      if (g >= d.ib.n) return;
      double* X = (s == 0) ? d.N : ((s == 1) ? d.A : d.B);
      ib_fill_one(X, d.lay, d.ib, d.gamma, d.wall, (int)g);
    });
  } else if constexpr (PH == RP_HALO) {
    rev_items(b, RK_HALO, [&](int k, long long h) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      if (h >= halo_count(d.lay)) return;
      double* X = (s == 0) ? d.N : ((s == 1) ? d.A : d.B);
      bc_fill_one(X, d.lay, d.bc, h);
    });
  } else if constexpr (PH == RP_STAGE) {
    for (int it = blockIdx.x; it < b.tile0[b.count]; it += gridDim.x) {
      const int k = find_inst(b.tile0, b.count, it);
      const InstDesc& d = b.inst[k];
      const InstRev& r = b.rev[k];
      const int t = it - b.tile0[k];
      const double dt = call.dt[k];
      StageArgs a;
      a.Uin = (s == 0) ? d.N : d.A;
      a.Un = d.N;
      a.Uout = (s == 0) ? d.A : d.B;
      a.tag = d.tag;
      a.acc = d.acc;
      a.acc2 = d.acc2;
      a.err = b.err;
      a.lay = d.lay;
      a.gamma = d.gamma;
      a.gm1 = d.gamma - 1.0;
      a.g1 = 1.0 / (d.gamma - 1.0);
      a.cx = dt / d.dx;
      a.cy = dt / d.dy;
      a.rk_a = (s == 0) ? 0.0 : 0.75;
      a.rk_b = (s == 0) ? 1.0 : 0.25;
      a.avx = dt * d.nu / (d.dx * d.dx);
      a.avy = dt * d.nu / (d.dy * d.dy);
      a.vx = d.vx;
      a.vy = d.vy;
      a.use_un = (s > 0) ? 1 : 0;
      a.has_av = d.has_av;
      a.wsave = r.wfwd + (long long)56 * s * r.a.splane;
      a.splane = r.a.splane;
      a.tpitch = r.a.tpitch;
      a.dtc = nullptr;
      if (d.visc) stage_tile_c<BTX, BTY, BLX, BLY, true, false, false, true>(a, t % d.ntx, t / d.ntx, smem);
      else stage_tile_c<BTX, BTY, BLX, BLY, false, false, false, true>(a, t % d.ntx, t / d.ntx, smem);
      __syncthreads();  // the next tile reuses shared memory
    }
  } else if constexpr (PH == RP_SEED) {
    const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
    const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
    // seed + primitives; the parameter-gradient partials of stage s+1 are reduced meanwhile
    rev_items(b, RK_PLANE, [&](int k, long long t) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      const InstRev& r = b.rev[k];
      if (t >= d.lay.plane) return;
      const AdjArgs a = rev_adj(r, d, s, call, k, even ? r.P1 : r.P0, false);
      adj_seed_one(a, t, even ? r.P0 : r.P1, r.Uacc, ra[s], rb[s], call.dt[k], 0);
      adj_prims_one(a, t);
    });
    if (s < 2 && call.pbar)
      for (int k = blockIdx.x; k < b.count; k += gridDim.x)
        if (call.pbar[k]) rev_reduce(b.rev[k], rev_saved(call, s + 1), call.pbar[k]);
  } else if constexpr (PH == RP_PASS1) {
    rev_pass1<0>(b, s);
  } else if constexpr (PH == RP_PASS2) {
    rev_items(b, RK_P2, [&](int k, long long item) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      const InstRev& r = b.rev[k];
      const AdjArgs a = rev_adj(r, d, s, call, k, even ? r.P1 : r.P0, false);
      if (item < r.xpad_p2) pass2_body<0>(a, r.seg2, item);
      else pass2_body<1>(a, r.seg2, item - r.xpad_p2);
    });
  } else if constexpr (PH == RP_PRIMVJP) {
    rev_items(b, RK_PLANE, [&](int k, long long t) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      const InstRev& r = b.rev[k];
      const AdjArgs a = rev_adj(r, d, s, call, k, even ? r.P1 : r.P0, true);
      double gb = 0.0, nb = 0.0;
      if (d.visc) adj_primvjp_one<true>(a, t, r.seg2, gb, nb);
      else adj_primvjp_one<false>(a, t, r.seg2, gb, nb);
      warp_partials(a.pp, r.off_prim + (t >> 5), gb, 0.0, 0.0, nb);
    });
  } else if constexpr (PH == RP_BCTY || PH == RP_BCTX) {
    rev_items(b, PH == RP_BCTY ? RK_BCTY : RK_BCTX, [&](int k, long long t) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      const InstRev& r = b.rev[k];
      const AdjArgs a = rev_adj(r, d, s, call, k, even ? r.P1 : r.P0, false);
      adj_bcT_one(a, d.bc, PH == RP_BCTY ? 1 : 0, r.inflow_part, r.tmax, t);
    });
  } else if constexpr (PH == RP_INFLOW_GHOST) {
    // inflow-state gradient (one block per instance) and the transposed IB ghosts
    for (int k = blockIdx.x; k < b.count; k += gridDim.x) {
      const InstDesc& d = b.inst[k];
      const InstRev& r = b.rev[k];
      const AdjArgs a = rev_adj(r, d, s, call, k, even ? r.P1 : r.P0, true);
      adj_inflow_block(a, d.bc, r.inflow_part, r.tmax, r.inflow_prim);
    }
    rev_items(b, RK_GHOST, [&](int k, long long g) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      const InstRev& r = b.rev[k];
      const AdjArgs a = rev_adj(r, d, s, call, k, even ? r.P1 : r.P0, true);
      double gb = 0.0;
      adj_ib_ghost_one(a, d.ib, d.wall, r.qIb, (int)g, gb);
      warp_partials(a.pp, r.off_g + (g >> 5), gb, 0.0, 0.0, 0.0);
    });
  } else if constexpr (PH == RP_SRC) {
    rev_items(b, RK_SRC, [&](int k, long long q) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      const InstRev& r = b.rev[k];
      const AdjArgs a = rev_adj(r, d, s, call, k, even ? r.P1 : r.P0, true);
      double gb = 0.0;
      adj_ib_src_one(a, r.ibt, r.qIb, (int)q, gb);
      warp_partials(a.pp, r.off_s + (q >> 5), gb, 0.0, 0.0, 0.0);
    });
  } else if constexpr (PH == RP_UNPACK) {
    // lambda_n = P1 + Uacc (stage 0 wrote P1); the last stage's parameter gradient
    rev_items(b, RK_USER4, [&](int k, long long t) {
      if (k < 0) return;
      const InstDesc& d = b.inst[k];
      if (t >= 4LL * d.lay.nx * d.lay.ny) return;
      adj_unpack_add_one(b.rev[k].P1, b.rev[k].Uacc, call.lam0[k], d.lay, t);
    });
    if (call.pbar)
      for (int k = blockIdx.x; k < b.count; k += gridDim.x)
        if (call.pbar[k]) rev_reduce(b.rev[k], rev_saved(call, 0), call.pbar[k]);
  }
}

__global__ void __launch_bounds__(BNT) batch_vjp_kernel(BatchRevArgs b) {
  extern __shared__ double smem[];
  rev_phase<RP_PACK>(b, 0, smem);
  if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
  // ---- forward recompute of the stage inputs X0 = N, X1 = A, X2 = B
  for (int s = 0; s < 3; ++s) {
    rev_phase<RP_GHOST>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    rev_phase<RP_HALO>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    if (s == 2) break;
    if (b.call.U1) continue;  // the stage states were given: only their ghosts and halos are filled
    rev_phase<RP_STAGE>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
  }
  // ---- reverse through the stages 2, 1, 0: P0 -> P1 -> P0 -> P1
  for (int s = 2; s >= 0; --s) {
    rev_phase<RP_SEED>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    rev_phase<RP_PASS1>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    rev_phase<RP_PASS2>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    rev_phase<RP_PRIMVJP>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    rev_phase<RP_BCTY>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    rev_phase<RP_BCTX>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    rev_phase<RP_INFLOW_GHOST>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
    rev_phase<RP_SRC>(b, s, smem);
    if (!grid_sync_on(b.bar, b.err, 0, b.budget)) return;
  }
  rev_phase<RP_UNPACK>(b, 0, smem);
}

// one phase of the reverse step as a kernel of its own (split launch); pass 1 has one kernel
// per WENO5-internals mode
template <int PH>
__global__ void __launch_bounds__(BNT) batch_vjp_phase_kernel(BatchRevArgs b, int s) {
  extern __shared__ double smem[];
  rev_phase<PH>(b, s, smem);
}
template <bool SV, bool VISC>
__global__ void __launch_bounds__(BNT) batch_vjp_pass1_kernel(BatchRevArgs b, int s) {
  rev_pass1<SV ? 1 : 2, VISC ? 1 : 2>(b, s);
}

// one launch copying every instance's state: dst[k][i] = src[k][i], i < pre[k+1] - pre[k]
__global__ void batch_copy_kernel(const double* const* src, double* const* dst, const long long* __restrict__ pre,
                                  int count) {
  const long long total = pre[count];
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int k = find_inst64(pre, count, g);
    const long long i = g - pre[k];
    dst[k][i] = src[k][i];
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
  int blocks = 0;          // persistent blocks of the forward launch (tuning: blocks per SM x SMs)
  int sms = 0, per_sm = 0;  // SMs and the forward kernel's resident blocks per SM
  int schedule = 0;        // tile order of the forward launch (js_batch_set_tuning)
  int* d_order = nullptr;  // its queue -> tile table (schedules 1 and 2)
  int ntiles = 0;
  long long cells = 0;
  bool states_set = false;
  // persistent reverse (prepared by the first reverse call)
  bool rev_ready = false;
  js::InstRev* d_rev = nullptr;
  long long* d_pre = nullptr;   // [RK_N][count + 1]
  int rev_blocks = 0;
  int rev_split = 0;                  // 1: one launch per phase (js_batch_set_reverse_launch)
  int rev_pblocks[js::RP_N] = {};     // grid of each phase kernel of the split launch
  int rev_p1blocks[2][2] = {};        // grid of its pass-1 kernels [stored internals][viscous]
  bool has_visc = false, has_inv = false;  // the batch holds viscous / inviscid instances
  void** d_tab = nullptr;       // call table of js_batch_step_vjp: U_n, lam_np1, lam_n, p_bar x count
  double* d_dt = nullptr;       // its step sizes
  // checkpointed rollout reverse (js_batch_rollout_vjp)
  int ro_steps = 0, ro_ckpt = 0, ro_nck = 0;
  std::vector<double*> ro_buf;  // per instance: nck checkpoints, ckpt segment states, 1 working state
  void** d_ro = nullptr;        // device tables: U, cp[nck], seg[ckpt], work, lam, p_bar (x count each)
  long long* d_spre = nullptr;  // prefix sums of the state sizes (4 nx ny)
  std::vector<void*> ro_lam, ro_pbar;  // the lam / p_bar pointers the tables hold
  const double* ro_fwd_log = nullptr;  // dt log of the rollout forward whose checkpoints are kept
  std::vector<void*> ro_U;             // the registered-state pointers table block 0 holds
};

// accessors of a context's internals (defined in js_host.cu)
void js_internal_desc(js_ctx* c, js::InstDesc* d);
int js_internal_rev_desc(js_ctx* c, js::InstRev* d);

namespace {
size_t batch_smem() { return js::BStageV::SMEM > js::BStageE::SMEM ? js::BStageV::SMEM : js::BStageE::SMEM; }
}  // namespace

namespace {

long long round32(long long n) { return (n + 31) / 32 * 32; }

// line items of pass 1 / pass 2 in one direction (dir 0: rows): lines x segments
long long line_items_of(const js::Lay& L, int dir, int extra, int seg) {
  const int nline = (dir == 0) ? L.ny : L.nx;
  const int ncell = (dir == 0) ? L.nx : L.ny;
  return (long long)nline * ((ncell + extra + seg - 1) / seg);
}

// the reverse descriptors and per-kind item prefix sums of the batch (first reverse call:
// allocates each instance's reverse workspace; call before any stream capture)
int rev_prepare(js_batch* b) {
  if (b->rev_ready) return JS_OK;
  const int n = b->count;
  std::vector<js::InstRev> rev(n);
  std::vector<long long> pre((size_t)js::RK_N * (n + 1), 0);
  for (int k = 0; k < n; ++k) {
    js::InstRev& r = rev[k];
    const int rc = js_internal_rev_desc(b->ctx[k], &r);
    if (rc) return rc;
    const js::InstDesc& d = b->desc[k];
    const js::Lay& L = d.lay;
    r.seg1_re = 16;  // the per-grid pass 1: recomputed WENO5 (2D), stored internals
    r.seg1_sv = 8;
    r.seg2 = js::ADJ_SEG2;
    const long long x_re = line_items_of(L, 0, 1, r.seg1_re), y_re = line_items_of(L, 1, 1, r.seg1_re);
    const long long x_sv = line_items_of(L, 0, 1, r.seg1_sv), y_sv = line_items_of(L, 1, 1, r.seg1_sv);
    const long long x_p2 = line_items_of(L, 0, 2, r.seg2), y_p2 = line_items_of(L, 1, 2, r.seg2);
    r.xpad_re = round32(x_re);
    r.xpad_sv = round32(x_sv);
    r.xpad_p2 = round32(x_p2);
    r.w1_re = (r.xpad_re + round32(y_re)) / 32;
    r.w1_sv = (r.xpad_sv + round32(y_sv)) / 32;
    r.off_prim = std::max(r.w1_re, r.w1_sv);
    r.w_prim = round32(L.plane) / 32;
    r.off_g = r.off_prim + r.w_prim;
    r.w_g = round32(d.ib.n) / 32;
    r.off_s = r.off_g + r.w_g;
    r.w_s = round32(r.ibt.nsrc) / 32;
    const long long cnt[js::RK_N] = {
        round32(L.plane), round32(4LL * L.nx * L.ny), round32(d.ib.n), round32(js::halo_count(L)),
        r.xpad_re + round32(y_re), r.xpad_sv + round32(y_sv), r.xpad_p2 + round32(y_p2),
        round32(6LL * (L.nx + 6)), round32(6LL * L.ny), round32(r.ibt.nsrc)};
    for (int q = 0; q < js::RK_N; ++q) pre[(size_t)q * (n + 1) + k + 1] = pre[(size_t)q * (n + 1) + k] + cnt[q];
  }
  const size_t smem = batch_smem();
  if (cudaFuncSetAttribute(js::batch_vjp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return JS_ERR_CUDA;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, js::batch_vjp_kernel, js::BNT, smem);
  if (per_sm < 1) return JS_ERR_CUDA;
  b->rev_blocks = sms * per_sm;
  // the split launch: each phase kernel's own resident blocks per SM
  if (cudaFuncSetAttribute(js::batch_vjp_phase_kernel<js::RP_STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return JS_ERR_CUDA;
  const void* kern[js::RP_N] = {
      (const void*)js::batch_vjp_phase_kernel<js::RP_PACK>, (const void*)js::batch_vjp_phase_kernel<js::RP_GHOST>,
      (const void*)js::batch_vjp_phase_kernel<js::RP_HALO>, (const void*)js::batch_vjp_phase_kernel<js::RP_STAGE>,
      (const void*)js::batch_vjp_phase_kernel<js::RP_SEED>, (const void*)js::batch_vjp_phase_kernel<js::RP_PASS1>,
      (const void*)js::batch_vjp_phase_kernel<js::RP_PASS2>, (const void*)js::batch_vjp_phase_kernel<js::RP_PRIMVJP>,
      (const void*)js::batch_vjp_phase_kernel<js::RP_BCTY>, (const void*)js::batch_vjp_phase_kernel<js::RP_BCTX>,
      (const void*)js::batch_vjp_phase_kernel<js::RP_INFLOW_GHOST>,
      (const void*)js::batch_vjp_phase_kernel<js::RP_SRC>, (const void*)js::batch_vjp_phase_kernel<js::RP_UNPACK>};
  for (int ph = 0; ph < js::RP_N; ++ph) {
    int ps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kern[ph], js::BNT, ph == js::RP_STAGE ? smem : 0) !=
            cudaSuccess ||
        ps < 1)
      return JS_ERR_CUDA;
    b->rev_pblocks[ph] = sms * ps;
  }
  const void* p1[2][2] = {
      {(const void*)js::batch_vjp_pass1_kernel<false, false>, (const void*)js::batch_vjp_pass1_kernel<false, true>},
      {(const void*)js::batch_vjp_pass1_kernel<true, false>, (const void*)js::batch_vjp_pass1_kernel<true, true>}};
  for (int sv = 0; sv < 2; ++sv)
    for (int v = 0; v < 2; ++v) {
      int ps = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, p1[sv][v], js::BNT, 0) != cudaSuccess || ps < 1)
        return JS_ERR_CUDA;
      b->rev_p1blocks[sv][v] = sms * ps;
    }
  b->has_visc = b->has_inv = false;
  for (int k = 0; k < n; ++k) (b->desc[k].visc ? b->has_visc : b->has_inv) = true;
  if (cudaMalloc(&b->d_rev, sizeof(js::InstRev) * n) != cudaSuccess ||
      cudaMalloc(&b->d_pre, sizeof(long long) * pre.size()) != cudaSuccess ||
      cudaMalloc(&b->d_tab, sizeof(void*) * 4 * n) != cudaSuccess ||
      cudaMalloc(&b->d_dt, sizeof(double) * n) != cudaSuccess)
    return JS_ERR_NOMEM;
  if (cudaMemcpy(b->d_rev, rev.data(), sizeof(js::InstRev) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_pre, pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return JS_ERR_CUDA;
  b->rev_ready = true;
  return JS_OK;
}

// one persistent cooperative launch reversing one step of every instance
int rev_launch(js_batch* b, const js::RevCall& call) {
  js::BatchRevArgs a;
  a.inst = b->d_desc;
  a.rev = b->d_rev;
  a.count = b->count;
  a.pre = b->d_pre;
  a.tile0 = b->d_tile0;
  a.call = call;
  a.bar = b->d_bar;
  a.err = b->d_err;
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  a.budget = (long long)(2.0 * (khz > 0 ? khz : 2000000) * 1e3);  // 2 s of SM clock cycles
  if (b->rev_split) {
    // one launch per phase, in the persistent kernel's order; kernel boundaries take the place
    // of its grid barriers
    bool ok = true;
    auto run = [&](auto kernel, int ph, int s) {
      if (!ok) return;
      kernel<<<b->rev_pblocks[ph], js::BNT, ph == js::RP_STAGE ? batch_smem() : 0, b->stream>>>(a, s);
      ok = cudaGetLastError() == cudaSuccess;
    };
    run(js::batch_vjp_phase_kernel<js::RP_PACK>, js::RP_PACK, 0);
    for (int s = 0; s < 3; ++s) {
      run(js::batch_vjp_phase_kernel<js::RP_GHOST>, js::RP_GHOST, s);
      run(js::batch_vjp_phase_kernel<js::RP_HALO>, js::RP_HALO, s);
      if (s == 2) break;
      if (call.U1) continue;
      run(js::batch_vjp_phase_kernel<js::RP_STAGE>, js::RP_STAGE, s);
    }
    for (int s = 2; s >= 0; --s) {
      run(js::batch_vjp_phase_kernel<js::RP_SEED>, js::RP_SEED, s);
      if (ok) {
        // pass 1 reads the WENO5 internals stored by the forward recompute of stages 0 and 1
        // when the stage states were not given (the device's rev_saved)
        // (one kernel for the viscous instances, one for the inviscid ones)
        const bool sv = s < 2 && call.U1 == nullptr;
        cudaStream_t st = b->stream;
        if (sv) {
          if (b->has_visc) js::batch_vjp_pass1_kernel<true, true><<<b->rev_p1blocks[1][1], js::BNT, 0, st>>>(a, s);
          if (b->has_inv) js::batch_vjp_pass1_kernel<true, false><<<b->rev_p1blocks[1][0], js::BNT, 0, st>>>(a, s);
        } else {
          if (b->has_visc) js::batch_vjp_pass1_kernel<false, true><<<b->rev_p1blocks[0][1], js::BNT, 0, st>>>(a, s);
          if (b->has_inv) js::batch_vjp_pass1_kernel<false, false><<<b->rev_p1blocks[0][0], js::BNT, 0, st>>>(a, s);
        }
        ok = cudaGetLastError() == cudaSuccess;
      }
      run(js::batch_vjp_phase_kernel<js::RP_PASS2>, js::RP_PASS2, s);
      run(js::batch_vjp_phase_kernel<js::RP_PRIMVJP>, js::RP_PRIMVJP, s);
      run(js::batch_vjp_phase_kernel<js::RP_BCTY>, js::RP_BCTY, s);
      run(js::batch_vjp_phase_kernel<js::RP_BCTX>, js::RP_BCTX, s);
      run(js::batch_vjp_phase_kernel<js::RP_INFLOW_GHOST>, js::RP_INFLOW_GHOST, s);
      run(js::batch_vjp_phase_kernel<js::RP_SRC>, js::RP_SRC, s);
    }
    run(js::batch_vjp_phase_kernel<js::RP_UNPACK>, js::RP_UNPACK, 0);
    return ok ? JS_OK : JS_ERR_CUDA;
  }
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((void*)js::batch_vjp_kernel, dim3(b->rev_blocks), dim3(js::BNT), args,
                                  batch_smem(), b->stream) != cudaSuccess)
    return JS_ERR_CUDA;
  return JS_OK;
}

}  // namespace

extern "C" {

void js_batch_destroy(js_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
  cudaFree(b->d_rev); cudaFree(b->d_pre); cudaFree(b->d_tab); cudaFree(b->d_dt); cudaFree(b->d_order);
  for (double* p : b->ro_buf) cudaFree(p);
  cudaFree(b->d_ro); cudaFree(b->d_spre);
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
  b->sms = sms;
  b->per_sm = per_sm;
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
  b->ro_fwd_log = nullptr;
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
                        double budget_s, const double* dt_in = nullptr, double* const* ustate = nullptr,
                        double* const* save = nullptr, double* const* save1 = nullptr,
                        double* const* save2 = nullptr) {
  if (!ustate) b->ro_fwd_log = nullptr;  // the registered states move: kept checkpoints are stale
  js::BatchArgs a;
  a.dt_in = dt_in;
  a.ustate = ustate;
  a.save = save;
  a.save1 = save1;
  a.save2 = save2;
  a.order = b->schedule ? b->d_order : nullptr;
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
  for (int k = 0; k < b->count; ++k)
    if (!U_n[k] || !lam_np1[k] || !lam_n[k] || !(dt[k] > 0.0)) return JS_ERR_ARG;
  int rc = rev_prepare(b);
  if (rc) return rc;
  // the call table: pointers and step sizes of this call (copied before the call returns)
  std::vector<void*> tab(4 * (size_t)b->count);
  for (int k = 0; k < b->count; ++k) {
    tab[k] = U_n[k];
    tab[b->count + k] = lam_np1[k];
    tab[2 * b->count + k] = lam_n[k];
    tab[3 * b->count + k] = p_bar ? p_bar[k] : nullptr;
  }
  if (cudaMemcpyAsync(b->d_tab, tab.data(), sizeof(void*) * tab.size(), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->d_dt, dt, sizeof(double) * b->count, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)  // the host arrays may change after the call
    return JS_ERR_CUDA;
  js::RevCall call;
  call.Un = reinterpret_cast<const double* const*>(b->d_tab);
  call.lam1 = reinterpret_cast<const double* const*>(b->d_tab + b->count);
  call.lam0 = reinterpret_cast<double* const*>(b->d_tab + 2 * b->count);
  call.pbar = p_bar ? reinterpret_cast<double* const*>(b->d_tab + 3 * b->count) : nullptr;
  call.dt = b->d_dt;
  call.U1 = call.U2 = nullptr;  // the reverse recomputes the stage states
  return rev_launch(b, call);
}

int js_batch_step_fixed(js_batch* b, int n_steps, const double* dt) {
  if (!b || !b->states_set || n_steps < 0 || (n_steps > 0 && !dt)) return JS_ERR_ARG;
  return batch_launch(b, 0.5, n_steps, nullptr, nullptr, 0, 2.0, dt);
}

namespace {
// one launch copying the states of table src into those of table dst (device tables of count
// pointers)
int batch_copy(js_batch* b, void* const* src, void* const* dst) {
  js::batch_copy_kernel<<<4 * 152, 256, 0, b->stream>>>(reinterpret_cast<const double* const*>(src),
                                                        reinterpret_cast<double* const*>(dst), b->d_spre, b->count);
  return cudaGetLastError() == cudaSuccess ? JS_OK : JS_ERR_CUDA;
}

// Rollout workspace for (n_steps, ckpt), per instance: nck checkpoints (the state after every
// ckpt-th step), the segment states U (ckpt + 1: a re-run saves the state after each of its
// steps), the stage states U1, U2 of m steps (m = ckpt; with ckpt = 1 every step's, which the
// forward keeps) and one working state; and the device pointer tables, one block of `count`
// pointers each (allocates and synchronises: before any stream capture)
struct RoLayout {
  int nck, ckpt, m;
  size_t cp(int c) const { return 1 + (size_t)c; }
  size_t segU(int j) const { return 1 + (size_t)nck + j; }
  size_t segU1(int j) const { return 1 + (size_t)nck + ckpt + 1 + j; }
  size_t segU2(int j) const { return 1 + (size_t)nck + ckpt + 1 + m + j; }
  size_t work() const { return 1 + (size_t)nck + ckpt + 1 + 2 * (size_t)m; }
  size_t lam() const { return work() + 1; }
  size_t pbar() const { return work() + 2; }
  size_t blocks() const { return work() + 3; }
  size_t states() const { return (size_t)nck + ckpt + 1 + 2 * (size_t)m + 1; }
};
RoLayout ro_layout(int n_steps, int ckpt) {
  RoLayout L;
  L.nck = (n_steps + ckpt - 1) / ckpt;
  L.ckpt = ckpt;
  L.m = (ckpt == 1) ? n_steps : ckpt;
  return L;
}

int rollout_prepare(js_batch* b, int n_steps, int ckpt) {
  const int n = b->count;
  const RoLayout L = ro_layout(n_steps, ckpt);
  if (b->ro_steps == n_steps && b->ro_ckpt == ckpt && b->d_ro) {
    // the registered states' pointers (table block 0) may have changed since
    bool same = true;
    for (int k = 0; k < n && same; ++k) same = b->ro_U[k] == (void*)b->desc[k].U;
    if (same) return JS_OK;
    for (int k = 0; k < n; ++k) b->ro_U[k] = b->desc[k].U;
    if (cudaMemcpyAsync(b->d_ro, b->ro_U.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
      return JS_ERR_CUDA;
    return JS_OK;
  }
  b->ro_fwd_log = nullptr;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return JS_ERR_CUDA;
  for (double* p : b->ro_buf) cudaFree(p);
  b->ro_buf.assign(n, nullptr);
  cudaFree(b->d_ro);
  b->d_ro = nullptr;
  b->ro_steps = b->ro_ckpt = b->ro_nck = 0;
  b->ro_lam.clear();
  b->ro_pbar.clear();
  std::vector<void*> tab(L.blocks() * n, nullptr);
  std::vector<long long> spre(n + 1, 0);
  for (int k = 0; k < n; ++k) {
    const size_t st = 4 * (size_t)b->desc[k].lay.nx * b->desc[k].lay.ny;
    spre[k + 1] = spre[k] + (long long)st;
    if (cudaMalloc(&b->ro_buf[k], sizeof(double) * st * L.states()) != cudaSuccess) return JS_ERR_NOMEM;
    double* q = b->ro_buf[k];
    tab[k] = b->desc[k].U;
    for (int c = 0; c < L.nck; ++c, q += st) tab[L.cp(c) * n + k] = q;
    for (int j = 0; j <= ckpt; ++j, q += st) tab[L.segU(j) * n + k] = q;
    for (int j = 0; j < L.m; ++j, q += st) tab[L.segU1(j) * n + k] = q;
    for (int j = 0; j < L.m; ++j, q += st) tab[L.segU2(j) * n + k] = q;
    tab[L.work() * n + k] = q;
  }
  if (!b->d_spre && cudaMalloc(&b->d_spre, sizeof(long long) * (n + 1)) != cudaSuccess) return JS_ERR_NOMEM;
  if (cudaMalloc(&b->d_ro, sizeof(void*) * tab.size()) != cudaSuccess) return JS_ERR_NOMEM;
  if (cudaMemcpy(b->d_ro, tab.data(), sizeof(void*) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_spre, spre.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess)
    return JS_ERR_CUDA;
  b->ro_U.assign(tab.begin(), tab.begin() + n);
  b->ro_steps = n_steps;
  b->ro_ckpt = ckpt;
  b->ro_nck = L.nck;
  return JS_OK;
}

// checkpoint spacing of a rollout of n_steps when the caller leaves it to the library (ckpt <= 0):
// the spacing of the workspace already prepared for n_steps; else 1 (every state and stage state
// kept: the reverse re-runs nothing) when that workspace takes at most half of the free device
// memory; else the integer nearest sqrt(n_steps)
int default_spacing(js_batch* b, int n_steps) {
  if (b->d_ro && b->ro_steps == n_steps) return b->ro_ckpt;
  double bytes = 0.0;
  for (int k = 0; k < b->count; ++k) bytes += 32.0 * (double)b->desc[k].lay.nx * b->desc[k].lay.ny;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (double)ro_layout(n_steps, 1).states() * bytes <= 0.5 * (double)fr)
    return 1;
  return (int)std::lround(std::sqrt((double)n_steps));
}

int spacing(js_batch* b, int n_steps, int ckpt) {
  if (ckpt <= 0) ckpt = default_spacing(b, n_steps);
  if (ckpt < 1) ckpt = 1;
  return ckpt > n_steps ? n_steps : ckpt;
}
}  // namespace

int js_batch_rollout_spacing(js_batch* b, int n_steps, int* ckpt) {
  if (!b || !b->states_set || n_steps < 1 || !ckpt) return JS_ERR_ARG;
  *ckpt = spacing(b, n_steps, 0);
  return JS_OK;
}

int js_batch_rollout_forward(js_batch* b, double cfl, int n_steps, int ckpt, double* dt_log) {
  if (!b || !b->states_set || n_steps < 1 || !dt_log || !(cfl > 0.0)) return JS_ERR_ARG;
  ckpt = spacing(b, n_steps, ckpt);
  int rc = rollout_prepare(b, n_steps, ckpt);
  if (rc) return rc;
  const int n = b->count;
  const RoLayout L = ro_layout(n_steps, ckpt);
  void** T = b->d_ro;
  auto tab = [&](size_t blk) { return reinterpret_cast<double* const*>(T + blk * n); };
  for (int c = 0; c < L.nck; ++c) {
    const int len = std::min(ckpt, n_steps - c * ckpt);
    if ((rc = batch_copy(b, T, T + L.cp(c) * n))) return rc;
    // with every state kept, the step's stage states too
    if ((rc = batch_launch(b, cfl, len, nullptr, dt_log + (size_t)c * ckpt * n, 0, 2.0, nullptr, nullptr, nullptr,
                           ckpt == 1 ? tab(L.segU1(c)) : nullptr, ckpt == 1 ? tab(L.segU2(c)) : nullptr)))
      return rc;
  }
  b->ro_fwd_log = dt_log;  // after the launches (which clear it)
  return JS_OK;
}

int js_batch_rollout_vjp(js_batch* b, int n_steps, const double* dt_log, int ckpt, double* const* lam,
                         double* const* p_bar) {
  if (!b || !b->states_set || n_steps < 1 || !dt_log || !lam) return JS_ERR_ARG;
  for (int k = 0; k < b->count; ++k)
    if (!lam[k]) return JS_ERR_ARG;
  ckpt = spacing(b, n_steps, ckpt);
  int rc = rev_prepare(b);
  if (rc) return rc;
  if ((rc = rollout_prepare(b, n_steps, ckpt))) return rc;
  const int n = b->count;
  const RoLayout L = ro_layout(n_steps, ckpt);
  void** T = b->d_ro;
  auto blk = [&](size_t i) { return T + i * n; };
  auto tab = [&](size_t i) { return reinterpret_cast<double* const*>(T + i * n); };
  auto ctab = [&](size_t i) { return reinterpret_cast<const double* const*>(T + i * n); };
  void** work = blk(L.work());
  // the lam / p_bar pointers of this call (uploaded when they differ from the previous call's)
  std::vector<void*> hl(lam, lam + n), hp(n, nullptr);
  if (p_bar)
    for (int k = 0; k < n; ++k) hp[k] = p_bar[k];
  if (hl != b->ro_lam || hp != b->ro_pbar) {
    if (cudaMemcpyAsync(blk(L.lam()), hl.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(blk(L.pbar()), hp.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
      return JS_ERR_CUDA;
    b->ro_lam = hl;
    b->ro_pbar = hp;
  }
  // forward: checkpoint c holds the state after c * ckpt steps (kept by js_batch_rollout_forward
  // when it ran these steps and nothing moved the registered states since); with ckpt = 1 every
  // step's stage states as well
  if (b->ro_fwd_log != dt_log) {
    if (ckpt == 1) {
      if ((rc = batch_copy(b, T, work))) return rc;
      for (int c = 0; c < n_steps; ++c) {
        if ((rc = batch_copy(b, work, blk(L.cp(c))))) return rc;
        if ((rc = batch_launch(b, 0.5, 1, nullptr, nullptr, 0, 2.0, dt_log + (size_t)c * n, tab(L.work()), nullptr,
                               tab(L.segU1(c)), tab(L.segU2(c)))))
          return rc;
      }
    } else {
      if ((rc = batch_copy(b, T, blk(L.cp(0))))) return rc;
      for (int c = 1; c < L.nck; ++c) {
        if ((rc = batch_copy(b, blk(L.cp(c - 1)), blk(L.cp(c))))) return rc;
        if ((rc = batch_launch(b, 0.5, ckpt, nullptr, nullptr, 0, 2.0, dt_log + (size_t)(c - 1) * ckpt * n,
                               tab(L.cp(c)))))
          return rc;
      }
    }
  }
  // reverse, segment by segment: re-run the segment keeping its states and stage states (not
  // needed with ckpt = 1), then reverse its steps from the last one
  for (int c = L.nck - 1; c >= 0; --c) {
    const int s0 = c * ckpt, len = std::min(ckpt, n_steps - s0);
    if (ckpt > 1) {
      if ((rc = batch_copy(b, blk(L.cp(c)), work))) return rc;
      if ((rc = batch_launch(b, 0.5, len, nullptr, nullptr, 0, 2.0, dt_log + (size_t)s0 * n, tab(L.work()),
                             tab(L.segU(1)), tab(L.segU1(0)), tab(L.segU2(0)))))
        return rc;
    }
    for (int j = len - 1; j >= 0; --j) {
      js::RevCall call;
      call.Un = ctab(j == 0 ? L.cp(c) : L.segU(j));
      call.U1 = ctab(ckpt == 1 ? L.segU1(c) : L.segU1(j));
      call.U2 = ctab(ckpt == 1 ? L.segU2(c) : L.segU2(j));
      call.lam1 = ctab(L.lam());
      call.lam0 = tab(L.lam());
      call.pbar = p_bar ? tab(L.pbar()) : nullptr;
      call.dt = dt_log + (size_t)(s0 + j) * n;
      if ((rc = rev_launch(b, call))) return rc;
    }
  }
  return JS_OK;
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

int js_batch_set_tuning(js_batch* b, int blocks_per_sm, int schedule) {
  if (!b || blocks_per_sm < 0 || blocks_per_sm > b->per_sm || schedule < 0 || schedule > 2) return JS_ERR_ARG;
  if (schedule != 0) {
    // queue position -> tile number
    std::vector<int> tile0(b->count + 1, 0);
    for (int k = 0; k < b->count; ++k) tile0[k + 1] = tile0[k] + b->desc[k].ntx * b->desc[k].nty;
    std::vector<int> order;
    order.reserve(b->ntiles);
    if (schedule == 1) {  // interleaved: tile j of every instance, then tile j + 1
      int most = 0;
      for (int k = 0; k < b->count; ++k) most = std::max(most, tile0[k + 1] - tile0[k]);
      for (int j = 0; j < most; ++j)
        for (int k = 0; k < b->count; ++k)
          if (tile0[k] + j < tile0[k + 1]) order.push_back(tile0[k] + j);
    } else {  // the largest instances first, each instance's tiles together
      std::vector<int> inst(b->count);
      for (int k = 0; k < b->count; ++k) inst[k] = k;
      std::stable_sort(inst.begin(), inst.end(), [&](int x, int y) {
        return tile0[x + 1] - tile0[x] > tile0[y + 1] - tile0[y];
      });
      for (int k : inst)
        for (int t = tile0[k]; t < tile0[k + 1]; ++t) order.push_back(t);
    }
    if (!b->d_order && cudaMalloc(&b->d_order, sizeof(int) * b->ntiles) != cudaSuccess) return JS_ERR_NOMEM;
    if (cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * b->ntiles, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
      return JS_ERR_CUDA;
  }
  b->schedule = schedule;
  b->blocks = b->sms * (blocks_per_sm == 0 ? b->per_sm : blocks_per_sm);
  return JS_OK;
}

int js_batch_set_reverse_launch(js_batch* b, int split) {
  if (!b || (split != 0 && split != 1)) return JS_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
  b->rev_split = split;
  return JS_OK;
}

int js_batch_get_reverse_launch(js_batch* b, int* split) {
  if (!b || !split) return JS_ERR_ARG;
  *split = b->rev_split;
  return JS_OK;
}

int js_batch_get_tuning(js_batch* b, int* blocks_per_sm, int* max_blocks_per_sm, int* schedule, int* n_schedules) {
  if (!b) return JS_ERR_ARG;
  if (blocks_per_sm) *blocks_per_sm = b->blocks / (b->sms > 0 ? b->sms : 1);
  if (max_blocks_per_sm) *max_blocks_per_sm = b->per_sm;
  if (schedule) *schedule = b->schedule;
  if (n_schedules) *n_schedules = 3;
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
