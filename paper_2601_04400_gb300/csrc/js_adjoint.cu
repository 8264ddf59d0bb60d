// Reverse mode of the FP64 finite-volume stage (gradient chain rule of Sec. 2 applied to
// the discrete operator; the hand-written counterpart of backpropagation through the solver
// step of Fig. 1(d)).
//
// One stage VJP, given the adjoint of the stage output and the filled stage state X:
//   seed      lambda' = b dt Ubar_next on fluid cells (0 elsewhere); Ubar(X) gets the
//             identity and carry terms; Ubar_0 += a Ubar_next on fluid cells
//   prims     Q = prim(X) on every padded cell (same arithmetic as the forward kernel)
//   pass 1    per line: WENO5 forward (internals saved to HBM; skipped when the forward
//             stage kernel already stored them, then the face states are re-formed from the
//             saved quotients), HLLC + viscous forward and reverse per face with
//             Fbar = (lambda'_right - lambda'_left)/h; face-state adjoints saved; the adjoints
//             that go straight to cells (positivity fallback, viscous terms) saved per face
//   pass 2    per line segment: WENO5 reverse from the saved internals; a 5-cell register
//             window emits each cell's adjoint into the segment's own output slots
//   primvjp   per cell, a gather in a fixed order: Qbar = the slots of the (at most three)
//             segments of its x line and of its y line that reach it + the per-face adjoints
//             of the faces that touch it; Ubar(X) += (dprim/dX)^T Qbar (+ nu * lap of lambda')
//   bcT       transposed halo fill (y sides, then x sides), written as gathers;
//             inflow halos accumulate into the inflow-state gradient
//   ibT       transposed immersed-boundary fill: ghost adjoint -> image-point adjoint ->
//             gathered onto the fluid source cells (CSR built on the host)
// Parameter gradients (gamma, mu, Pr, nu, inflow states) are accumulated in pbar.
// No floating-point atomics: every sum runs in a fixed order (per-block partials of the
// parameter gradient reduced in block order by one block at the end of the stage), so the
// reverse pass gives the same bits on every run.
#include <cuda_runtime.h>

#include <algorithm>

#include "js_adjoint_body.cuh"
#include "js_internal.h"

namespace js {

// =======================================================================================
// per-grid launches: one thread per element (or line segment) of each phase
// =======================================================================================
__global__ void adj_seed_kernel(AdjArgs a, const double* __restrict__ Unext, double* __restrict__ Uacc, double ra,
                                double rb, double dt, int rhs_mode) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.lay.plane) adj_seed_one(a, t, Unext, Uacc, ra, rb, dt, rhs_mode);
}

__global__ void adj_prims_kernel(AdjArgs a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.lay.plane) adj_prims_one(a, t);
}

// x lines in blocks [0, bx), y lines (2D) in the blocks after them: one launch, both directions
template <bool VISC, bool HAS_T, bool SAVED>
__global__ void __launch_bounds__(64) adj_pass1_kernel(AdjArgs a, int seg_len, int bx) {
  if ((int)blockIdx.x < bx)
    pass1_body<0, VISC, HAS_T, SAVED>(a, seg_len, (long long)blockIdx.x * blockDim.x + threadIdx.x, 0);
  else
    pass1_body<1, VISC, HAS_T, SAVED>(a, seg_len, (long long)(blockIdx.x - bx) * blockDim.x + threadIdx.x,
                                      ((long long)bx * blockDim.x) >> 5);
}

__global__ void __launch_bounds__(64) adj_pass2_kernel(AdjArgs a, int seg_len, int bx) {
  if ((int)blockIdx.x < bx)
    pass2_body<0>(a, seg_len, (long long)blockIdx.x * blockDim.x + threadIdx.x);
  else
    pass2_body<1>(a, seg_len, (long long)(blockIdx.x - bx) * blockDim.x + threadIdx.x);
}

template <bool VISC>
__global__ void adj_primvjp_kernel(AdjArgs a, int seg_len) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double gb = 0.0, nb = 0.0;
  adj_primvjp_one<VISC>(a, t, seg_len, gb, nb);
  warp_partials(a.pp, global_warp(), gb, 0.0, 0.0, nb);
}

__global__ void adj_bcT_kernel(AdjArgs a, BcArgs bc, int phase_y, double* inflow_part, int tmax) {
  adj_bcT_one(a, bc, phase_y, inflow_part, tmax, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(128) adj_inflow_kernel(AdjArgs a, BcArgs bc, const double* inflow_part, int tmax,
                                                         const double* inflow_prim) {
  adj_inflow_block(a, bc, inflow_part, tmax, inflow_prim);
}

__global__ void __launch_bounds__(256) adj_pbar_reduce_kernel(const double* __restrict__ pp, long long nslot,
                                                              double* pbar) {
  const long long off = 0;
  adj_pbar_reduce_block(pp, &off, &nslot, 1, pbar);
}

__global__ void adj_ib_ghost_kernel(AdjArgs a, IbArgs ib, int wall, double* qIb) {
  double gb = 0.0;
  adj_ib_ghost_one(a, ib, wall, qIb, blockIdx.x * blockDim.x + threadIdx.x, gb);
  warp_partials(a.pp, global_warp(), gb, 0.0, 0.0, 0.0);
}

__global__ void adj_ib_src_kernel(AdjArgs a, IbTArgs tb, const double* qIb) {
  double gb = 0.0;
  adj_ib_src_one(a, tb, qIb, blockIdx.x * blockDim.x + threadIdx.x, gb);
  warp_partials(a.pp, global_warp(), gb, 0.0, 0.0, 0.0);
}

__global__ void adj_unpack_add_kernel(const double* __restrict__ P, const double* __restrict__ P2,
                                      double* __restrict__ U, Lay lay) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 4LL * lay.nx * lay.ny) adj_unpack_add_one(P, P2, U, lay, t);
}

// =======================================================================================
// launchers
// =======================================================================================
namespace {
// short segments and small blocks: enough blocks to fill every SM (one line per thread
// would leave most of the GPU idle); pass 1 pays one extra WENO cell per segment, except
// when the forward stored the internals: then a segment costs almost nothing to start and
// shorter ones split the work into finer waves
constexpr int kSeg1 = 16, kSeg1Saved = 8, kSeg1D = 4, kBlk = 64;

unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

long long line_items(const AdjArgs& a, int dir, int extra, int seg) {
  const int nline = (dir == 0) ? a.lay.ny : a.lay.nx;
  const int ncell = (dir == 0) ? a.lay.nx : a.lay.ny;
  return (long long)nline * ((ncell + extra + seg - 1) / seg);
}

// blocks of pass 1 for the x lines (bx) and the y lines (by); seg = segment length
void pass1_shape(const AdjArgs& a, bool two_d, int& seg, int& bx, int& by) {
  if (a.weno_saved) {
    seg = kSeg1Saved;
  } else {
    seg = two_d ? kSeg1 : kSeg1D;  // a 1D grid is one line: short segments give it more threads
  }
  bx = (int)blocks_for(line_items(a, 0, 1, seg), kBlk);
  by = two_d ? (int)blocks_for(line_items(a, 1, 1, seg), kBlk) : 0;
}

cudaError_t pass1(const AdjArgs& a, bool visc, bool two_d, cudaStream_t s) {
  int seg, bx, by;
  pass1_shape(a, two_d, seg, bx, by);
  if (a.weno_saved) {
    if (!two_d) return cudaErrorInvalidValue;  // the forward saves exist for 2D grids only
    if (visc) adj_pass1_kernel<true, true, true><<<bx + by, kBlk, 0, s>>>(a, seg, bx);
    else adj_pass1_kernel<false, false, true><<<bx + by, kBlk, 0, s>>>(a, seg, bx);
    return cudaGetLastError();
  }
  if (visc) {
    if (two_d) adj_pass1_kernel<true, true, false><<<bx + by, kBlk, 0, s>>>(a, seg, bx);
    else adj_pass1_kernel<true, false, false><<<bx + by, kBlk, 0, s>>>(a, seg, bx);
  } else {
    adj_pass1_kernel<false, false, false><<<bx + by, kBlk, 0, s>>>(a, seg, bx);
  }
  return cudaGetLastError();
}

int seg2_of(const Lay& L) { return L.ny > 1 ? ADJ_SEG2 : ADJ_SEG2_1D; }

cudaError_t pass2(const AdjArgs& a, bool two_d, cudaStream_t s) {
  const int seg = seg2_of(a.lay);
  const int bx = (int)blocks_for(line_items(a, 0, 2, seg), kBlk);
  const int by = two_d ? (int)blocks_for(line_items(a, 1, 2, seg), kBlk) : 0;
  adj_pass2_kernel<<<bx + by, kBlk, 0, s>>>(a, seg, bx);
  return cudaGetLastError();
}

unsigned ib_blocks(int n) { return n > 0 ? blocks_for(n, 128) : 0; }
}  // namespace

long long adj_wrev_doubles(const Lay& L) {
  const int seg = seg2_of(L);
  long long n = 4LL * ((L.nx + 2 + seg - 1) / seg) * (seg + 4) * L.ny;
  if (L.ny > 1) n += 4LL * ((L.ny + 2 + seg - 1) / seg) * (seg + 4) * L.nx;
  return n;
}

long long adj_ppart_doubles(const Lay& L, int n_ghost, int n_src, long long nn_blocks) {
  // pass 1 takes the most blocks with the shortest segments (saved internals)
  AdjArgs a;
  a.lay = L;
  const bool two_d = L.ny > 1;
  long long b1 = 0;
  for (int saved = 0; saved < 2; ++saved) {
    if (saved && !two_d) continue;
    a.weno_saved = saved;
    int seg, bx, by;
    pass1_shape(a, two_d, seg, bx, by);
    b1 = std::max(b1, (long long)bx + by);
  }
  // warps: pass 1 (64-thread blocks), the neural image reverse and primvjp (256), IB (128)
  const long long warps = 2 * b1 + 8 * nn_blocks + 8 * (long long)blocks_for(L.plane, 256) +
                          4 * (long long)(ib_blocks(n_ghost) + ib_blocks(n_src));
  return 4 * warps;
}

cudaError_t launch_adj_stage(const AdjArgs& a0, const BcArgs& bc, const IbArgs& ib, const IbTArgs& ibt, int wall,
                             const double* Unext, double* Uacc, double ra, double rb, double dt, bool rhs_mode,
                             double* inflow_part, const double* inflow_prim, double* qIb, cudaStream_t s,
                             long long* launches, const NnArgs* nn) {
  AdjArgs a = a0;
  const Lay& L = a.lay;
  const unsigned gp = blocks_for(L.plane, 256);
  long long n = 0;
  // warp partials of pbar[0..3]: consecutive slices for the launches that produce them
  double* const pp0 = a0.pbar ? a0.pp : nullptr;
  long long used = 0;
  auto slice = [&](long long warps) {
    double* p = pp0 ? pp0 + 4 * used : nullptr;
    used += warps;
    return p;
  };
  a.pp = nullptr;
  adj_seed_kernel<<<gp, 256, 0, s>>>(a, Unext, Uacc, ra, rb, dt, rhs_mode ? 1 : 0);
  adj_prims_kernel<<<gp, 256, 0, s>>>(a);
  n += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool two_d = L.ny > 1;
  {
    int seg, bx, by;
    pass1_shape(a, two_d, seg, bx, by);
    a.pp = slice(2LL * (bx + by));
    if ((e = pass1(a, a.visc != 0, two_d, s)) != cudaSuccess) return e;
  }
  if (nn) {
    // the neural flux: its face-state adjoints join the HLLC ones before the WENO5 reverse
    a.pp = slice(8 * nn_image_vjp_blocks(L));
    if ((e = nn_reverse(*nn, a, s)) != cudaSuccess) return e;
    n += nn->w_bar ? 13 : 9;
  }
  a.pp = nullptr;
  if ((e = pass2(a, two_d, s)) != cudaSuccess) return e;
  n += 2;
  a.pp = slice(8LL * gp);
  if (a.visc) adj_primvjp_kernel<true><<<gp, 256, 0, s>>>(a, seg2_of(L));
  else adj_primvjp_kernel<false><<<gp, 256, 0, s>>>(a, seg2_of(L));
  ++n;
  a.pp = nullptr;
  const int tmax = std::max(L.nx + 6, L.ny);
  if (two_d) {
    adj_bcT_kernel<<<blocks_for(6LL * (L.nx + 6), 128), 128, 0, s>>>(a, bc, 1, inflow_part, tmax);
    ++n;
  }
  adj_bcT_kernel<<<blocks_for(6LL * L.ny, 128), 128, 0, s>>>(a, bc, 0, inflow_part, tmax);
  adj_inflow_kernel<<<1, 128, 0, s>>>(a, bc, inflow_part, tmax, inflow_prim);
  n += 2;
  if (ib.n > 0) {
    a.pp = slice(4LL * ib_blocks(ib.n));
    adj_ib_ghost_kernel<<<ib_blocks(ib.n), 128, 0, s>>>(a, ib, wall, qIb);
    if (ibt.nsrc > 0) {
      a.pp = slice(4LL * ib_blocks(ibt.nsrc));
      adj_ib_src_kernel<<<ib_blocks(ibt.nsrc), 128, 0, s>>>(a, ibt, qIb);
    }
    n += 2;
  }
  if (pp0) {
    adj_pbar_reduce_kernel<<<1, 256, 0, s>>>(pp0, used, a0.pbar);
    ++n;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}

cudaError_t launch_adj_unpack(const double* P, const double* P2, double* U, const Lay& lay, cudaStream_t s) {
  adj_unpack_add_kernel<<<blocks_for(4LL * lay.nx * lay.ny, 256), 256, 0, s>>>(P, P2, U, lay);
  return cudaGetLastError();
}

}  // namespace js
