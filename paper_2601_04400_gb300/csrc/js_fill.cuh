// Per-element pieces of the forward step shared by the per-grid kernels and the persistent
// batched kernel: one domain-halo cell, one immersed-boundary ghost cell (Sec. 2, Fig. 1(c))
// and the CFL wave-speed rate of one cell.
#pragma once
#include <math_constants.h>
#include "js_device.cuh"
#include "js_internal.h"

namespace js {

// number of halo cells filled per grid: x sides on interior rows, y sides on the full width
__host__ __device__ __forceinline__ long long halo_count(const Lay& lay) {
  return 6LL * lay.ny + ((lay.ny > 1) ? 6LL * (lay.nx + 6) : 0);
}

// Fill halo cell number t (0 <= t < halo_count).  The y rule is resolved first (it reads
// x-ghost columns, which the x rule defines from interior cells), then the x rule;
// reflective sides flip the normal momentum, inflow sides hold a fixed state.
__device__ __forceinline__ void bc_fill_one(double* __restrict__ U, const Lay& lay, const BcArgs& bc, long long t) {
  const int nx = lay.nx, ny = lay.ny;
  const long long nxg = 6LL * ny;
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
  int i = di, j = dj;
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
  const long long d = lay.idx(di, dj);
#pragma unroll
  for (int c = 0; c < 4; ++c) U[c * lay.plane + d] = v[c];
}

// Ghost cell k: slip-wall (or no-slip) mirror of the bilinear interpolation of fluid cells
// at its image point.
__device__ __forceinline__ void ib_fill_one(double* __restrict__ U, const Lay& lay, const IbArgs& ib, double gamma,
                                            int wall, int k) {
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

// CFL rate (|u| + a)/dx [+ (|v| + a)/dy] of one cell with conserved values (r, mx, my, E),
// IEEE-rounded in the oracle's operation order.  A non-physical cell (rho or p not positive,
// or not finite) gets the rate +infinity: it dominates every maximum, so the step size of a
// state holding one is 0 and the CFL entry points report JS_ERR_NONPHYSICAL.
__device__ __forceinline__ double cfl_rate(double r, double mx, double my, double E, double gamma, double dx,
                                           double dy, bool two_d) {
  const double u = __ddiv_rn(mx, r), v = __ddiv_rn(my, r);
  const double ke = __dmul_rn(__dmul_rn(0.5, r), __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)));
  const double p = __dmul_rn(gamma - 1.0, __dsub_rn(E, ke));
  if (!(r > 0.0) || !(r < CUDART_INF) || !(p > 0.0) || !(p < CUDART_INF)) return CUDART_INF;
  const double a = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), r));
  double s = __ddiv_rn(__dadd_rn(fabs(u), a), dx);
  if (two_d) s = __dadd_rn(s, __ddiv_rn(__dadd_rn(fabs(v), a), dy));
  return s;
}

}  // namespace js
