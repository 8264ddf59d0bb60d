// Device bodies of the reverse-mode stage (gradient chain rule of Sec. 2 applied to the
// discrete operator), shared by the per-grid launches of js_adjoint.cu and the persistent
// batched reverse kernel of js_batch.cu: one element, line segment or block of each phase.
#pragma once
#include <cuda_runtime.h>

#include "js_adjoint_device.cuh"
#include "js_internal.h"

namespace js {


__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-warp partial sums of the parameter gradient's gamma, mu, Pr and nu entries:
// pp[4 * w + k] = the sum over warp w's lanes (a fixed shuffle tree), w = the warp's global
// index (thread index / 32 over the launch).  Every lane calls it (no lane may have left);
// pp == nullptr (no pbar) skips it.  The partials are summed in warp order at the end of the
// stage, so the parameter gradient does not depend on timing, and two launch shapes that map
// the same items to the same warps give the same bits.
__device__ __forceinline__ void warp_partials(double* pp, long long w, double g, double m, double pr, double n) {
  if (pp == nullptr) return;
  g = warp_sum(g);
  m = warp_sum(m);
  pr = warp_sum(pr);
  n = warp_sum(n);
  if ((threadIdx.x & 31) == 0) {
    double* o = pp + 4 * w;
    o[0] = g;
    o[1] = m;
    o[2] = pr;
    o[3] = n;
  }
}
__device__ __forceinline__ long long global_warp() {
  return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

__device__ __forceinline__ bool valid_padded(const Lay& L, long long t, int& i, int& j) {
  const int col = (int)(t % L.pitch);
  const int row = (int)(t / L.pitch);
  if (col >= L.nx + 6 || row >= L.H) return false;
  i = col - 3;
  j = row - L.gy;
  return true;
}

// Position of cell k of line `line` in the saved arrays: y lines use the padded layout
// (lanes = consecutive columns); x lines are stored transposed so that the lanes of a warp
// (consecutive rows) also write consecutive addresses.
template <int DIR>
__device__ __forceinline__ long long save_id(const AdjArgs& a, int k, int line) {
  return (DIR == 0) ? (long long)(k + 3) * a.tpitch + (line + a.lay.gy) : a.lay.idx(line, k);
}

// =======================================================================================
// seed + prims
// =======================================================================================
__device__ __forceinline__ void adj_seed_one(const AdjArgs& a, long long t, const double* __restrict__ Unext,
                                             double* __restrict__ Uacc, double ra, double rb, double dt,
                                             int rhs_mode) {
  const Lay& L = a.lay;
  if (t >= L.plane) return;
  int i, j;
  if (!valid_padded(L, t, i, j)) return;
  const bool interior = i >= 0 && i < L.nx && j >= 0 && j < L.ny;
  const bool fluid = interior && (a.tag == nullptr || a.tag[(long long)j * L.nx + i] == 0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const long long o = c * L.plane + t;
    const double un = interior ? Unext[o] : 0.0;
    double lam, ub;
    if (rhs_mode) {
      lam = fluid ? un : 0.0;
      ub = 0.0;
    } else {
      lam = fluid ? rb * dt * un : 0.0;
      ub = fluid ? rb * un : un;  // identity on fluid cells, carry on solid and ghost cells
      if (fluid && ra != 0.0) Uacc[o] += ra * un;
    }
    a.lam[o] = lam;
    a.Ub[o] = ub;
  }
}

__device__ __forceinline__ void adj_prims_one(const AdjArgs& a, long long t) {
  const Lay& L = a.lay;
  if (t >= L.plane) return;
  int i, j;
  if (!valid_padded(L, t, i, j)) return;
  double u, v, p, T;
  const double r = a.X[t];
  cons_to_prim(r, a.X[L.plane + t], a.X[2 * L.plane + t], a.X[3 * L.plane + t], a.gas, u, v, p, T);
  a.Q[t] = r;
  a.Q[L.plane + t] = u;
  a.Q[2 * L.plane + t] = v;
  a.Q[3 * L.plane + t] = p;
  a.Q[4 * L.plane + t] = T;
}

// =======================================================================================
// pass 1: WENO forward (saved), HLLC + viscous forward and reverse per face
// =======================================================================================
// DIR 0: lines are rows, faces f in [0, nx] (face f between cells f-1 and f).
// DIR 1: lines are columns, faces f in [0, ny].
template <int DIR, bool VISC, bool HAS_T, bool SAVED>
__device__ __forceinline__ void pass1_body(const AdjArgs& a, int seg_len, long long item, long long wbase) {
  const Lay& L = a.lay;
  const int nline = (DIR == 0) ? L.ny : L.nx;
  const int ncell = (DIR == 0) ? L.nx : L.ny;
  const int nseg = (ncell + 1 + seg_len - 1) / seg_len;
  const bool active = item < (long long)nline * nseg;
  double gb = 0.0, mub = 0.0, prb = 0.0;
  if (active) {
    const int line = (int)(item % nline), seg = (int)(item / nline);
    const int f0 = seg * seg_len;
    const int f1 = min(f0 + seg_len, ncell + 1);
    const long long st = (DIR == 0) ? 1 : L.pitch;   // stride along the line
    const long long ts = (DIR == 0) ? L.pitch : 1;   // stride across it
    constexpr int PN = (DIR == 0) ? 1 : 2, PT = (DIR == 0) ? 2 : 1;
    const double invh = (DIR == 0) ? a.inv_dx : a.inv_dy;
    const ViscC& vc = (DIR == 0) ? a.vx : a.vy;
    const int wdir = DIR * 4 * WENO_SAVE;
    auto cell_id = [&](int k) { return (DIR == 0) ? L.idx(k, line) : L.idx(line, k); };
    // window at cell i = f0 - 1: q_{i-2..i+1}
    double q0[4], q1[4];
    Dl d[4];
    if (!SAVED) {
      const long long b = cell_id(f0 - 1);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double* q = a.Q + c * L.plane;
        const double qm2 = q[b - 2 * st], qm1 = q[b - st], qc = q[b], qp1 = q[b + st];
        q0[c] = qc;
        q1[c] = qp1;
        d[c].m2 = 0.0;
        d[c].m1 = qm1 - qm2;
        d[c].p1 = qc - qm1;
        d[c].p2 = qp1 - qc;
      }
    }
    double prevL[4];
#pragma unroll 1
    for (int i = f0 - 1; i < f1; ++i) {
      const long long ci = cell_id(i);
      const long long si = save_id<DIR>(a, i, line);
      double Lf[4], Rf[4];
      if (SAVED) {
        // face states of cell i from the quotients the forward stage stored
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double qc = a.Q[c * L.plane + ci];
          const double* sv = a.wsave + (long long)(wdir + c * WENO_SAVE) * a.splane + si;
          Lf[c] = fma(sv[3 * a.splane], SIXTH, qc);
          Rf[c] = fma(sv[5 * a.splane], SIXTH, qc);
        }
      } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        // slide: d.m2 <- d.m1 ... and bring in q_{i+2}
        const double q2 = a.Q[c * L.plane + ci + 2 * st];
        d[c].m2 = d[c].m1;
        d[c].m1 = d[c].p1;
        d[c].p1 = d[c].p2;
        d[c].p2 = q2 - q1[c];
        double sv[WENO_SAVE];
        weno_cell_fwd(q0[c], d[c], Lf[c], Rf[c], sv);
#pragma unroll
        for (int k = 0; k < WENO_SAVE; ++k) a.wsave[(long long)(wdir + c * WENO_SAVE + k) * a.splane + si] = sv[k];
        q0[c] = q1[c];
        q1[c] = q2;
      }
      }
      if (i >= f0) {
        // face f = i between cells i-1 (state prevL) and i (state Rf)
        const long long ca = ci - st, cb = ci;
        double ql[4], qr[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) { ql[c] = prevL[c]; qr[c] = Rf[c]; }
        const bool fallback = !(ql[0] > 0.0 && ql[3] > 0.0 && qr[0] > 0.0 && qr[3] > 0.0);
        if (fallback) {
#pragma unroll
          for (int c = 0; c < 4; ++c) { ql[c] = a.Q[c * L.plane + ca]; qr[c] = a.Q[c * L.plane + cb]; }
        }
        double Fb[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) Fb[c] = (a.lam[c * L.plane + cb] - a.lam[c * L.plane + ca]) * invh;
        const Face4 FL{ql[0], ql[PN], ql[PT], ql[3]}, FR{qr[0], qr[PN], qr[PT], qr[3]};
        Face4 bL{0.0, 0.0, 0.0, 0.0}, bR{0.0, 0.0, 0.0, 0.0};
        const double Fbn[4] = {Fb[0], Fb[PN], Fb[PT], Fb[3]};
        hllc_vjp(FL, FR, a.gas, Fbn, bL, bR, gb);
        double bql[4], bqr[4];
        bql[0] = bL.r; bql[PN] = bL.un; bql[PT] = bL.ut; bql[3] = bL.p;
        bqr[0] = bR.r; bqr[PN] = bR.un; bqr[PT] = bR.ut; bqr[3] = bR.p;
        const int fdir = DIR * 8;
        // adjoints that go straight to the face's cells ca (left) and cb (right): rho, u, v, p, T
        double dca[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, dcb[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (fallback) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            dca[c] = bql[c];
            dcb[c] = bqr[c];
            a.fadj[(long long)(fdir + c) * a.splane + si] = 0.0;
            a.fadj[(long long)(fdir + 4 + c) * a.splane + si] = 0.0;
          }
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            a.fadj[(long long)(fdir + c) * a.splane + si] = bql[c];      // left state of face
            a.fadj[(long long)(fdir + 4 + c) * a.splane + si] = bqr[c];  // right state of face
          }
        }
        double* fc = a.fcell + (long long)(DIR * 12) * a.splane + si;
        if (VISC) {
          // F[n] -= tnn; F[t] -= tnt; F[3] -= 0.5 (sbn tnn + sbt tnt) + ck dT
          const double* un = a.Q + PN * L.plane;
          const double* ut = a.Q + PT * L.plane;
          const double* Tq = a.Q + 4 * L.plane;
          const double dun = un[cb] - un[ca], dut = ut[cb] - ut[ca], dT = Tq[cb] - Tq[ca];
          double sun = 0.0, sut = 0.0, tnn, tnt;
          if (HAS_T) {
            sun = (un[ca + ts] - un[ca - ts]) + (un[cb + ts] - un[cb - ts]);
            sut = (ut[ca + ts] - ut[ca - ts]) + (ut[cb + ts] - ut[cb - ts]);
            tnn = fma(vc.c43n, dun, -vc.c23t * sut);
            tnt = fma(vc.cn, dut, vc.ct * sun);
          } else {
            tnn = vc.c43n * dun;
            tnt = vc.cn * dut;
          }
          const double sbn = un[ca] + un[cb], sbt = ut[ca] + ut[cb];
          const double btnn = -Fb[PN] - 0.5 * Fb[3] * sbn;
          const double btnt = -Fb[PT] - 0.5 * Fb[3] * sbt;
          const double bsbn = -0.5 * Fb[3] * tnn, bsbt = -0.5 * Fb[3] * tnt;
          const double bck = -Fb[3] * dT;
          const double bdT = -Fb[3] * vc.ck;
          const double bdun = vc.c43n * btnn, bdut = vc.cn * btnt;
          dca[PN] += bsbn - bdun;
          dcb[PN] += bsbn + bdun;
          dca[PT] += bsbt - bdut;
          dcb[PT] += bsbt + bdut;
          dca[4] = -bdT;
          dcb[4] = bdT;
          // tangential differences: +(bsun, bsut) to the cells ca + ts and cb + ts, minus to
          // ca - ts and cb - ts (gathered by those cells)
          fc[10 * a.splane] = HAS_T ? vc.ct * btnt : 0.0;
          fc[11 * a.splane] = HAS_T ? -vc.c23t * btnn : 0.0;
          const double ckck = bck * vc.ck;
          mub += a.inv_mu * fma(btnn, tnn, fma(btnt, tnt, ckck));
          gb += a.kg * ckck;
          prb += a.kp * ckck;
        }
#pragma unroll
        for (int c = 0; c < (VISC ? 5 : 4); ++c) {
          fc[c * a.splane] = dca[c];
          fc[(5 + c) * a.splane] = dcb[c];
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) prevL[c] = Lf[c];
    }
  }
  warp_partials(a.pp, wbase + (item >> 5), gb, mub, prb, 0.0);
}

// =======================================================================================
// pass 2: WENO reverse from the saved internals, along line segments.  Segment `seg` of a
// line runs cells c0 = -1 + seg * L .. c1 - 1 and emits the adjoints of cells c0 - 2 .. c1 + 1
// (its whole reach) into its own slots; a cell's total is gathered later from the (at most
// three) segments that reach it, in segment order.
// =======================================================================================
// slot k of segment seg, variable c, in direction DIR's part of wrev (lines fastest)
template <int DIR>
__device__ __forceinline__ long long wrev_slot(const Lay& L, int seg_len, int c, int seg, int k, int line) {
  const int nline = (DIR == 0) ? L.ny : L.nx;
  const int ncell = (DIR == 0) ? L.nx : L.ny;
  const long long nseg = (ncell + 2 + seg_len - 1) / seg_len;
  const long long base = (DIR == 0) ? 0 : 4LL * ((L.nx + 2 + seg_len - 1) / seg_len) * (seg_len + 4) * L.ny;
  return base + ((c * nseg + seg) * (seg_len + 4) + k) * nline + line;
}

template <int DIR>
__device__ __forceinline__ void pass2_body(const AdjArgs& a, int seg_len, long long item) {
  const Lay& L = a.lay;
  const int nline = (DIR == 0) ? L.ny : L.nx;
  const int ncell = (DIR == 0) ? L.nx : L.ny;
  const int nseg = (ncell + 2 + seg_len - 1) / seg_len;  // cells -1 .. ncell
  if (item >= (long long)nline * nseg) return;
  const int line = (int)(item % nline), seg = (int)(item / nline);
  const int c0 = -1 + seg * seg_len;
  const int c1 = min(c0 + seg_len, ncell + 1);
  const long long st = (DIR == 0) ? 1 : L.pitch;
  const int wdir = DIR * 4 * WENO_SAVE;
  const int fdir = DIR * 8;
  auto cell_id = [&](int k) { return (DIR == 0) ? L.idx(k, line) : L.idx(line, k); };
  for (int c = 0; c < 4; ++c) {
    // one variable at a time keeps the register window small
    const double* q = a.Q + c * L.plane;
    double* out = a.wrev + wrev_slot<DIR>(L, seg_len, c, seg, 0, line);
    long long ci = cell_id(c0);
    const long long sst = (DIR == 0) ? a.tpitch : L.pitch;  // stride along the line in saved arrays
    long long si = save_id<DIR>(a, c0, line);
    WenoRev w;
    w.init(q[ci - 2 * st], q[ci - st], q[ci], q[ci + st]);
    int k = 0;  // slot of cell c0 - 2 + k
#pragma unroll 1
    for (int i = c0; i < c1; ++i, ci += st, si += sst, ++k) {
      double sv[WENO_SAVE];
#pragma unroll
      for (int m = 0; m < WENO_SAVE; ++m) sv[m] = a.wsave[(long long)(wdir + c * WENO_SAVE + m) * a.splane + si];
      const double Lb = a.fadj[(long long)(fdir + c) * a.splane + si + sst];  // left state of face i+1/2
      const double Rb = a.fadj[(long long)(fdir + 4 + c) * a.splane + si];    // right state of face i-1/2
      // cell i-2: this segment's contribution is complete
      out[(long long)k * nline] = w.step(q[ci + 2 * st], sv, Lb, Rb);
    }
    // cells c1-2 .. c1+1
    double rest[4];
    w.flush(rest);
    for (int m = 0; m < 4; ++m) out[(long long)(k + m) * nline] = rest[m];
  }
}

// sum of the pass-2 slots of the segments of a DIR line that reach cell m (-3 <= m <= ncell + 2),
// in segment order
template <int DIR>
__device__ __forceinline__ double wrev_gather(const AdjArgs& a, int seg_len, int c, int m, int line) {
  const Lay& L = a.lay;
  const int ncell = (DIR == 0) ? L.nx : L.ny;
  const int nseg = (ncell + 2 + seg_len - 1) / seg_len;
  int s = (m + 1 >= 0) ? (m + 1) / seg_len : 0;
  s = min(s, nseg - 1);
  double t = 0.0;
  for (int q = s - 1; q <= s + 1; ++q) {
    if (q < 0 || q >= nseg) continue;
    const int c0 = -1 + q * seg_len;
    const int c1 = min(c0 + seg_len, ncell + 1);
    if (m < c0 - 2 || m >= c1 + 2) continue;
    t += a.wrev[wrev_slot<DIR>(L, seg_len, c, q, m - (c0 - 2), line)];
  }
  return t;
}

// =======================================================================================
// prim reverse (+ artificial viscosity), after gathering each cell's primitive adjoint
// =======================================================================================
// per-face adjoints of direction DIR that reach padded cell (i, j), added to qb in a fixed
// order: the face to its low side (the cell is its right cell), the face to its high side,
// then (viscous, 2D) the tangential-difference terms of the faces of the two neighbouring
// lines: + from the line below, - from the line above
template <int DIR, bool VISC>
__device__ __forceinline__ void face_gather(const AdjArgs& a, int i, int j, double qb[5]) {
  const Lay& L = a.lay;
  const int m = (DIR == 0) ? i : j, line = (DIR == 0) ? j : i;
  const int nline = (DIR == 0) ? L.ny : L.nx, ncell = (DIR == 0) ? L.nx : L.ny;
  constexpr int PN = (DIR == 0) ? 1 : 2, PT = (DIR == 0) ? 2 : 1, NC = VISC ? 5 : 4;
  const long long sp = a.splane;
  const double* fc = a.fcell + (long long)(DIR * 12) * sp;
  if (line >= 0 && line < nline) {
    if (m >= 0 && m <= ncell) {
      const long long f = save_id<DIR>(a, m, line);
#pragma unroll
      for (int c = 0; c < NC; ++c) qb[c] += fc[(5 + c) * sp + f];
    }
    if (m + 1 >= 0 && m + 1 <= ncell) {
      const long long f = save_id<DIR>(a, m + 1, line);
#pragma unroll
      for (int c = 0; c < NC; ++c) qb[c] += fc[c * sp + f];
    }
  }
  if (VISC && a.two_d) {
#pragma unroll
    for (int dl = -1; dl <= 1; dl += 2) {
      const int ln = line + dl;
      if (ln < 0 || ln >= nline) continue;
      for (int f = m; f <= m + 1; ++f) {
        if (f < 0 || f > ncell) continue;
        const long long id = save_id<DIR>(a, f, ln);
        if (dl < 0) {
          qb[PN] += fc[10 * sp + id];
          qb[PT] += fc[11 * sp + id];
        } else {
          qb[PN] -= fc[10 * sp + id];
          qb[PT] -= fc[11 * sp + id];
        }
      }
    }
  }
}

// padded cell t; the gamma and nu parameter-gradient contributions are added to gb, nb
template <bool VISC>
__device__ __forceinline__ void adj_primvjp_one(const AdjArgs& a, long long t, int seg_len, double& gb, double& nb) {
  const Lay& L = a.lay;
  int i = 0, j = 0;
  if (t < L.plane && valid_padded(L, t, i, j)) {
    // primitive adjoint: WENO5 reverse of the cell's x line and y line, then the faces
    double qb[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (j >= 0 && j < L.ny) {
#pragma unroll
      for (int c = 0; c < 4; ++c) qb[c] += wrev_gather<0>(a, seg_len, c, i, j);
    }
    if (a.two_d && i >= 0 && i < L.nx) {
#pragma unroll
      for (int c = 0; c < 4; ++c) qb[c] += wrev_gather<1>(a, seg_len, c, j, i);
    }
    face_gather<0, VISC>(a, i, j, qb);
    if (a.two_d) face_gather<1, VISC>(a, i, j, qb);
    double ub[4];
    prim_vjp(a.X[t], a.X[L.plane + t], a.X[2 * L.plane + t], a.X[3 * L.plane + t], a.gas, qb, ub, gb);
    if (a.has_av) {
      const bool near = i >= -1 && i <= L.nx && j >= (a.two_d ? -1 : 0) && j <= (a.two_d ? L.ny : 0);
      const bool interior = i >= 0 && i < L.nx && j >= 0 && j < L.ny;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double* lam = a.lam + c * L.plane;
        if (near) {
          double add = a.nu_x * ((lam[t - 1] - 2.0 * lam[t]) + lam[t + 1]);
          if (a.two_d) add += a.nu_y * ((lam[t - L.pitch] - 2.0 * lam[t]) + lam[t + L.pitch]);
          ub[c] += add;
        }
        if (interior && lam[t] != 0.0) {
          const double* X = a.X + c * L.plane;
          double lap = a.nu_x1 * ((X[t - 1] - 2.0 * X[t]) + X[t + 1]);
          if (a.two_d) lap += a.nu_y1 * ((X[t - L.pitch] - 2.0 * X[t]) + X[t + L.pitch]);
          nb += lam[t] * lap;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) a.Ub[c * L.plane + t] += ub[c];
  }
}

// =======================================================================================
// transposed halo fill (gathers).  y sides first: targets are cells of interior rows (all
// padded columns); then x sides: targets are interior cells.
// =======================================================================================
__device__ __forceinline__ bool halo_source(int kind, int k, int n, bool low, int& src, bool& flip) {
  flip = false;
  switch (kind) {
    case 0: src = low ? 0 : n - 1; return true;
    case 1: src = low ? k - 1 : n - k; flip = true; return true;
    case 2: src = low ? n - k : k - 1; return true;
    default: return false;  // inflow
  }
}

__device__ __forceinline__ void adj_bcT_one(const AdjArgs& a, const BcArgs& bc, int phase_y, double* inflow_part,
                                            int tmax, long long t) {
  const Lay& L = a.lay;
  // targets: 6 source rows/columns next to each boundary
  const int ntan = phase_y ? L.nx + 6 : L.ny;
  if (t < 6LL * ntan) {
    const int r = (int)(t % 6);
    const int tan = (int)(t / 6) - (phase_y ? 3 : 0);
    const int n = phase_y ? L.ny : L.nx;
    const int tgt = (r < 3) ? r : n - 6 + r;  // 0,1,2, n-3,n-2,n-1
    const int comp = phase_y ? 2 : 1;          // momentum component normal to the side
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s = 0; s < 2; ++s) {
      const int side = (phase_y ? 2 : 0) + s;
      for (int k = 1; k <= 3; ++k) {
        int src;
        bool flip;
        if (!halo_source(bc.kind[side], k, n, s == 0, src, flip) || src != tgt) continue;
        const int h = (s == 0) ? -k : n - 1 + k;
        const long long hid = phase_y ? L.idx(tan, h) : L.idx(h, tan);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double v = a.Ub[c * L.plane + hid];
          acc[c] += (flip && c == comp) ? -v : v;
        }
      }
    }
    const long long tid = phase_y ? L.idx(tan, tgt) : L.idx(tgt, tan);
#pragma unroll
    for (int c = 0; c < 4; ++c) a.Ub[c * L.plane + tid] += acc[c];
  }
  // inflow sides: the halo adjoints of each (side, tangential position), its three layers in
  // order, into inflow_part[side][position] (summed over positions by adj_inflow_kernel)
  if (t < 2LL * ntan) {
    const int s = (int)(t % 2);
    const int tpos = (int)(t / 2);  // 0 .. ntan - 1
    const int tan = tpos - (phase_y ? 3 : 0);
    const int side = (phase_y ? 2 : 0) + s;
    if (bc.kind[side] == 3) {
      const int n = phase_y ? L.ny : L.nx;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = 1; k <= 3; ++k) {
        const int h = (s == 0) ? -k : n - 1 + k;
        const long long hid = phase_y ? L.idx(tan, h) : L.idx(h, tan);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += a.Ub[c * L.plane + hid];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) inflow_part[((long long)side * tmax + tpos) * 4 + c] = acc[c];
    }
  }
}

// inflow halo adjoints (conserved) -> gradient of the inflow primitive state and gamma; one
// warp per side sums its partials in a fixed order, then one thread adds to pbar side by side
__device__ __forceinline__ void adj_inflow_block(const AdjArgs& a, const BcArgs& bc, const double* inflow_part,
                                                 int tmax, const double* inflow_prim) {
  __shared__ double S[4][4];
  const int side = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Lay& L = a.lay;
  if (bc.kind[side] == 3 && a.pbar != nullptr) {
    const int ntan = (side < 2) ? L.ny : L.nx + 6;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = lane; k < ntan; k += 32)
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] += inflow_part[((long long)side * tmax + k) * 4 + c];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = warp_sum(v[c]);
    if (lane == 0)
#pragma unroll
      for (int c = 0; c < 4; ++c) S[side][c] = v[c];
  }
  __syncthreads();
  if (threadIdx.x != 0 || a.pbar == nullptr) return;
  for (int sd = 0; sd < 4; ++sd) {
    if (bc.kind[sd] != 3) continue;
    const double* s = S[sd];
    const double r = inflow_prim[4 * sd], u = inflow_prim[4 * sd + 1], v = inflow_prim[4 * sd + 2],
                 p = inflow_prim[4 * sd + 3];
    // U = (r, r u, r v, p/(gamma-1) + r (u^2 + v^2)/2)
    a.pbar[4 + 4 * sd + 0] += s[0] + s[1] * u + s[2] * v + s[3] * 0.5 * (u * u + v * v);
    a.pbar[4 + 4 * sd + 1] += s[1] * r + s[3] * r * u;
    a.pbar[4 + 4 * sd + 2] += s[2] * r + s[3] * r * v;
    a.pbar[4 + 4 * sd + 3] += s[3] * a.gas.g1;
    a.pbar[0] += -s[3] * p * a.gas.g1 * a.gas.g1;
  }
}

// pbar[0..3] += the warp partials pp[4 * b + k] of the slot ranges [off[r], off[r] + cnt[r]),
// r < nr: each thread over a fixed set of slots, then a fixed reduction tree over the block
// (blockDim.x a power of two, at most 256)
__device__ __forceinline__ void adj_pbar_reduce_block(const double* __restrict__ pp, const long long* off,
                                                      const long long* cnt, int nr, double* pbar) {
  __shared__ double red[4][256];
  const int nt = blockDim.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r = 0; r < nr; ++r)
    for (long long b = threadIdx.x; b < cnt[r]; b += nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] += pp[4 * (off[r] + b) + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = nt / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) pbar[threadIdx.x] += red[threadIdx.x][0];
  __syncthreads();
}

// =======================================================================================
// transposed immersed-boundary fill
// =======================================================================================
__device__ __forceinline__ void adj_ib_ghost_one(const AdjArgs& a, const IbArgs& ib, int wall, double* qIb, int k,
                                                 double& gb) {
  if (k < ib.n) {
    const Lay& L = a.lay;
    const double gamma = a.gas.gamma;
    double q[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double w = ib.w[4 * k + m];
      if (w == 0.0) continue;
      const long long s = ib.src[4 * k + m];
      const double r = a.X[s], u = a.X[L.plane + s] / r, v = a.X[2 * L.plane + s] / r;
      const double p = (gamma - 1.0) * (a.X[3 * L.plane + s] - 0.5 * r * (u * u + v * v));
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
    double G[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      G[c] = a.Ub[c * L.plane + d];
      a.Ub[c * L.plane + d] = 0.0;  // the ghost's own input value is overwritten by the fill
    }
    // G = (r, r ug, r vg, p/(gamma-1) + r (ug^2 + vg^2)/2)
    const double br = G[0] + G[1] * ug + G[2] * vg + G[3] * 0.5 * (ug * ug + vg * vg);
    const double bug = G[1] * q[0] + G[3] * q[0] * ug;
    const double bvg = G[2] * q[0] + G[3] * q[0] * vg;
    const double g1 = a.gas.g1;
    gb -= G[3] * q[3] * g1 * g1;
    double bu, bv;
    if (wall == 0) {  // (ug, vg) = (I - 2 n n^T)(u, v): symmetric
      const double bn = bug * nx + bvg * ny;
      bu = bug - 2.0 * bn * nx;
      bv = bvg - 2.0 * bn * ny;
    } else {
      bu = -bug;
      bv = -bvg;
    }
    qIb[4 * k] = br;
    qIb[4 * k + 1] = bu;
    qIb[4 * k + 2] = bv;
    qIb[4 * k + 3] = G[3] * g1;
  }
}

__device__ __forceinline__ void adj_ib_src_one(const AdjArgs& a, const IbTArgs& tb, const double* qIb, int s,
                                               double& gb) {
  if (s < tb.nsrc) {
    double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int e = tb.ptr[s]; e < tb.ptr[s + 1]; ++e) {
      const int k = tb.ghost[e];
      const double w = tb.w[e];
#pragma unroll
      for (int c = 0; c < 4; ++c) S[c] += w * qIb[4 * k + c];
    }
    const Lay& L = a.lay;
    const long long id = tb.cell[s];
    // the fill used IEEE-rounded primitives; their derivative is the same map
    double ub[4];
    prim_vjp(a.X[id], a.X[L.plane + id], a.X[2 * L.plane + id], a.X[3 * L.plane + id], a.gas, S, ub, gb);
#pragma unroll
    for (int c = 0; c < 4; ++c) a.Ub[c * L.plane + id] += ub[c];
  }
}

// =======================================================================================
// small elementwise helpers
// =======================================================================================
__device__ __forceinline__ void adj_unpack_add_one(const double* __restrict__ P, const double* __restrict__ P2,
                                                   double* __restrict__ U, const Lay& lay, long long t) {
  const long long n = (long long)lay.nx * lay.ny;
  if (t >= 4 * n) return;
  const int c = (int)(t / n);
  const long long o = t % n;
  const int i = (int)(o % lay.nx), j = (int)(o / lay.nx);
  const long long id = c * lay.plane + lay.idx(i, j);
  U[t] = P2 ? P[id] + P2[id] : P[id];
}

}  // namespace js
