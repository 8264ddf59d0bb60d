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
//             Fbar = (lambda'_right - lambda'_left)/h; face-state adjoints saved, viscous and
//             positivity-fallback adjoints added to Qbar
//   pass 2    per line: WENO5 reverse from the saved internals; a 5-cell register window
//             accumulates Qbar along the line
//   primvjp   Ubar(X) += (dprim/dX)^T Qbar (+ nu * lap of lambda')
//   bcT       transposed halo fill (y sides, then x sides), written as gathers;
//             inflow halos accumulate into the inflow-state gradient
//   ibT       transposed immersed-boundary fill: ghost adjoint -> image-point adjoint ->
//             gathered onto the fluid source cells (CSR built on the host)
// Parameter gradients (gamma, mu, Pr, nu, inflow states) are accumulated in pbar.
#include <cuda_runtime.h>

#include "js_adjoint_device.cuh"
#include "js_internal.h"

namespace js {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// add a per-thread partial to pbar[k] (one atomic per warp)
__device__ __forceinline__ void pbar_add(double* pbar, int k, double v) {
  v = warp_sum(v);
  if (pbar && (threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(pbar + k, v);
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

}  // namespace

// =======================================================================================
// seed + prims
// =======================================================================================
__global__ void adj_seed_kernel(AdjArgs a, const double* __restrict__ Unext, double* __restrict__ Uacc, double ra,
                                double rb, double dt, int rhs_mode) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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
#pragma unroll
  for (int c = 0; c < 5; ++c) a.Qb[c * L.plane + t] = 0.0;
}

__global__ void adj_prims_kernel(AdjArgs a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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
__device__ __forceinline__ void pass1_body(const AdjArgs& a, int seg_len, long long item) {
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
        if (fallback) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            atomicAdd(a.Qb + c * L.plane + ca, bql[c]);
            atomicAdd(a.Qb + c * L.plane + cb, bqr[c]);
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
          double* bun = a.Qb + PN * L.plane;
          double* but = a.Qb + PT * L.plane;
          double* bT = a.Qb + 4 * L.plane;
          atomicAdd(bun + ca, bsbn - bdun);
          atomicAdd(bun + cb, bsbn + bdun);
          atomicAdd(but + ca, bsbt - bdut);
          atomicAdd(but + cb, bsbt + bdut);
          atomicAdd(bT + ca, -bdT);
          atomicAdd(bT + cb, bdT);
          if (HAS_T) {
            const double bsun = vc.ct * btnt, bsut = -vc.c23t * btnn;
            atomicAdd(bun + ca + ts, bsun);
            atomicAdd(bun + ca - ts, -bsun);
            atomicAdd(bun + cb + ts, bsun);
            atomicAdd(bun + cb - ts, -bsun);
            atomicAdd(but + ca + ts, bsut);
            atomicAdd(but + ca - ts, -bsut);
            atomicAdd(but + cb + ts, bsut);
            atomicAdd(but + cb - ts, -bsut);
          }
          const double ckck = bck * vc.ck;
          mub += a.inv_mu * fma(btnn, tnn, fma(btnt, tnt, ckck));
          gb += a.kg * ckck;
          prb += a.kp * ckck;
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) prevL[c] = Lf[c];
    }
  }
  pbar_add(a.pbar, 0, gb);
  if (VISC) {
    pbar_add(a.pbar, 1, mub);
    pbar_add(a.pbar, 2, prb);
  }
}

// x lines in blocks [0, bx), y lines (2D) in the blocks after them: one launch, both directions
template <bool VISC, bool HAS_T, bool SAVED>
__global__ void __launch_bounds__(64) adj_pass1_kernel(AdjArgs a, int seg_len, int bx) {
  if ((int)blockIdx.x < bx)
    pass1_body<0, VISC, HAS_T, SAVED>(a, seg_len, (long long)blockIdx.x * blockDim.x + threadIdx.x);
  else
    pass1_body<1, VISC, HAS_T, SAVED>(a, seg_len, (long long)(blockIdx.x - bx) * blockDim.x + threadIdx.x);
}

// =======================================================================================
// pass 2: WENO reverse from the saved internals, accumulated along the line
// =======================================================================================
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
    double* qb = a.Qb + c * L.plane;
    long long ci = cell_id(c0);
    const long long sst = (DIR == 0) ? a.tpitch : L.pitch;  // stride along the line in saved arrays
    long long si = save_id<DIR>(a, c0, line);
    WenoRev w;
    w.init(q[ci - 2 * st], q[ci - st], q[ci], q[ci + st]);
#pragma unroll 1
    for (int i = c0; i < c1; ++i, ci += st, si += sst) {
      double sv[WENO_SAVE];
#pragma unroll
      for (int k = 0; k < WENO_SAVE; ++k) sv[k] = a.wsave[(long long)(wdir + c * WENO_SAVE + k) * a.splane + si];
      const double Lb = a.fadj[(long long)(fdir + c) * a.splane + si + sst];  // left state of face i+1/2
      const double Rb = a.fadj[(long long)(fdir + 4 + c) * a.splane + si];    // right state of face i-1/2
      // cell i-2 is complete
      atomicAdd(qb + ci - 2 * st, w.step(q[ci + 2 * st], sv, Lb, Rb));
    }
    // flush cells c1-2 .. c1+1
    double rest[4];
    w.flush(rest);
    for (int k = 0; k < 4; ++k) atomicAdd(qb + ci + (k - 2) * st, rest[k]);
  }
}

__global__ void __launch_bounds__(64) adj_pass2_kernel(AdjArgs a, int seg_len, int bx) {
  if ((int)blockIdx.x < bx)
    pass2_body<0>(a, seg_len, (long long)blockIdx.x * blockDim.x + threadIdx.x);
  else
    pass2_body<1>(a, seg_len, (long long)(blockIdx.x - bx) * blockDim.x + threadIdx.x);
}

// =======================================================================================
// prim reverse (+ artificial viscosity)
// =======================================================================================
__global__ void adj_primvjp_kernel(AdjArgs a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const Lay& L = a.lay;
  double gb = 0.0, nb = 0.0;
  int i = 0, j = 0;
  if (t < L.plane && valid_padded(L, t, i, j)) {
    double qb[5], ub[4];
#pragma unroll
    for (int c = 0; c < 5; ++c) qb[c] = a.Qb[c * L.plane + t];
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
  pbar_add(a.pbar, 0, gb);
  if (a.has_av) pbar_add(a.pbar, 3, nb);
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

__global__ void adj_bcT_kernel(AdjArgs a, BcArgs bc, int phase_y, double* inflow_acc) {
  const Lay& L = a.lay;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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
  // inflow sides: sum the halo adjoints of each inflow side
  const long long nh = 6LL * ntan;
  if (t < nh) {
    const int r = (int)(t % 6);
    const int tan = (int)(t / 6) - (phase_y ? 3 : 0);
    const int s = (r < 3) ? 0 : 1;
    const int k = (r < 3) ? r + 1 : r - 2;
    const int side = (phase_y ? 2 : 0) + s;
    if (bc.kind[side] == 3) {
      const int n = phase_y ? L.ny : L.nx;
      const int h = (s == 0) ? -k : n - 1 + k;
      const long long hid = phase_y ? L.idx(tan, h) : L.idx(h, tan);
#pragma unroll
      for (int c = 0; c < 4; ++c) atomicAdd(inflow_acc + 4 * side + c, a.Ub[c * L.plane + hid]);
    }
  }
}

// inflow halo adjoints (conserved) -> gradient of the inflow primitive state and gamma
__global__ void adj_inflow_kernel(AdjArgs a, BcArgs bc, const double* inflow_acc, const double* inflow_prim) {
  const int side = threadIdx.x;
  if (side >= 4 || bc.kind[side] != 3 || a.pbar == nullptr) return;
  const double* S = inflow_acc + 4 * side;
  const double r = inflow_prim[4 * side], u = inflow_prim[4 * side + 1], v = inflow_prim[4 * side + 2],
               p = inflow_prim[4 * side + 3];
  // U = (r, r u, r v, p/(gamma-1) + r (u^2 + v^2)/2)
  atomicAdd(a.pbar + 4 + 4 * side + 0, S[0] + S[1] * u + S[2] * v + S[3] * 0.5 * (u * u + v * v));
  atomicAdd(a.pbar + 4 + 4 * side + 1, S[1] * r + S[3] * r * u);
  atomicAdd(a.pbar + 4 + 4 * side + 2, S[2] * r + S[3] * r * v);
  atomicAdd(a.pbar + 4 + 4 * side + 3, S[3] * a.gas.g1);
  atomicAdd(a.pbar + 0, -S[3] * p * a.gas.g1 * a.gas.g1);
}

// =======================================================================================
// transposed immersed-boundary fill
// =======================================================================================
__global__ void adj_ib_ghost_kernel(AdjArgs a, IbArgs ib, int wall, double* qIb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double gb = 0.0;
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
  pbar_add(a.pbar, 0, gb);
}

__global__ void adj_ib_src_kernel(AdjArgs a, IbTArgs tb, const double* qIb) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double gb = 0.0;
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
  pbar_add(a.pbar, 0, gb);
}

// =======================================================================================
// small elementwise helpers
// =======================================================================================
__global__ void adj_unpack_add_kernel(const double* __restrict__ P, const double* __restrict__ P2,
                                      double* __restrict__ U, Lay lay) {
  const long long n = (long long)lay.nx * lay.ny;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * n) return;
  const int c = (int)(t / n);
  const long long o = t % n;
  const int i = (int)(o % lay.nx), j = (int)(o / lay.nx);
  const long long id = c * lay.plane + lay.idx(i, j);
  U[t] = P2 ? P[id] + P2[id] : P[id];
}

// =======================================================================================
// launchers
// =======================================================================================
namespace {
// short segments and small blocks: enough blocks to fill every SM (one line per thread
// would leave most of the GPU idle); pass 1 pays one extra WENO cell per segment, except
// when the forward stored the internals: then a segment costs almost nothing to start and
// shorter ones split the work into finer waves
constexpr int kSeg1 = 16, kSeg1Saved = 8, kSeg2 = 8, kSeg1D = 4, kBlk = 64;

unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

long long line_items(const AdjArgs& a, int dir, int extra, int seg) {
  const int nline = (dir == 0) ? a.lay.ny : a.lay.nx;
  const int ncell = (dir == 0) ? a.lay.nx : a.lay.ny;
  return (long long)nline * ((ncell + extra + seg - 1) / seg);
}

cudaError_t pass1(const AdjArgs& a, bool visc, bool two_d, cudaStream_t s) {
  if (a.weno_saved) {
    if (!two_d) return cudaErrorInvalidValue;  // the forward saves exist for 2D grids only
    const int sx = (int)blocks_for(line_items(a, 0, 1, kSeg1Saved), kBlk);
    const int sy = (int)blocks_for(line_items(a, 1, 1, kSeg1Saved), kBlk);
    if (visc) adj_pass1_kernel<true, true, true><<<sx + sy, kBlk, 0, s>>>(a, kSeg1Saved, sx);
    else adj_pass1_kernel<false, false, true><<<sx + sy, kBlk, 0, s>>>(a, kSeg1Saved, sx);
    return cudaGetLastError();
  }
  // a 1D grid is one line: short segments give it more threads
  const int seg = two_d ? kSeg1 : kSeg1D;
  const int bx = (int)blocks_for(line_items(a, 0, 1, seg), kBlk);
  const int by = two_d ? (int)blocks_for(line_items(a, 1, 1, seg), kBlk) : 0;
  if (visc) {
    if (two_d) adj_pass1_kernel<true, true, false><<<bx + by, kBlk, 0, s>>>(a, seg, bx);
    else adj_pass1_kernel<true, false, false><<<bx + by, kBlk, 0, s>>>(a, seg, bx);
  } else {
    adj_pass1_kernel<false, false, false><<<bx + by, kBlk, 0, s>>>(a, seg, bx);
  }
  return cudaGetLastError();
}

cudaError_t pass2(const AdjArgs& a, bool two_d, cudaStream_t s) {
  const int seg = two_d ? kSeg2 : kSeg1D;
  const int bx = (int)blocks_for(line_items(a, 0, 2, seg), kBlk);
  const int by = two_d ? (int)blocks_for(line_items(a, 1, 2, seg), kBlk) : 0;
  adj_pass2_kernel<<<bx + by, kBlk, 0, s>>>(a, seg, bx);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_adj_stage(const AdjArgs& a, const BcArgs& bc, const IbArgs& ib, const IbTArgs& ibt, int wall,
                             const double* Unext, double* Uacc, double ra, double rb, double dt, bool rhs_mode,
                             double* inflow_acc, const double* inflow_prim, double* qIb, cudaStream_t s,
                             long long* launches, const NnArgs* nn) {
  const Lay& L = a.lay;
  const unsigned gp = blocks_for(L.plane, 256);
  long long n = 0;
  adj_seed_kernel<<<gp, 256, 0, s>>>(a, Unext, Uacc, ra, rb, dt, rhs_mode ? 1 : 0);
  adj_prims_kernel<<<gp, 256, 0, s>>>(a);
  n += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool two_d = L.ny > 1;
  if ((e = pass1(a, a.visc != 0, two_d, s)) != cudaSuccess) return e;
  if (nn) {
    // the neural flux: its face-state adjoints join the HLLC ones before the WENO5 reverse
    if ((e = nn_reverse(*nn, a, s)) != cudaSuccess) return e;
    n += nn->w_bar ? 13 : 9;
  }
  if ((e = pass2(a, two_d, s)) != cudaSuccess) return e;
  n += 2;
  adj_primvjp_kernel<<<gp, 256, 0, s>>>(a);
  ++n;
  cudaMemsetAsync(inflow_acc, 0, 16 * sizeof(double), s);
  if (two_d) {
    adj_bcT_kernel<<<blocks_for(6LL * (L.nx + 6), 128), 128, 0, s>>>(a, bc, 1, inflow_acc);
    ++n;
  }
  adj_bcT_kernel<<<blocks_for(6LL * L.ny, 128), 128, 0, s>>>(a, bc, 0, inflow_acc);
  adj_inflow_kernel<<<1, 32, 0, s>>>(a, bc, inflow_acc, inflow_prim);
  n += 2;
  if (ib.n > 0) {
    adj_ib_ghost_kernel<<<blocks_for(ib.n, 128), 128, 0, s>>>(a, ib, wall, qIb);
    adj_ib_src_kernel<<<blocks_for(ibt.nsrc, 128), 128, 0, s>>>(a, ibt, qIb);
    n += 2;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}

cudaError_t launch_adj_unpack(const double* P, const double* P2, double* U, const Lay& lay, cudaStream_t s) {
  adj_unpack_add_kernel<<<blocks_for(4LL * lay.nx * lay.ny, 256), 256, 0, s>>>(P, P2, U, lay);
  return cudaGetLastError();
}

}  // namespace js
