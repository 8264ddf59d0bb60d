// IEEE-order arithmetic mode of the forward step (js_set_arith(ctx, JS_ARITH_IEEE)).
//
// The same finite-volume right-hand side and SSP-RK3 stage as the fused stage kernel
// (Sec. 2: WENO5 reconstruction of the primitive variables, HLLC flux with the positivity
// fallback, viscous and heat fluxes, flux divergence, Laplacian artificial viscosity), but
// every operation is one IEEE-rounded double operation (this file is compiled with
// -fmad=false: no fused multiply-add; division and square root are the correctly rounded
// ones) in one fixed expression order per formula, the canonical order below.  Every face and
// cell is computed independently of the others, so the result does not depend on the launch
// shape: any implementation that follows the same order on IEEE doubles gets the same bits.
//
// Canonical order (a . b = one rounded product, left-to-right sums as parenthesised):
//   EOS        E = p/(g-1) + (0.5 r)(u u + v v);  p = (g-1)(E - (0.5 r)(u u + v v));
//              u = (r u)/r, v = (r v)/r
//   WENO5      at the right edge of cell c from (a, b, c, d, e) = cells c-2 .. c+2; the left
//              edge value of cell c is the same formula on (e, d, c, b, a) of its mirror:
//              s0 = (a - 2b) + c, t0 = (a - 4b) + 3c, s1 = (b - 2c) + d, t1 = b - d,
//              s2 = (c - 2d) + e, t2 = (3c - 4d) + e,
//              beta_k = ((13/12) s_k) s_k + (0.25 t_k) t_k,
//              p0 = ((2a - 7b) + 11c)/6, p1 = ((-b + 5c) + 2d)/6, p2 = ((2c + 5d) - e)/6,
//              alpha_k = d_k / ((1e-6 + beta_k)(1e-6 + beta_k)), d = (0.1, 0.6, 0.3),
//              w_k = alpha_k / ((alpha_0 + alpha_1) + alpha_2),
//              value = (w0 p0 + w1 p1) + w2 p2
//   fallback   if a reconstructed rho or p of either side is not > 0, both sides take the
//              adjacent cell states
//   HLLC       a = sqrt((g p)/r); sL = min(uL - aL, uR - aR), sR = max(uL + aL, uR + aR)
//              (ties keep the left argument); s- = min(0, sL), s+ = max(0, sR) (ties keep 0);
//              s* = (((pR - pL) + (rL uL)(sL - uL)) - (rR uR)(sR - uR))
//                   / (rL (sL - uL) - rR (sR - uR));
//              side k: U = (r, r u, r v, E), F = (r u, (r u) u + p, (r u) v, u (E + p)),
//              f = (s_k - u)/(s_k - s*),
//              U* = (f r, f (r s*), f (r v), f (E + (s* - u)((r s*) + p/(s_k - u))));
//              flux = F_L + s-(U*L - U_L) if s* > 0, F_R + s+(U*R - U_R) if s* < 0, else
//              0.5 (F_L + s-(U*L - U_L)) + 0.5 (F_R + s+(U*R - U_R))
//   viscous    (mu != 0) with h_n, h_t the spacings normal to and along the face:
//              un_n = (un_R - un_L)/h_n, ut_n = (ut_R - ut_L)/h_n, T = p/r,
//              T_n = (T_R - T_L)/h_n, un_t = ((un_L+ - un_L-) + (un_R+ - un_R-))/(4 h_t)
//              (likewise ut_t; both 0 on a 1D grid),
//              tau_nn = mu((4/3) un_n - (2/3) ut_t), tau_nt = mu(ut_n + un_t),
//              kappa = (mu g)/((g - 1) Pr), F_n -= tau_nn, F_t -= tau_nt,
//              F_E -= ((ubar_n tau_nn + ubar_t tau_nt) + kappa T_n), ubar = 0.5 (L + R)
//   RHS        L = (-(F_i+1/2 - F_i-1/2))/dx - (G_j+1/2 - G_j-1/2)/dy
//              [+ nu lap, lap = ((U_E - 2U) + U_W)/(dx dx) + ((U_N - 2U) + U_S)/(dy dy)]
//   stage      X + dt L (stage 0), a U^n + b (X + dt L) (stages 1, 2); non-fluid cells keep X
//   IB ghost   q = sum over the 4 weights w != 0, in order, of q + w q_m; slip:
//              vn = q_u n_x + q_v n_y, u_g = q_u - (2 vn) n_x, v_g = q_v - (2 vn) n_y
#include <cuda_runtime.h>
#include <math_constants.h>

#include "js_device.cuh"
#include "js_internal.h"

namespace js {
namespace {

__device__ __forceinline__ double eos_energy(double r, double u, double v, double p, double gamma) {
  return p / (gamma - 1.0) + (0.5 * r) * (u * u + v * v);
}
__device__ __forceinline__ double eos_pressure(double r, double u, double v, double E, double gamma) {
  return (gamma - 1.0) * (E - (0.5 * r) * (u * u + v * v));
}

// WENO5 value at the right edge of the centre cell of (a, b, c, d, e)
__device__ __forceinline__ double weno5_ieee(double a, double b, double c, double d, double e) {
  const double k13 = 13.0 / 12.0;
  const double s0 = (a - 2.0 * b) + c, t0 = (a - 4.0 * b) + 3.0 * c;
  const double s1 = (b - 2.0 * c) + d, t1 = b - d;
  const double s2 = (c - 2.0 * d) + e, t2 = (3.0 * c - 4.0 * d) + e;
  const double b0 = (k13 * s0) * s0 + (0.25 * t0) * t0;
  const double b1 = (k13 * s1) * s1 + (0.25 * t1) * t1;
  const double b2 = (k13 * s2) * s2 + (0.25 * t2) * t2;
  const double p0 = ((2.0 * a - 7.0 * b) + 11.0 * c) / 6.0;
  const double p1 = ((-b + 5.0 * c) + 2.0 * d) / 6.0;
  const double p2 = ((2.0 * c + 5.0 * d) - e) / 6.0;
  const double e0 = 1e-6 + b0, e1 = 1e-6 + b1, e2 = 1e-6 + b2;
  const double a0 = 0.1 / (e0 * e0), a1 = 0.6 / (e1 * e1), a2 = 0.3 / (e2 * e2);
  const double sum = (a0 + a1) + a2;
  const double w0 = a0 / sum, w1 = a1 / sum, w2 = a2 / sum;
  return (w0 * p0 + w1 * p1) + w2 * p2;
}

__device__ __forceinline__ double min_keep_first(double a, double b) { return (b < a) ? b : a; }
__device__ __forceinline__ double max_keep_first(double a, double b) { return (a < b) ? b : a; }

// conserved state, physical flux and star state of one side of the HLLC fan
__device__ __forceinline__ void hllc_side_ieee(double r, double u, double v, double p, double E, double s, double ss,
                                               double Uk[4], double Fk[4], double Us[4]) {
  Uk[0] = r;
  Uk[1] = r * u;
  Uk[2] = r * v;
  Uk[3] = E;
  Fk[0] = r * u;
  Fk[1] = (r * u) * u + p;
  Fk[2] = (r * u) * v;
  Fk[3] = u * (E + p);
  const double f = (s - u) / (s - ss);
  Us[0] = f * r;
  Us[1] = f * (r * ss);
  Us[2] = f * (r * v);
  Us[3] = f * (E + (ss - u) * ((r * ss) + p / (s - u)));
}

// HLLC flux of the face-normal frame (rho, normal velocity, tangential velocity, p)
__device__ __forceinline__ void hllc_ieee(const double qL[4], const double qR[4], double gamma, double F[4]) {
  const double rL = qL[0], uL = qL[1], vL = qL[2], pL = qL[3];
  const double rR = qR[0], uR = qR[1], vR = qR[2], pR = qR[3];
  const double EL = eos_energy(rL, uL, vL, pL, gamma), ER = eos_energy(rR, uR, vR, pR, gamma);
  const double aL = sqrt((gamma * pL) / rL), aR = sqrt((gamma * pR) / rR);
  const double sL = min_keep_first(uL - aL, uR - aR);
  const double sR = max_keep_first(uL + aL, uR + aR);
  const double sm = min_keep_first(0.0, sL);
  const double sp = max_keep_first(0.0, sR);
  const double ss = (((pR - pL) + (rL * uL) * (sL - uL)) - (rR * uR) * (sR - uR)) /
                    (rL * (sL - uL) - rR * (sR - uR));
  double UkL[4], FkL[4], UsL[4], UkR[4], FkR[4], UsR[4];
  if (!(ss < 0.0)) hllc_side_ieee(rL, uL, vL, pL, EL, sL, ss, UkL, FkL, UsL);
  if (!(ss > 0.0)) hllc_side_ieee(rR, uR, vR, pR, ER, sR, ss, UkR, FkR, UsR);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (ss > 0.0)
      F[c] = FkL[c] + sm * (UsL[c] - UkL[c]);
    else if (ss < 0.0)
      F[c] = FkR[c] + sp * (UsR[c] - UkR[c]);
    else
      F[c] = 0.5 * (FkL[c] + sm * (UsL[c] - UkL[c])) + 0.5 * (FkR[c] + sp * (UsR[c] - UkR[c]));
  }
}

struct IeeeArgs {
  Lay lay;
  const double* Q;           // padded primitives rho, u, v, p (4 planes of lay.plane)
  double* F;                 // x-face fluxes [4][ny][nx + 1]
  double* G;                 // y-face fluxes [4][ny + 1][nx]
  double gamma, mu, Pr, dx, dy;
  int two_d, visc;
};

// numerical + viscous flux through the face between padded cells il (low side) and ir;
// dir 0: x face (stride 1, tangential stride = pitch), dir 1: y face (stride pitch, 1)
template <int DIR>
__device__ __forceinline__ void face_flux_ieee(const IeeeArgs& a, long long il, long long ir, double out[4]) {
  const long long st = DIR == 0 ? 1 : a.lay.pitch;
  const long long ts = DIR == 0 ? a.lay.pitch : 1;
  const long long P = a.lay.plane;
  const double* Q = a.Q;
  double qL[4], qR[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double* q = Q + c * P;
    qL[c] = weno5_ieee(q[il - 2 * st], q[il - st], q[il], q[il + st], q[il + 2 * st]);
    qR[c] = weno5_ieee(q[ir + 2 * st], q[ir + st], q[ir], q[ir - st], q[ir - 2 * st]);
  }
  if (!(qL[0] > 0.0) || !(qL[3] > 0.0) || !(qR[0] > 0.0) || !(qR[3] > 0.0)) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      qL[c] = Q[c * P + il];
      qR[c] = Q[c * P + ir];
    }
  }
  constexpr int n = DIR == 0 ? 1 : 2, t = DIR == 0 ? 2 : 1;
  const double fl[4] = {qL[0], qL[n], qL[t], qL[3]}, fr[4] = {qR[0], qR[n], qR[t], qR[3]};
  double F[4];
  hllc_ieee(fl, fr, a.gamma, F);
  out[0] = F[0];
  out[n] = F[1];
  out[t] = F[2];
  out[3] = F[3];
  if (!a.visc) return;
  const double hn = DIR == 0 ? a.dx : a.dy, ht = DIR == 0 ? a.dy : a.dx;
  const double* Qn = Q + n * P;
  const double* Qt = Q + t * P;
  const double un_n = (Qn[ir] - Qn[il]) / hn;
  const double ut_n = (Qt[ir] - Qt[il]) / hn;
  const double TL = Q[3 * P + il] / Q[il], TR = Q[3 * P + ir] / Q[ir];
  const double T_n = (TR - TL) / hn;
  double un_t = 0.0, ut_t = 0.0;
  if (a.two_d) {
    un_t = ((Qn[il + ts] - Qn[il - ts]) + (Qn[ir + ts] - Qn[ir - ts])) / (4.0 * ht);
    ut_t = ((Qt[il + ts] - Qt[il - ts]) + (Qt[ir + ts] - Qt[ir - ts])) / (4.0 * ht);
  }
  const double tau_nn = a.mu * ((4.0 / 3.0) * un_n - (2.0 / 3.0) * ut_t);
  const double tau_nt = a.mu * (ut_n + un_t);
  const double unb = 0.5 * (Qn[il] + Qn[ir]);
  const double utb = 0.5 * (Qt[il] + Qt[ir]);
  const double kappa = (a.mu * a.gamma) / ((a.gamma - 1.0) * a.Pr);
  out[n] = out[n] - tau_nn;
  out[t] = out[t] - tau_nt;
  out[3] = out[3] - ((unb * tau_nn + utb * tau_nt) + kappa * T_n);
}

// primitives of every padded cell (halo included); a fluid cell whose density or pressure is
// not positive, or not finite, sets the error flag
__global__ void ieee_prims_kernel(const double* __restrict__ X, double* __restrict__ Q, Lay lay,
                                  const unsigned char* __restrict__ tag, double gamma, int* err) {
  const int W = lay.nx + 6;
  const long long n = (long long)W * lay.H;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int col = (int)(t % W), row = (int)(t / W);
  const long long id = (long long)row * lay.pitch + col;
  const double r = X[id];
  const double u = X[lay.plane + id] / r, v = X[2 * lay.plane + id] / r;
  const double p = eos_pressure(r, u, v, X[3 * lay.plane + id], gamma);
  Q[id] = r;
  Q[lay.plane + id] = u;
  Q[2 * lay.plane + id] = v;
  Q[3 * lay.plane + id] = p;
  const int i = col - 3, j = row - lay.gy;
  if (i >= 0 && i < lay.nx && j >= 0 && j < lay.ny && !(tag && tag[(long long)j * lay.nx + i] != 0)) {
    if (!(r > 0.0) || !(p > 0.0) || !(r < CUDART_INF) || !(p < CUDART_INF))
      atomicOr(err, ERR_NONPHYSICAL_BIT);
  }
}

__global__ void ieee_flux_x_kernel(IeeeArgs a) {
  const int nf = a.lay.nx + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nf * a.lay.ny) return;
  const int f = (int)(t % nf), j = (int)(t / nf);
  double out[4];
  face_flux_ieee<0>(a, a.lay.idx(f - 1, j), a.lay.idx(f, j), out);
  const long long m = (long long)nf * a.lay.ny;
#pragma unroll
  for (int c = 0; c < 4; ++c) a.F[c * m + t] = out[c];
}

__global__ void ieee_flux_y_kernel(IeeeArgs a) {
  const int nx = a.lay.nx;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nx * (a.lay.ny + 1)) return;
  const int i = (int)(t % nx), f = (int)(t / nx);
  double out[4];
  face_flux_ieee<1>(a, a.lay.idx(i, f - 1), a.lay.idx(i, f), out);
  const long long m = (long long)nx * (a.lay.ny + 1);
#pragma unroll
  for (int c = 0; c < 4; ++c) a.G[c * m + t] = out[c];
}

struct CombineArgs {
  Lay lay;
  const double* X;           // padded filled stage input
  const double* Un;          // padded U^n (stages 1, 2) or nullptr
  double* out;               // padded stage output, or [4][ny][nx] in RHS mode
  const double* F;
  const double* G;
  const unsigned char* tag;
  double dx, dy, nu, dt, ra, rb;
  int two_d, av, rhs, stage;
  const double* dtc;         // device step size (dtc[5]) and activity (dtc[4]), or nullptr
};

__global__ void ieee_combine_kernel(CombineArgs a) {
  const int nx = a.lay.nx, ny = a.lay.ny;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nx * ny) return;
  if (a.dtc) {
    if (a.dtc[4] == 0.0) return;
    a.dt = a.dtc[5];
  }
  const int i = (int)(t % nx), j = (int)(t / nx);
  const long long id = a.lay.idx(i, j);
  const long long P = a.lay.plane, n = (long long)nx * ny;
  const long long mF = (long long)(nx + 1) * ny, mG = (long long)nx * (ny + 1);
  const bool fluid = !(a.tag && a.tag[t] != 0);
  const long long W = a.lay.pitch;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double* X = a.X + c * P;
    if (!fluid) {
      if (a.rhs)
        a.out[c * n + t] = 0.0;
      else
        a.out[c * P + id] = X[id];
      continue;
    }
    const double* Fc = a.F + c * mF + (long long)j * (nx + 1);
    double L = (-(Fc[i + 1] - Fc[i])) / a.dx;
    if (a.two_d) {
      const double* Gc = a.G + c * mG;
      L = L - (Gc[(long long)(j + 1) * nx + i] - Gc[(long long)j * nx + i]) / a.dy;
    }
    if (a.av) {
      double lap = ((X[id + 1] - 2.0 * X[id]) + X[id - 1]) / (a.dx * a.dx);
      if (a.two_d) lap = lap + ((X[id + W] - 2.0 * X[id]) + X[id - W]) / (a.dy * a.dy);
      L = L + a.nu * lap;
    }
    if (a.rhs) {
      a.out[c * n + t] = L;
      continue;
    }
    const double adv = X[id] + a.dt * L;
    a.out[c * P + id] = (a.stage == 0) ? adv : a.ra * a.Un[c * P + id] + a.rb * adv;
  }
}

// immersed-boundary ghost cell k in the canonical order (weights of non-fluid cells are 0
// and skipped, so the ghosts read fluid cells only and their order does not matter)
__global__ void ieee_ib_fill_kernel(double* __restrict__ U, Lay lay, IbArgs ib, double gamma, int wall) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ib.n) return;
  const long long P = lay.plane;
  double q[4] = {0.0, 0.0, 0.0, 0.0};
  for (int m = 0; m < 4; ++m) {
    const double w = ib.w[4 * k + m];
    if (w == 0.0) continue;
    const long long s = ib.src[4 * k + m];
    const double r = U[s], u = U[P + s] / r, v = U[2 * P + s] / r;
    const double p = eos_pressure(r, u, v, U[3 * P + s], gamma);
    q[0] = q[0] + w * r;
    q[1] = q[1] + w * u;
    q[2] = q[2] + w * v;
    q[3] = q[3] + w * p;
  }
  const double nx = ib.nrm[2 * k], ny = ib.nrm[2 * k + 1];
  double ug, vg;
  if (wall == 0) {
    const double vn = q[1] * nx + q[2] * ny;
    ug = q[1] - (2.0 * vn) * nx;
    vg = q[2] - (2.0 * vn) * ny;
  } else {
    ug = -q[1];
    vg = -q[2];
  }
  const long long d = ib.dst[k];
  U[d] = q[0];
  U[P + d] = q[0] * ug;
  U[2 * P + d] = q[0] * vg;
  U[3 * P + d] = eos_energy(q[0], ug, vg, q[3], gamma);
}

unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_ieee_ib_fill(double* U, const Lay& lay, const IbArgs& ib, double gamma, int wall,
                                cudaStream_t s) {
  if (ib.n == 0) return cudaSuccess;
  ieee_ib_fill_kernel<<<blocks_for(ib.n, 128), 128, 0, s>>>(U, lay, ib, gamma, wall);
  return cudaGetLastError();
}

cudaError_t launch_ieee_stage(const StageArgs& a, const IeeeBufs& b, double dt, int stage, bool rhs,
                              double mu, double Pr, double nu, double dx, double dy, cudaStream_t s) {
  const Lay& lay = a.lay;
  const int bs = 128;
  ieee_prims_kernel<<<blocks_for((long long)(lay.nx + 6) * lay.H, 256), 256, 0, s>>>(a.Uin, b.Q, lay, a.tag,
                                                                                     a.gamma, a.err);
  IeeeArgs f;
  f.lay = lay;
  f.Q = b.Q;
  f.F = b.F;
  f.G = b.G;
  f.gamma = a.gamma;
  f.mu = mu;
  f.Pr = Pr;
  f.dx = dx;
  f.dy = dy;
  f.two_d = lay.ny > 1 ? 1 : 0;
  f.visc = mu != 0.0 ? 1 : 0;
  ieee_flux_x_kernel<<<blocks_for((long long)(lay.nx + 1) * lay.ny, bs), bs, 0, s>>>(f);
  if (lay.ny > 1) ieee_flux_y_kernel<<<blocks_for((long long)lay.nx * (lay.ny + 1), bs), bs, 0, s>>>(f);
  CombineArgs c;
  c.lay = lay;
  c.X = a.Uin;
  c.Un = a.Un;
  c.out = a.Uout;
  c.F = b.F;
  c.G = b.G;
  c.tag = a.tag;
  c.dx = dx;
  c.dy = dy;
  c.nu = nu;
  c.dt = dt;
  c.ra = a.rk_a;
  c.rb = a.rk_b;
  c.two_d = lay.ny > 1 ? 1 : 0;
  c.av = nu != 0.0 ? 1 : 0;
  c.rhs = rhs ? 1 : 0;
  c.stage = stage;
  c.dtc = a.dtc;
  ieee_combine_kernel<<<blocks_for((long long)lay.nx * lay.ny, 256), 256, 0, s>>>(c);
  return cudaGetLastError();
}

}  // namespace js
