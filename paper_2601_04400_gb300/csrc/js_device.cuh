// Device building blocks of the FP64 finite-volume right-hand side (arXiv 2601.04400, Sec. 2).
//
// GB300 has a narrow FP64 pipe (about 1/64 of the FP32 rate) while integer, FP32, MUFU and
// min/max work issue on other units.  Everything here is therefore written to minimise
// FP64 add/mul/fma instructions:
//   * no IEEE division or square root: MUFU seeds (rcp.approx / rsqrt.approx) refined by
//     Newton steps and a residual correction, accurate to about one ulp;
//   * WENO5 is cell-centred: the smoothness indicators of a cell's three stencils are
//     computed once and shared by the state at its right face (left-biased weights) and
//     the state at its left face (right-biased weights); first and second differences are
//     carried along the line in registers;
//   * the nonlinear weights use the products of the other stencils' (eps + beta)^2 instead
//     of 1/(eps + beta)^2, so one division per face state remains;
//   * HLLC evaluates the star state of the upwind side only (selected with integer
//     selects), and the sound speed as gamma*p*rsqrt(gamma*p*rho).
#pragma once
#include <cstdint>

namespace js {

// ---------------------------------------------------------------------------------------
// padded SoA layout of the state: 4 planes [H][pitch], interior cell (i, j) at
// (j + gy) * pitch + i + 3; gy = 3 in 2D and 0 in 1D (ny == 1).
// ---------------------------------------------------------------------------------------
struct Lay {
  int nx, ny, gy, pitch, H;
  long long plane;
  __host__ __device__ long long idx(int i, int j) const { return (long long)(j + gy) * pitch + (i + 3); }
};

constexpr int ERR_NONPHYSICAL_BIT = 1;
constexpr int ERR_TIMEOUT_BIT = 2;

// ---------------------------------------------------------------------------------------
// FP64 reciprocal / quotient / reciprocal square root with few FP64-pipe instructions
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double rcp_seed(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rsqrt_seed(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
// The seeds are accurate to about 2^-20 (measured on GB300), so one cubic (Halley) step
// reaches full FP64 precision.
// 1/x: seed + one Halley step r (1 + e + e^2), e = 1 - x r (3 FP64 instructions)
__device__ __forceinline__ double recip(double x) {
  const double r = rcp_seed(x);
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
// a/b as a * (1/b) (4 FP64 instructions; within about 1.5 ulp)
__device__ __forceinline__ double quot(double a, double b) { return a * recip(b); }
// 1/sqrt(x): seed + one Halley step y (1 + e/2 + 3e^2/8), e = 1 - x y^2 (5 FP64 instructions)
__device__ __forceinline__ double rsqrt_nr(double x) {
  const double y = rsqrt_seed(x);
  const double e = fma(-x * y, y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}

// ---------------------------------------------------------------------------------------
// gas constants of one launch
// ---------------------------------------------------------------------------------------
struct Gas {
  double gamma, gm1, g1;  // gamma, gamma - 1, 1/(gamma - 1)
};

// primitive variables of a conserved state; returns T = p/rho as well
__device__ __forceinline__ void cons_to_prim(double r, double mx, double my, double E, const Gas& g,
                                             double& u, double& v, double& p, double& T) {
  const double ir = recip(r);
  u = mx * ir;
  v = my * ir;
  const double k2 = fma(mx, u, my * v);  // rho (u^2 + v^2)
  p = g.gm1 * fma(-0.5, k2, E);
  T = p * ir;
}

// ---------------------------------------------------------------------------------------
// WENO5 (Jiang-Shu, eps = 1e-6, power 2) on a line, cell-centred with a sliding window.
// For cell i with neighbours q_{i-2..i+2} (Sec. 2: reconstruction of primitive variables):
//   d_{i+1/2} = q_{i+1} - q_i,  D_i = q_{i-1} - 2 q_i + q_{i+1}
//   4 beta_0 = 13/3 D_{i-1}^2 + (D_{i-1} + 2 d_{i-1/2})^2
//   4 beta_1 = 13/3 D_i^2     + (d_{i-1/2} + d_{i+1/2})^2
//   4 beta_2 = 13/3 D_{i+1}^2 + (D_{i+1} - 2 d_{i+1/2})^2
// s_k = 4 beta_k + 4 eps; the weights alpha_k = d_k / s_k^2 are scaled by (s0 s1 s2)^2.
// Candidate values minus q_i, times 6, are two-term combinations of the d's.
// ---------------------------------------------------------------------------------------
constexpr double K13 = 13.0 / 3.0;
constexpr double EPS4 = 4.0e-6;
constexpr double SIXTH = 1.0 / 6.0;

// Network input of one face (neural flux, Sec. 2.3): the mean of its two WENO5 face states
// (primitive rho, u, v, p in wl / wr; un / ut the planes of the face-normal and tangential
// velocity) in conserved variables of the face frame, normalised by mean and 1/sd per channel,
// in arithmetic R: double for the FP64 network, float for the FP32 and BF16 networks (whose input
// is FP32: the face states are rounded to FP32 first, sparing the FP64 pipe).  One definition for
// every kernel that forms face images, so that they agree bit for bit.
template <class R>
__device__ __forceinline__ void face_image(const double wl[4], const double wr[4], int un, int ut, R g1,
                                           const R mean[4], const R inv_sd[4], R m[4]) {
  const R rL = (R)wl[0], rR = (R)wr[0], nL = (R)wl[un], nR = (R)wr[un], tL = (R)wl[ut], tR = (R)wr[ut];
  const R pL = (R)wl[3], pR = (R)wr[3], h = (R)0.5;
  const R EL = fma(h * rL, fma(nL, nL, tL * tL), pL * g1);
  const R ER = fma(h * rR, fma(nR, nR, tR * tR), pR * g1);
  m[0] = h * (rL + rR);
  m[1] = h * fma(rL, nL, rR * nR);
  m[2] = h * fma(rL, tL, rR * tR);
  m[3] = h * (EL + ER);
#pragma unroll
  for (int k = 0; k < 4; ++k) m[k] = (m[k] - mean[k]) * inv_sd[k];
}

struct Win {
  double q0, q1;          // q_i, q_{i+1}
  double dm2, dm1, dp1;   // d_{i-3/2}, d_{i-1/2}, d_{i+1/2}
  double D0, D1;          // D_{i-1}, D_i
  double cD0, cD1;        // 13/3 D
  double f5m1, f5p1;      // 5 d_{i-1/2}, 5 d_{i+1/2}

  // start at cell i from q_{i-2}, q_{i-1}, q_i, q_{i+1}
  __device__ __forceinline__ void init(double qm2, double qm1, double q, double qp1) {
    q0 = q;
    q1 = qp1;
    dm2 = qm1 - qm2;
    dm1 = q - qm1;
    dp1 = qp1 - q;
    D0 = dm1 - dm2;
    D1 = dp1 - dm1;
    cD0 = K13 * D0;
    cD1 = K13 * D1;
    f5m1 = 5.0 * dm1;
    f5p1 = 5.0 * dp1;
  }

  // given q_{i+2}: face states at i+1/2 (Lf, left-biased; if NL) and i-1/2 (Rf,
  // right-biased; if NR), then slide to cell i+1.  With SV the internals the reverse pass
  // needs go to sv[0..6] = s0, s1, s2, qL, rL, qR, rR (state = q_i + q/6, q = num r, r the
  // reciprocal of den; zeros for a side not formed).
  template <bool NL = true, bool NR = true, bool SV = false>
  __device__ __forceinline__ void step(double q2, double& Lf, double& Rf, double* sv = nullptr) {
    const double dp2 = q2 - q1;
    const double D2 = dp2 - dp1;
    const double cD2 = K13 * D2;
    const double t0 = fma(2.0, dm1, D0);
    const double t1 = dm1 + dp1;
    const double t2 = fma(-2.0, dp1, D2);
    const double s0 = fma(cD0, D0, fma(t0, t0, EPS4));
    const double s1 = fma(cD1, D1, fma(t1, t1, EPS4));
    const double s2 = fma(cD2, D2, fma(t2, t2, EPS4));
    const double p01 = s0 * s1, p02 = s0 * s2, p12 = s1 * s2;
    const double w0 = p12 * p12, w1 = p02 * p02, w2 = p01 * p01;  // proportional to 1/s_k^2
    const double w1_6 = 6.0 * w1;
    // left-biased (linear weights 0.1 : 0.6 : 0.3)
    if (NL) {
      const double w2_3 = 3.0 * w2;
      const double e0 = fma(-2.0, dm2, f5m1);   // 2q_{i-2} - 7q_{i-1} + 5q_i
      const double e1 = fma(2.0, dp1, dm1);     // -q_{i-1} - q_i + 2q_{i+1}
      const double e2 = fma(4.0, dp1, -dp2);    // -4q_i + 5q_{i+1} - q_{i+2}
      const double num = fma(w0, e0, fma(w1_6, e1, w2_3 * e2));
      const double den = w0 + w1_6 + w2_3;
      const double r = recip(den), q = num * r;  // = quot(num, den)
      Lf = fma(q, SIXTH, q0);
      if (SV) { sv[3] = q; sv[4] = r; }
    } else if (SV) {
      sv[3] = 0.0;
      sv[4] = 0.0;
    }
    // right-biased (linear weights 0.3 : 0.6 : 0.1)
    const double f5p2 = 5.0 * dp2;
    if (NR) {
      const double w0_3 = 3.0 * w0;
      const double e0 = fma(-4.0, dm1, dm2);    // -q_{i-2} + 5q_{i-1} - 4q_i
      const double e1 = fma(-2.0, dm1, -dp1);   // 2q_{i-1} - q_i - q_{i+1}
      const double e2 = fma(2.0, dp2, -f5p1);   // 5q_i - 7q_{i+1} + 2q_{i+2}
      const double num = fma(w0_3, e0, fma(w1_6, e1, w2 * e2));
      const double den = w0_3 + w1_6 + w2;
      const double r = recip(den), q = num * r;  // = quot(num, den)
      Rf = fma(q, SIXTH, q0);
      if (SV) { sv[5] = q; sv[6] = r; }
    } else if (SV) {
      sv[5] = 0.0;
      sv[6] = 0.0;
    }
    if (SV) { sv[0] = s0; sv[1] = s1; sv[2] = s2; }
    // slide
    q0 = q1;
    q1 = q2;
    dm2 = dm1;
    dm1 = dp1;
    dp1 = dp2;
    D0 = D1;
    D1 = D2;
    cD0 = cD1;
    cD1 = cD2;
    f5m1 = f5p1;
    f5p1 = f5p2;
  }
};

// ---------------------------------------------------------------------------------------
// HLLC (Sec. 2) in the face-normal frame.  State (rho, un, ut, p) on each side; returns
// [mass, normal momentum, tangential momentum, energy].  Star-state energy in the
// standard (Toro) form; sign(s*) = 0 averages both branches.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void hllc_branch(double r, double un, double ut, double p, double s, double d,
                                            double m, double spm, double ss, const Gas& g, double F[4]) {
  // d = s - un, m = rho (s - un)
  const double ke = fma(un, un, ut * ut);
  const double E = fma(0.5 * r, ke, p * g.g1);
  const double inv = recip(s - ss);
  const double rs = m * inv;               // rho* = rho (s - u)/(s - s*)
  const double fac = d * inv;              // (s - u)/(s - s*)
  const double Us1 = rs * ss;              // rho* s*
  const double Us2 = rs * ut;              // rho* v
  const double Es = fma(ss - un, fma(p, inv, Us1), fac * E);
  const double mom = r * un;
  F[0] = fma(spm, rs - r, mom);
  F[1] = fma(spm, Us1 - mom, fma(mom, un, p));
  F[2] = fma(spm, Us2 - r * ut, mom * ut);
  F[3] = fma(spm, Es - E, (E + p) * un);
}

__device__ __forceinline__ void hllc(double rL, double uL, double vL, double pL, double rR, double uR,
                                     double vR, double pR, const Gas& g, double F[4]) {
  const double gpL = g.gamma * pL, gpR = g.gamma * pR;
  const double aL = gpL * rsqrt_nr(gpL * rL);
  const double aR = gpR * rsqrt_nr(gpR * rR);
  const double sL = fmin(uL - aL, uR - aR);
  const double sR = fmax(uL + aL, uR + aR);
  const double dL = sL - uL, dR = sR - uR;
  const double mL = rL * dL, mR = rR * dR;
  const double num = fma(-uR, mR, fma(uL, mL, pR - pL));
  const double ss = quot(num, mL - mR);
  if (ss == 0.0) {
    if (sL < 0.0 && sR > 0.0) {
      // With s* = 0 and sL < 0 < sR each branch's star flux F_K + s_K (U*_K - U_K) reduces,
      // in exact arithmetic, to (0, p_K - m_K u_K, 0, 0): the mass, tangential-momentum and
      // energy terms cancel identically and the normal momentum is the star pressure.  The
      // average of the two branches is therefore formed directly (4 instead of ~66 FP64
      // instructions; quiescent gas, u = 0 on both sides of a face, always lands here).
      F[0] = 0.0;
      F[1] = 0.5 * (fma(-mL, uL, pL) + fma(-mR, uR, pR));
      F[2] = 0.0;
      F[3] = 0.0;
      return;
    }
    double FL[4], FR[4];
    hllc_branch(rL, uL, vL, pL, sL, dL, mL, fmin(0.0, sL), ss, g, FL);
    hllc_branch(rR, uR, vR, pR, sR, dR, mR, fmax(0.0, sR), ss, g, FR);
#pragma unroll
    for (int c = 0; c < 4; ++c) F[c] = 0.5 * (FL[c] + FR[c]);
    return;
  }
  const bool left = ss > 0.0;
  hllc_branch(left ? rL : rR, left ? uL : uR, left ? vL : vR, left ? pL : pR, left ? sL : sR,
              left ? dL : dR, left ? mL : mR, left ? fmin(0.0, sL) : fmax(0.0, sR), ss, g, F);
}

// ---------------------------------------------------------------------------------------
// Navier-Stokes viscous and heat flux through a face (constant mu, Stokes hypothesis,
// R = 1).  Normal derivatives by two-point differences, tangential ones by the mean of the
// central differences of the two adjacent cells.  Constants (per face orientation):
//   c43n = 4/3 mu / h_n, c23t = 2/3 mu / (4 h_t), cn = mu / h_n, ct = mu / (4 h_t),
//   ck = kappa / h_n with kappa = mu gamma / ((gamma - 1) Pr).
// ---------------------------------------------------------------------------------------
struct ViscC {
  double c43n, c23t, cn, ct, ck;
};

}  // namespace js
