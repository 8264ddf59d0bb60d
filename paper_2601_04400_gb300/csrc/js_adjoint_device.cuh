// Reverse-mode building blocks of the FP64 right-hand side (gradient chain rule of Sec. 2,
// applied to the discrete operator).  Each routine differentiates exactly the forward
// formulation used by the stage kernel (js_device.cuh): cell-centred WENO5 with product
// weights, HLLC on the upwind side with the standard star-state energy, the viscous face flux
// and the cons -> prim map.  Non-smooth points follow the oracle's convention: min/max pass
// the derivative to their first argument on ties, sign(s*) = 0 averages both branches.
#pragma once
#include "js_device.cuh"

namespace js {

// quotient a/b exactly as the forward kernel forms it (quot), with the reciprocal it used
__device__ __forceinline__ double quot_r(double a, double b, double& r) {
  r = recip(b);
  return a * r;
}

// ---------------------------------------------------------------------------------------
// WENO5, cell-centred: forward with the internals the reverse pass needs
// ---------------------------------------------------------------------------------------
// saved per cell and variable: s0, s1, s2 (4 beta_k + 4 eps), qL, rL, qR, rR where
// q = num/den of the face state (state = q_i + q/6) and r ~ 1/den.
constexpr int WENO_SAVE = 7;

struct Dl {  // first differences d_{i-3/2}, d_{i-1/2}, d_{i+1/2}, d_{i+3/2}
  double m2, m1, p1, p2;
};

__device__ __forceinline__ void weno_cell_fwd(double q0, const Dl& d, double& Lf, double& Rf, double sv[WENO_SAVE]) {
  const double D0 = d.m1 - d.m2, D1 = d.p1 - d.m1, D2 = d.p2 - d.p1;
  const double t0 = fma(2.0, d.m1, D0), t1 = d.m1 + d.p1, t2 = fma(-2.0, d.p1, D2);
  const double s0 = fma(K13 * D0, D0, fma(t0, t0, EPS4));
  const double s1 = fma(K13 * D1, D1, fma(t1, t1, EPS4));
  const double s2 = fma(K13 * D2, D2, fma(t2, t2, EPS4));
  const double p01 = s0 * s1, p02 = s0 * s2, p12 = s1 * s2;
  const double w0 = p12 * p12, w1 = p02 * p02, w2 = p01 * p01;
  const double w1_6 = 6.0 * w1;
  double rL, rR;
  const double w2_3 = 3.0 * w2;
  const double e0L = fma(-2.0, d.m2, 5.0 * d.m1), e1L = fma(2.0, d.p1, d.m1), e2L = fma(4.0, d.p1, -d.p2);
  const double qL = quot_r(fma(w0, e0L, fma(w1_6, e1L, w2_3 * e2L)), w0 + w1_6 + w2_3, rL);
  const double w0_3 = 3.0 * w0;
  const double e0R = fma(-4.0, d.m1, d.m2), e1R = fma(-2.0, d.m1, -d.p1), e2R = fma(2.0, d.p2, -5.0 * d.p1);
  const double qR = quot_r(fma(w0_3, e0R, fma(w1_6, e1R, w2 * e2R)), w0_3 + w1_6 + w2, rR);
  Lf = fma(qL, SIXTH, q0);
  Rf = fma(qR, SIXTH, q0);
  sv[0] = s0; sv[1] = s1; sv[2] = s2;
  sv[3] = qL; sv[4] = rL; sv[5] = qR; sv[6] = rR;
}

// Reverse of the cell-centred WENO5 along one line, for one variable.  Like the forward
// window it slides over the first differences d (d_{i+3/2} = q_{i+2} - q_{i+1} is the only
// new one per cell); it also slides over the adjoints of the differences, so that each cell
// emits the complete adjoint of q_{i-2} (d_{i-5/2} adds, d_{i-3/2} subtracts, plus the
// direct term Lb + Rb of the face states q_{i-2} + q/6).
//
// Algebra per cell, with n = Lb rL / 6 and Rb rR / 6 the adjoints of the two quotients
// num/den (scaled by 4 below, which the fma constants undo):
//   dq/dw_k = c_k (e_k - q) / den        (c = 1, 6, 3 left-biased; 3, 6, 1 right-biased)
//   w0 = (s1 s2)^2, w1 = (s0 s2)^2, w2 = (s0 s1)^2
//   s_k = 13/3 D_k^2 + t_k^2 + 4 eps, t0 = 3 d_{i-1/2} - d_{i-3/2}, t1 = d_{i-1/2} + d_{i+1/2},
//   t2 = d_{i+3/2} - 3 d_{i+1/2}
//   the candidate corrections e_k are fixed 2-term combinations of d.
struct WenoRev {
  double q1;                // q_{i+1}
  double m2, m1, p1;        // d_{i-3/2}, d_{i-1/2}, d_{i+1/2}
  double D0, D1, cD0, cD1;  // D_{i-1}, D_i and 13/3 of them
  double bprev;             // adjoint of d_{i-5/2} (complete)
  double b0, b1, b2;        // adjoints of d_{i-3/2}, d_{i-1/2}, d_{i+1/2} so far
  double dir1, dir2;        // direct adjoints of cells i-1, i-2

  __device__ __forceinline__ void init(double qm2, double qm1, double q, double qp1) {
    q1 = qp1;
    m2 = qm1 - qm2;
    m1 = q - qm1;
    p1 = qp1 - q;
    D0 = m1 - m2;
    D1 = p1 - m1;
    cD0 = K13 * D0;
    cD1 = K13 * D1;
    bprev = b0 = b1 = b2 = 0.0;
    dir1 = dir2 = 0.0;
  }

  // cell i: q_{i+2}, its saved internals sv (s0, s1, s2, qL, rL, qR, rR), the adjoints Lb
  // (state at i+1/2) and Rb (state at i-1/2).  Returns the adjoint of q_{i-2}, then
  // slides to cell i+1.
  __device__ __forceinline__ double step(double q2, const double sv[WENO_SAVE], double Lb, double Rb) {
    const double p2 = q2 - q1, D2 = p2 - p1, cD2 = K13 * D2;
    const double t0 = fma(2.0, m1, D0), t1 = m1 + p1, t2 = fma(-2.0, p1, D2);
    const double s0 = sv[0], s1 = sv[1], s2 = sv[2];
    const double p01 = s0 * s1, p02 = s0 * s2, p12 = s1 * s2;
    const double w0 = p12 * p12, w1 = p02 * p02, w2 = p01 * p01;
    constexpr double TWO_THIRDS = 2.0 / 3.0;  // 4 x 1/6
    const double nL = (TWO_THIRDS * Lb) * sv[4], nR = (TWO_THIRDS * Rb) * sv[6];
    const double dL = -nL * sv[3], dR = -nR * sv[5];
    const double e0L = fma(-2.0, m2, 5.0 * m1), e1L = fma(2.0, p1, m1), e2L = fma(4.0, p1, -p2);
    const double e0R = fma(-4.0, m1, m2), e1R = fma(-2.0, m1, -p1), e2R = fma(2.0, p2, -5.0 * p1);
    // 4 x adjoints of w0, w1 / 6, w2
    const double bw0 = fma(3.0, fma(nR, e0R, dR), fma(nL, e0L, dL));
    const double bw1 = fma(nL, e1L, dL) + fma(nR, e1R, dR);
    const double bw2 = fma(3.0, fma(nL, e2L, dL), fma(nR, e2R, dR));
    // 2 x adjoints of p12, p02, p01 and of s0, s1, s2
    const double bp12 = p12 * bw0, bp02 = (6.0 * p02) * bw1, bp01 = p01 * bw2;
    const double bs0 = fma(bp01, s1, bp02 * s2);
    const double bs1 = fma(bp01, s0, bp12 * s2);
    const double bs2 = fma(bp02, s0, bp12 * s1);
    // half the derivatives of s_k with respect to the differences
    const double a0 = cD0 + t0, c0 = fma(3.0, t0, cD0);  // -ds0/dm2, ds0/dm1
    const double a1 = t1 - cD1, c1 = t1 + cD1;           // ds1/dm1, ds1/dp1
    const double a2 = fma(3.0, t2, cD2), c2 = cD2 + t2;  // -ds2/dp1, ds2/dp2
    // candidate-correction terms: products of the (scaled) quotient adjoints and the weights
    const double A = w0 * nL, B = w0 * nR, C = w1 * nL, Dd = w1 * nR, E = w2 * nL, F = w2 * nR;
    const double gm2 = fma(-0.5, A, fma(0.75, B, -a0 * bs0));
    const double gm1 = fma(1.25, A, fma(-3.0, B, fma(1.5, C, fma(-3.0, Dd, fma(c0, bs0, a1 * bs1)))));
    const double gp1 = fma(3.0, C, fma(-1.5, Dd, fma(3.0, E, fma(-1.25, F, fma(c1, bs1, -a2 * bs2)))));
    const double gp2 = fma(-0.75, E, fma(0.5, F, c2 * bs2));
    // d_{i-3/2} is complete: emit q_{i-2}
    const double done = b0 + gm2;
    const double out = (bprev - done) + dir2;
    bprev = done;
    b0 = b1 + gm1;
    b1 = b2 + gp1;
    b2 = gp2;
    dir2 = dir1;
    dir1 = Lb + Rb;
    // slide
    q1 = q2;
    m2 = m1;
    m1 = p1;
    p1 = p2;
    D0 = D1;
    D1 = D2;
    cD0 = cD1;
    cD1 = cD2;
    return out;
  }

  // after the last cell c1 - 1 of a segment: adjoints of q_{c1-2}, q_{c1-1}, q_{c1}, q_{c1+1}
  __device__ __forceinline__ void flush(double out[4]) const {
    out[0] = (bprev - b0) + dir2;
    out[1] = (b0 - b1) + dir1;
    out[2] = b1 - b2;
    out[3] = b2;
  }
};

// ---------------------------------------------------------------------------------------
// HLLC forward + reverse (face-normal frame)
// ---------------------------------------------------------------------------------------
struct Face4 {
  double r, un, ut, p;
};

// reverse of hllc_branch for one side; adds to the side adjoints and returns the adjoints
// of s, d, m, spm, ss; gb accumulates d/dgamma.
__device__ __forceinline__ void hllc_branch_vjp(double r, double un, double ut, double p, double s, double d, double m,
                                                double spm, double ss, const Gas& g, const double Fb[4], double& br,
                                                double& bun, double& but, double& bp, double& bs, double& bd,
                                                double& bm, double& bspm, double& bss, double& gb) {
  const double ke = fma(un, un, ut * ut);
  const double E = fma(0.5 * r, ke, p * g.g1);
  const double inv = recip(s - ss);
  const double rs = m * inv, fac = d * inv;
  const double Us1 = rs * ss, Us2 = rs * ut;
  const double X = fma(p, inv, Us1);
  const double Es = fma(ss - un, X, fac * E);
  const double mom = r * un;
  // F0 = mom + spm (rs - r); F1 = mom un + p + spm (Us1 - mom);
  // F2 = mom ut + spm (Us2 - r ut); F3 = (E + p) un + spm (Es - E)
  bspm = Fb[0] * (rs - r) + Fb[1] * (Us1 - mom) + Fb[2] * (Us2 - r * ut) + Fb[3] * (Es - E);
  double bmom = Fb[0] + Fb[1] * (un - spm) + Fb[2] * ut;
  double brs = Fb[0] * spm;
  br = -spm * (Fb[0] + Fb[2] * ut);
  bun = Fb[1] * mom + Fb[3] * (E + p);
  but = Fb[2] * (mom - spm * r);
  bp = Fb[1] + Fb[3] * un;
  double bUs1 = Fb[1] * spm;
  const double bUs2 = Fb[2] * spm;
  double bE = Fb[3] * (un - spm);
  const double bEs = Fb[3] * spm;
  // Es = fac E + (ss - un) X
  const double bfac = bEs * E;
  bE += bEs * fac;
  const double bX = bEs * (ss - un);
  bss = bEs * X;
  bun -= bEs * X;
  // X = p inv + Us1
  bp += bX * inv;
  double binv = bX * p;
  bUs1 += bX;
  // Us2 = rs ut, Us1 = rs ss
  brs += bUs2 * ut + bUs1 * ss;
  but += bUs2 * rs;
  bss += bUs1 * rs;
  // fac = d inv, rs = m inv
  bd = bfac * inv;
  bm = brs * inv;
  binv += bfac * d + brs * m;
  // inv = 1/(s - ss)
  const double t = binv * inv * inv;
  bs = -t;
  bss += t;
  // mom = r un
  br += bmom * un;
  bun += bmom * r;
  // E = 0.5 r ke + p/(gamma - 1)
  br += bE * 0.5 * ke;
  const double bke = bE * 0.5 * r;
  bp += bE * g.g1;
  gb -= bE * p * g.g1 * g.g1;
  bun += 2.0 * un * bke;
  but += 2.0 * ut * bke;
}

// Reverse of hllc(): F adjoint Fb (normal frame) -> adjoints of both face states (added).
__device__ __forceinline__ void hllc_vjp(const Face4& L, const Face4& R, const Gas& g, const double Fb[4], Face4& bL,
                                         Face4& bR, double& gb) {
  const double gpL = g.gamma * L.p, gpR = g.gamma * R.p;
  const double yL = rsqrt_nr(gpL * L.r), yR = rsqrt_nr(gpR * R.r);
  const double aL = gpL * yL, aR = gpR * yR;
  const double xL = L.un - aL, xR = R.un - aR;  // candidates of sL
  const double zL = L.un + aL, zR = R.un + aR;  // candidates of sR
  const bool sL_right = xR < xL;                // min ties go to the first argument
  const bool sR_right = zL < zR;                // max ties go to the first argument
  const double sL = sL_right ? xR : xL, sR = sR_right ? zR : zL;
  const double dL = sL - L.un, dR = sR - R.un;
  const double mL = L.r * dL, mR = R.r * dR;
  const double num = fma(-R.un, mR, fma(L.un, mL, R.p - L.p));
  const double den = mL - mR;
  double rden;
  const double ss = quot_r(num, den, rden);
  double bsL = 0.0, bsR = 0.0, bdL = 0.0, bdR = 0.0, bmL = 0.0, bmR = 0.0, bss = 0.0;
  auto side = [&](bool left, double scale) {
    double Fs[4] = {scale * Fb[0], scale * Fb[1], scale * Fb[2], scale * Fb[3]};
    double br, bun, but, bp, bs, bd, bm, bspm, bs2;
    if (left) {
      const double spm = fmin(0.0, sL);
      hllc_branch_vjp(L.r, L.un, L.ut, L.p, sL, dL, mL, spm, ss, g, Fs, br, bun, but, bp, bs, bd, bm, bspm, bs2, gb);
      bL.r += br; bL.un += bun; bL.ut += but; bL.p += bp;
      bsL += bs + ((sL < 0.0) ? bspm : 0.0);
      bdL += bd;
      bmL += bm;
    } else {
      const double spm = fmax(0.0, sR);
      hllc_branch_vjp(R.r, R.un, R.ut, R.p, sR, dR, mR, spm, ss, g, Fs, br, bun, but, bp, bs, bd, bm, bspm, bs2, gb);
      bR.r += br; bR.un += bun; bR.ut += but; bR.p += bp;
      bsR += bs + ((sR > 0.0) ? bspm : 0.0);
      bdR += bd;
      bmR += bm;
    }
    bss += bs2;
  };
  if (ss == 0.0 && sL < 0.0 && sR > 0.0) {
    // Reverse of the s* = 0 closed form of the forward flux: at s* = 0 (spm = s on both sides)
    // the derivatives of a branch's star flux F_K + s_K (U*_K - U_K) reduce to
    //   dF0 = (m/s) ds*,   dF1 = -u d drho + rho (2u - s) du + dp - rho u ds + m ds*,
    //   dF2 = (m ut/s) ds*,   dF3 = (d (E + p)/s - m u) ds*      (d = s - u, m = rho d),
    // with d and m already substituted (no separate d, m adjoints) and no gamma dependence
    // (dF/dE = 0 there); each branch carries half of the face's flux adjoint.
    auto side0 = [&](const Face4& Q, double s, double d, double m, Face4& bQ, double& bsK) {
      const double f1 = 0.5 * Fb[1];
      const double is = recip(s);
      const double E = fma(0.5 * Q.r, fma(Q.un, Q.un, Q.ut * Q.ut), Q.p * g.g1);
      bss += 0.5 * (fma(fma(Fb[2], Q.ut, Fb[0]), m * is, Fb[1] * m) + Fb[3] * fma(d * (E + Q.p), is, -m * Q.un));
      bQ.r -= f1 * Q.un * d;
      bQ.un += f1 * Q.r * (2.0 * Q.un - s);
      bQ.p += f1;
      bsK -= f1 * Q.r * Q.un;
    };
    side0(L, sL, dL, mL, bL, bsL);
    side0(R, sR, dR, mR, bR, bsR);
  } else if (ss == 0.0) {
    side(true, 0.5);
    side(false, 0.5);
  } else {
    side(ss > 0.0, 1.0);
  }
  // ss = num/den, den = mL - mR, num = (pR - pL) + uL mL - uR mR
  const double bnum = bss * rden, bden = -bss * ss * rden;
  bmL += bden + bnum * L.un;
  bmR += -bden - bnum * R.un;
  bR.p += bnum;
  bL.p -= bnum;
  double buL = bnum * mL, buR = -bnum * mR;
  // m = r d, d = s - u
  bL.r += bmL * dL;
  bR.r += bmR * dR;
  bdL += bmL * L.r;
  bdR += bmR * R.r;
  bsL += bdL;
  bsR += bdR;
  buL -= bdL;
  buR -= bdR;
  // sL = min(uL - aL, uR - aR), sR = max(uL + aL, uR + aR)
  double baL = 0.0, baR = 0.0;
  if (sL_right) { buR += bsL; baR -= bsL; } else { buL += bsL; baL -= bsL; }
  if (sR_right) { buR += bsR; baR += bsR; } else { buL += bsR; baL += bsR; }
  bL.un += buL;
  bR.un += buR;
  // a = sqrt(gamma p / rho) = gp y with y = 1/sqrt(gp rho):
  // da/dp = gamma y / 2, da/drho = -a gp y^2 / 2, da/dgamma = a p rho y^2 / 2
  bL.p += baL * 0.5 * g.gamma * yL;
  bR.p += baR * 0.5 * g.gamma * yR;
  bL.r -= baL * 0.5 * aL * gpL * yL * yL;
  bR.r -= baR * 0.5 * aR * gpR * yR * yR;
  gb += 0.5 * (baL * aL * L.p * L.r * yL * yL + baR * aR * R.p * R.r * yR * yR);
}

// ---------------------------------------------------------------------------------------
// cons -> prim reverse: prim adjoints (rho, u, v, p, T) -> conserved adjoints; gb += d/dgamma
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void prim_vjp(double r, double mx, double my, double E, const Gas& g, const double qb[5],
                                         double ub[4], double& gb) {
  const double ir = recip(r);
  const double u = mx * ir, v = my * ir;
  const double p = g.gm1 * fma(-0.5, fma(mx, u, my * v), E);
  const double T = p * ir;
  const double bp = fma(qb[4], ir, qb[3]);
  const double brq = fma(-qb[4], T * ir, qb[0]);
  ub[3] = g.gm1 * bp;
  ub[1] = fma(qb[1], ir, -g.gm1 * u * bp);
  ub[2] = fma(qb[2], ir, -g.gm1 * v * bp);
  ub[0] = brq - fma(u, qb[1], v * qb[2]) * ir + 0.5 * g.gm1 * fma(u, u, v * v) * bp;
  gb += bp * p * g.g1;
}

}  // namespace js
