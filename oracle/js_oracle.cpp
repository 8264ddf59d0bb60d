// FP64 CPU ORACLE for the JAX-Shock finite-volume right-hand side (arXiv 2601.04400).
//
// TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU-baseline leg of
// bench.py load this library; the CUDA library never does, and the two share no code.
//
// What it computes, in the paper's order and notation:
//   * state U = [rho, rho u, rho v, E] and ideal-gas EOS p = (gamma-1)(E - rho(u^2+v^2)/2)
//     (Sec. 2, Eq. 1 and the EOS that follows it);
//   * fifth-order WENO reconstruction of the primitive variables at every cell face
//     (Sec. 2, "WENO schemes with convex reconstruction of candidate stencils"), textbook
//     Jiang-Shu form with eps = 1e-6 and power 2, component-wise;
//   * the HLLC flux of Sec. 2 (flux, star states, wave speeds s^L, s^R, s^+, s^-, contact
//     speed s^*), y-flux by interchanging u and v.  The star-state energy uses the standard
//     (Toro) expression; the literally printed energy entry is kept behind `hllc_literal`
//     for documentation and fails the HLLC consistency condition (see tests);
//   * optional Navier-Stokes viscous and heat fluxes (constant mu, Stokes hypothesis, R = 1,
//     kappa = mu gamma / ((gamma-1) Pr)), central differences at faces: the paper names
//     the Navier-Stokes equations but prints no viscous terms, so this is a stated reading;
//   * flux divergence plus the Laplacian artificial viscosity nu * lap(U) of the update
//     equation in Sec. 2;
//   * the ghost-cell immersed boundary (Sec. 2, Fig. 1(c); Mittal & Iaccarino): cells are
//     fluid (sdf >= 0) or solid; ghost cells are solid cells with a fluid cell in their 7x7
//     box; each ghost state is the slip-wall mirror of the bilinear interpolation (fluid
//     cells only, weights renormalised) at the image point x_G - 2 sdf_G n;
//   * domain boundary halos (transmissive, reflective, periodic, inflow; Sec. 3 cylinder
//     case) three cells deep, x sides on interior rows first, then y sides on the full
//     padded width;
//   * three-stage SSP Runge-Kutta (Shu-Osher) in place of the forward-Euler update that the
//     paper prints; CFL time step from the maximum wave speed;
//   * optionally the neural flux of Sec. 2.3 (or_nn_set): a three-layer 3x3 convolutional
//     network (4 -> 16 -> 32 -> 4 channels, ReLU, ReLU, tanh, zero "SAME" padding; 6388
//     parameters, the paper's count) on the normalised mean of the two WENO5 face states in
//     conserved variables, per direction, added to the HLLC flux of every face; both
//     directions share the network, y faces enter as transposed images with the normal
//     momentum first (readings: the paper fixes the layers and the parameter count, not the
//     channel widths, the input's face frame or the normalisation).
//
// Every routine is templated on the scalar type so that the same plain code gives FP64
// values (double), forward-mode tangents (Dual<N>, the oracle's discrete derivative) and
// operation counts (Cnt).  Compile with -ffp-contract=off: no fused multiply-adds.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------------------
// scalar types
// ---------------------------------------------------------------------------------------
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int k = 0; k < N; ++k) d[k] = 0.0; }
  Dual(double x) : v(x) { for (int k = 0; k < N; ++k) d[k] = 0.0; }
};
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v); for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v); for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r(-a.v); for (int k = 0; k < N; ++k) r.d[k] = -a.d[k]; return r; }
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v); for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v / b.v);
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
  return r; }
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r(a.v * b); for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b; return r; }
template <int N> Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) {
  Dual<N> r(a.v / b); for (int k = 0; k < N; ++k) r.d[k] = a.d[k] / b; return r; }
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N> bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }
template <int N> bool operator<=(const Dual<N>& a, const Dual<N>& b) { return a.v <= b.v; }
template <int N> bool operator>=(const Dual<N>& a, const Dual<N>& b) { return a.v >= b.v; }
template <int N> bool operator<(const Dual<N>& a, double b) { return a.v < b; }
template <int N> bool operator>(const Dual<N>& a, double b) { return a.v > b; }
template <int N> bool operator<=(const Dual<N>& a, double b) { return a.v <= b; }
template <int N> bool operator>=(const Dual<N>& a, double b) { return a.v >= b; }
template <int N> bool operator==(const Dual<N>& a, double b) { return a.v == b; }
template <int N> Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r(std::sqrt(a.v));
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] / (2.0 * r.v);
  return r; }

// Operation counter: every arithmetic operation on Cnt increments a global tally.
struct OpTally { long long add, mul, div, sqrt, cmp; };
OpTally g_tally;
struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_tally.add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_tally.add; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_tally.mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_tally.div; return Cnt(a.v / b.v); }
inline Cnt operator+(Cnt a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, Cnt b) { return Cnt(a) + b; }
inline Cnt operator-(Cnt a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, Cnt b) { return Cnt(a) - b; }
inline Cnt operator*(Cnt a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, Cnt b) { return Cnt(a) * b; }
inline Cnt operator/(Cnt a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, Cnt b) { return Cnt(a) / b; }
inline bool operator<(Cnt a, Cnt b) { ++g_tally.cmp; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { ++g_tally.cmp; return a.v > b.v; }
inline bool operator<=(Cnt a, Cnt b) { ++g_tally.cmp; return a.v <= b.v; }
inline bool operator>=(Cnt a, Cnt b) { ++g_tally.cmp; return a.v >= b.v; }
inline bool operator<(Cnt a, double b) { ++g_tally.cmp; return a.v < b; }
inline bool operator>(Cnt a, double b) { ++g_tally.cmp; return a.v > b; }
inline bool operator<=(Cnt a, double b) { ++g_tally.cmp; return a.v <= b; }
inline bool operator>=(Cnt a, double b) { ++g_tally.cmp; return a.v >= b; }
inline bool operator==(Cnt a, double b) { ++g_tally.cmp; return a.v == b; }
inline Cnt sqrt(Cnt a) { ++g_tally.sqrt; return Cnt(std::sqrt(a.v)); }

inline double val(double x) { return x; }
template <int N> double val(const Dual<N>& x) { return x.v; }
inline double val(Cnt x) { return x.v; }

// A parameter that is exactly zero with no tangent switches its term off.
inline bool is_off(double x) { return x == 0.0; }
template <int N> bool is_off(const Dual<N>& x) {
  if (x.v != 0.0) return false;
  for (int k = 0; k < N; ++k) if (x.d[k] != 0.0) return false;
  return true; }
inline bool is_off(Cnt x) { return x.v == 0.0; }

using std::sqrt;
template <class T> T tmin(const T& a, const T& b) { return (b < a) ? b : a; }  // tie -> a
template <class T> T tmax(const T& a, const T& b) { return (a < b) ? b : a; }  // tie -> a
template <class T> T tabs(const T& a) { return (a < 0.0) ? -a : a; }

// tanh and a value carrying a tangent (slot 0 of a dual number)
inline double ttanh(double x) { return std::tanh(x); }
template <int N> Dual<N> ttanh(const Dual<N>& a) {
  const double t = std::tanh(a.v);
  Dual<N> r(t);
  for (int k = 0; k < N; ++k) r.d[k] = (1.0 - t * t) * a.d[k];
  return r;
}
inline Cnt ttanh(Cnt a) { return Cnt(std::tanh(a.v)); }
template <class T> T seeded(double v, double) { return T(v); }
template <> Dual<1> seeded<Dual<1>>(double v, double d) { Dual<1> r(v); r.d[0] = d; return r; }

// ---------------------------------------------------------------------------------------
// Neural flux (Sec. 2.3): a fully convolutional network of three 3x3 layers with zero
// ("SAME") padding, 4 -> 16 -> 32 -> 4 channels, ReLU, ReLU, tanh (6388 parameters), maps
// the normalised WENO5 face states of one direction to a flux correction added to HLLC.
// Parameter layout: w1[16][4][3][3], b1[16], w2[32][16][3][3], b2[32], w3[4][32][3][3], b3[4].
// ---------------------------------------------------------------------------------------
const int NN_C[4] = {4, 16, 32, 4};
const int NN_NPARAM = 16 * 4 * 9 + 16 + 32 * 16 * 9 + 32 + 4 * 32 * 9 + 4;  // 6388

struct NnCfg {
  bool on = false;
  std::vector<double> w, dw;               // parameters and their tangent
  double mean[4], sd[4], scale[4];         // input normalisation and output scale (frame channels)
};
NnCfg g_nn;

// one 3x3 layer with zero padding: out[co][h][x] = b[co] + sum_ci,ky,kx w[co][ci][ky][kx] in[ci][h+ky-1][x+kx-1]
template <class T>
void nn_conv(const std::vector<T>& in, int cin, int H, int Wd, const T* w, const T* b, int cout, std::vector<T>& out) {
  out.assign((size_t)cout * H * Wd, T(0.0));
  for (int co = 0; co < cout; ++co)
    for (int h = 0; h < H; ++h)
      for (int x = 0; x < Wd; ++x) {
        T acc = b[co];
        for (int ci = 0; ci < cin; ++ci)
          for (int ky = 0; ky < 3; ++ky) {
            const int hh = h + ky - 1;
            if (hh < 0 || hh >= H) continue;
            for (int kx = 0; kx < 3; ++kx) {
              const int xx = x + kx - 1;
              if (xx < 0 || xx >= Wd) continue;
              acc = acc + w[((co * cin + ci) * 3 + ky) * 3 + kx] * in[((size_t)ci * H + hh) * Wd + xx];
            }
          }
        out[((size_t)co * H + h) * Wd + x] = acc;
      }
}

// the network on one image x[4][H][W] (normalised frame channels) -> y[4][H][W] (scaled flux)
template <class T>
void nn_forward(const std::vector<T>& x, int H, int Wd, const std::vector<T>& P, std::vector<T>& y) {
  const T* w1 = P.data();
  const T* b1 = w1 + 16 * 4 * 9;
  const T* w2 = b1 + 16;
  const T* b2 = w2 + 32 * 16 * 9;
  const T* w3 = b2 + 32;
  const T* b3 = w3 + 4 * 32 * 9;
  std::vector<T> a1, a2, z3;
  nn_conv(x, 4, H, Wd, w1, b1, 16, a1);
  for (auto& v : a1) v = (v > 0.0) ? v : T(0.0);
  nn_conv(a1, 16, H, Wd, w2, b2, 32, a2);
  for (auto& v : a2) v = (v > 0.0) ? v : T(0.0);
  nn_conv(a2, 32, H, Wd, w3, b3, 4, z3);
  y.resize(z3.size());
  const size_t plane = (size_t)H * Wd;
  for (int c = 0; c < 4; ++c)
    for (size_t o = 0; o < plane; ++o) y[c * plane + o] = g_nn.scale[c] * ttanh(z3[c * plane + o]);
}

template <class T>
std::vector<T> nn_params() {
  std::vector<T> P(NN_NPARAM);
  for (int k = 0; k < NN_NPARAM; ++k) P[k] = seeded<T>(g_nn.w[k], g_nn.dw.empty() ? 0.0 : g_nn.dw[k]);
  return P;
}

// ---------------------------------------------------------------------------------------
// problem description
// ---------------------------------------------------------------------------------------
enum { BC_TRANSMISSIVE = 0, BC_REFLECTIVE = 1, BC_PERIODIC = 2, BC_INFLOW = 3 };
enum { OK = 0, ERR_ARG = -1, ERR_NONPHYSICAL = -3, ERR_IB = -5 };
const int NG = 3;  // halo depth

// faces at which face_flux took the positivity fallback (reading of "positivity-preserving
// HLLC", Sec. 2): counted for the tests, reset by or_fallback_faces
long long g_fallback_faces = 0;

}  // namespace

extern "C" {
typedef struct {
  int nx, ny;          // cells; ny == 1 is a one-dimensional problem (no y fluxes)
  double x0, y0;       // lower-left corner of the domain
  double dx, dy;       // uniform spacing
  int bc[4];           // x-low, x-high, y-low, y-high
  int wall;            // immersed wall: 0 slip (the paper), 1 no-slip
  int hllc_literal;    // 1: the star-state energy exactly as printed (documentation only)
} or_grid;
}

namespace {

// theta = [gamma, mu, Pr, nu, inflow[side][rho, u, v, p]]  (20 entries)
const int NTHETA = 20;
template <class T>
struct Par {
  T gamma, mu, Pr, nu;
  T inflow[4][4];
};

template <class T>
Par<T> make_par(const double* th) {
  Par<T> P;
  P.gamma = T(th[0]); P.mu = T(th[1]); P.Pr = T(th[2]); P.nu = T(th[3]);
  for (int s = 0; s < 4; ++s) for (int c = 0; c < 4; ++c) P.inflow[s][c] = T(th[4 + 4 * s + c]);
  return P;
}

struct Layout {
  int nx, ny, W, H, gy;
  explicit Layout(const or_grid& g) : nx(g.nx), ny(g.ny) {
    gy = (ny == 1) ? 0 : NG;
    W = nx + 2 * NG;
    H = ny + 2 * gy;
  }
  long idx(int i, int j) const { return (long)(j + gy) * W + (i + NG); }
  long size() const { return (long)W * H; }
};

// ---------------------------------------------------------------------------------------
// immersed-boundary tables (geometry only; plain doubles)
// ---------------------------------------------------------------------------------------
struct IbTable {
  std::vector<unsigned char> tag;  // nx*ny: 0 fluid, 1 solid, 2 ghost
  std::vector<int> gcell;          // ghost cell j*nx+i
  std::vector<int> icell;          // 4 per ghost: interpolation cells j*nx+i
  std::vector<double> w;           // 4 per ghost, renormalised over fluid cells
  std::vector<double> nrm;         // 2 per ghost: outward (into fluid) unit normal
};

int build_ib(const or_grid& g, const double* sdf, IbTable& ib) {
  const int nx = g.nx, ny = g.ny;
  ib.tag.assign((size_t)nx * ny, 0);
  ib.gcell.clear(); ib.icell.clear(); ib.w.clear(); ib.nrm.clear();
  if (!sdf) return OK;
  if (ny < 2) return ERR_ARG;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      ib.tag[(size_t)j * nx + i] = (sdf[(size_t)j * nx + i] < 0.0) ? 1 : 0;
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      if (ib.tag[(size_t)j * nx + i] == 0) continue;
      bool near_fluid = false;
      for (int b = -3; b <= 3 && !near_fluid; ++b)
        for (int a = -3; a <= 3; ++a) {
          int ii = i + a, jj = j + b;
          if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
          if (sdf[(size_t)jj * nx + ii] >= 0.0) { near_fluid = true; break; }
        }
      if (near_fluid) ib.tag[(size_t)j * nx + i] = 2;
    }
  }
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      if (ib.tag[(size_t)j * nx + i] != 2) continue;
      const double phi = sdf[(size_t)j * nx + i];
      // unit normal n = grad(phi)/|grad(phi)|: central differences, one-sided at grid edges
      const int il = (i > 0) ? i - 1 : i, ir = (i < nx - 1) ? i + 1 : i;
      const int jl = (j > 0) ? j - 1 : j, jr = (j < ny - 1) ? j + 1 : j;
      const double gx = (sdf[(size_t)j * nx + ir] - sdf[(size_t)j * nx + il]) / ((ir - il) * g.dx);
      const double gyv = (sdf[(size_t)jr * nx + i] - sdf[(size_t)jl * nx + i]) / ((jr - jl) * g.dy);
      const double gn = std::sqrt(gx * gx + gyv * gyv);
      if (!(gn > 0.0)) return ERR_IB;
      const double nxv = gx / gn, nyv = gyv / gn;
      // image point: mirror of the ghost centre across the wall
      const double xg = g.x0 + (i + 0.5) * g.dx, yg = g.y0 + (j + 0.5) * g.dy;
      const double xi = xg - 2.0 * phi * nxv, yi = yg - 2.0 * phi * nyv;
      // fractional cell-centre coordinates of the image point; it must lie in the domain
      const double fx = (xi - g.x0) / g.dx - 0.5, fy = (yi - g.y0) / g.dy - 0.5;
      if (!(fx >= -0.5) || !(fy >= -0.5) || !(fx <= nx - 0.5) || !(fy <= ny - 0.5)) return ERR_IB;
      // 2x2 block of cell centres around it, clamped into the grid
      int i0 = (int)std::floor(fx), j0 = (int)std::floor(fy);
      if (i0 < 0) i0 = 0;
      if (i0 > nx - 2) i0 = nx - 2;
      if (j0 < 0) j0 = 0;
      if (j0 > ny - 2) j0 = ny - 2;
      const double tx = fx - i0, ty = fy - j0;
      int cells[4] = {j0 * nx + i0, j0 * nx + i0 + 1, (j0 + 1) * nx + i0, (j0 + 1) * nx + i0 + 1};
      double w[4] = {(1.0 - tx) * (1.0 - ty), tx * (1.0 - ty), (1.0 - tx) * ty, tx * ty};
      double s = 0.0;
      for (int k = 0; k < 4; ++k) {
        if (ib.tag[cells[k]] != 0) w[k] = 0.0;
        s = s + w[k];
      }
      if (!(s > 0.0)) return ERR_IB;
      for (int k = 0; k < 4; ++k) w[k] = w[k] / s;
      ib.gcell.push_back(j * nx + i);
      for (int k = 0; k < 4; ++k) { ib.icell.push_back(cells[k]); ib.w.push_back(w[k]); }
      ib.nrm.push_back(nxv); ib.nrm.push_back(nyv);
    }
  }
  return OK;
}

// ---------------------------------------------------------------------------------------
// EOS and conversions (Sec. 2, EOS)
// ---------------------------------------------------------------------------------------
template <class T>
T energy(const T& r, const T& u, const T& v, const T& p, const T& gamma) {
  return p / (gamma - 1.0) + 0.5 * r * (u * u + v * v);
}
template <class T>
T pressure(const T& r, const T& u, const T& v, const T& E, const T& gamma) {
  return (gamma - 1.0) * (E - 0.5 * r * (u * u + v * v));
}

// ---------------------------------------------------------------------------------------
// WENO5 (Jiang-Shu): value at the right edge of cell c from cell averages a,b,c,d,e
// (cells c-2 .. c+2).  The left-edge value is the same routine on the mirrored stencil.
// ---------------------------------------------------------------------------------------
const double WENO_EPS = 1e-6;

template <class T>
void weno5_parts(const T& a, const T& b, const T& c, const T& d, const T& e, T beta[3], T p[3]) {
  const double k13 = 13.0 / 12.0;
  // smoothness indicators of the three candidate stencils
  const T s0 = a - 2.0 * b + c, t0 = a - 4.0 * b + 3.0 * c;
  const T s1 = b - 2.0 * c + d, t1 = b - d;
  const T s2 = c - 2.0 * d + e, t2 = 3.0 * c - 4.0 * d + e;
  beta[0] = k13 * s0 * s0 + 0.25 * t0 * t0;
  beta[1] = k13 * s1 * s1 + 0.25 * t1 * t1;
  beta[2] = k13 * s2 * s2 + 0.25 * t2 * t2;
  // candidate reconstructions at the right edge of the centre cell
  p[0] = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  p[1] = (-b + 5.0 * c + 2.0 * d) / 6.0;
  p[2] = (2.0 * c + 5.0 * d - e) / 6.0;
}

template <class T>
T weno5(const T& a, const T& b, const T& c, const T& d, const T& e, bool linear = false) {
  T beta[3], p[3];
  weno5_parts(a, b, c, d, e, beta, p);
  const double dlin[3] = {0.1, 0.6, 0.3};
  if (linear) return dlin[0] * p[0] + dlin[1] * p[1] + dlin[2] * p[2];
  T al[3];
  for (int k = 0; k < 3; ++k) {
    const T den = WENO_EPS + beta[k];
    al[k] = dlin[k] / (den * den);
  }
  const T sum = al[0] + al[1] + al[2];
  const T w0 = al[0] / sum, w1 = al[1] / sum, w2 = al[2] / sum;
  return w0 * p[0] + w1 * p[1] + w2 * p[2];
}

// ---------------------------------------------------------------------------------------
// HLLC flux in the normal direction (Sec. 2): states (rho, un, ut, p) on each side.
// Returns [mass, normal momentum, tangential momentum, energy] fluxes.
// ---------------------------------------------------------------------------------------
template <class T>
struct HllcDiag {
  T sL, sR, ss, UsL[4], UsR[4], UL[4], UR[4], FL[4], FR[4];
};

template <class T>
void hllc_side(const T& r, const T& u, const T& v, const T& p, const T& E, const T& s, const T& ss,
               int literal, T Uk[4], T Fk[4], T Us[4]) {
  Uk[0] = r; Uk[1] = r * u; Uk[2] = r * v; Uk[3] = E;
  Fk[0] = r * u; Fk[1] = r * u * u + p; Fk[2] = r * u * v; Fk[3] = u * (E + p);
  const T fac = (s - u) / (s - ss);
  Us[0] = fac * r;
  Us[1] = fac * (r * ss);
  Us[2] = fac * (r * v);
  if (literal)
    Us[3] = fac * (E * (s - ss) / (s - u) + (ss - u) * (r * ss - r * u * (s - ss) / (s - u)));
  else
    Us[3] = fac * (E + (ss - u) * (r * ss + p / (s - u)));
}

template <class T>
void hllc(const T& rL, const T& uL, const T& vL, const T& pL, const T& rR, const T& uR, const T& vR,
          const T& pR, const T& gamma, int literal, T F[4], HllcDiag<T>* diag = nullptr) {
  const T EL = energy(rL, uL, vL, pL, gamma);
  const T ER = energy(rR, uR, vR, pR, gamma);
  const T aL = sqrt(gamma * pL / rL);
  const T aR = sqrt(gamma * pR / rR);
  const T sL = tmin(uL - aL, uR - aR);
  const T sR = tmax(uL + aL, uR + aR);
  const T sm = tmin(T(0.0), sL);
  const T sp = tmax(T(0.0), sR);
  const T ss = (pR - pL + rL * uL * (sL - uL) - rR * uR * (sR - uR)) / (rL * (sL - uL) - rR * (sR - uR));
  T UkL[4], FkL[4], UsL[4], UkR[4], FkR[4], UsR[4];
  const bool needL = !(ss < 0.0), needR = !(ss > 0.0);
  if (needL) hllc_side(rL, uL, vL, pL, EL, sL, ss, literal, UkL, FkL, UsL);
  if (needR) hllc_side(rR, uR, vR, pR, ER, sR, ss, literal, UkR, FkR, UsR);
  for (int c = 0; c < 4; ++c) {
    // F = (1+sign s*)/2 [F^L + s^-(U*L - U^L)] + (1-sign s*)/2 [F^R + s^+(U*R - U^R)]
    if (ss > 0.0) F[c] = FkL[c] + sm * (UsL[c] - UkL[c]);
    else if (ss < 0.0) F[c] = FkR[c] + sp * (UsR[c] - UkR[c]);
    else F[c] = 0.5 * (FkL[c] + sm * (UsL[c] - UkL[c])) + 0.5 * (FkR[c] + sp * (UsR[c] - UkR[c]));
  }
  if (diag) {
    // diagnostics need both branches
    if (!needL) hllc_side(rL, uL, vL, pL, EL, sL, ss, literal, UkL, FkL, UsL);
    if (!needR) hllc_side(rR, uR, vR, pR, ER, sR, ss, literal, UkR, FkR, UsR);
    diag->sL = sL; diag->sR = sR; diag->ss = ss;
    for (int c = 0; c < 4; ++c) {
      diag->UsL[c] = UsL[c]; diag->UsR[c] = UsR[c]; diag->UL[c] = UkL[c]; diag->UR[c] = UkR[c];
      diag->FL[c] = FkL[c]; diag->FR[c] = FkR[c];
    }
  }
}

// ---------------------------------------------------------------------------------------
// the solver on a padded state
// ---------------------------------------------------------------------------------------
template <class T>
struct Solver {
  const or_grid& g;
  Par<T> P;
  const IbTable& ib;
  Layout L;
  bool parallel;
  std::vector<T> U[4];   // padded conserved state being evaluated
  std::vector<T> Q[4];   // padded primitives r,u,v,p
  std::vector<T> Fx[4];  // (nx+1)*ny x faces, face f between cells f-1 and f
  std::vector<T> Gy[4];  // nx*(ny+1) y faces

  Solver(const or_grid& g_, const Par<T>& P_, const IbTable& ib_, bool par)
      : g(g_), P(P_), ib(ib_), L(g_), parallel(par) {
    for (int c = 0; c < 4; ++c) {
      U[c].assign(L.size(), T(0.0));
      Q[c].assign(L.size(), T(0.0));
      Fx[c].assign((size_t)(g.nx + 1) * g.ny, T(0.0));
      if (g.ny > 1) Gy[c].assign((size_t)g.nx * (g.ny + 1), T(0.0));
    }
  }

  void load(const std::vector<T> src[4]) {  // src: nx*ny unpadded
    for (int c = 0; c < 4; ++c)
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) U[c][L.idx(i, j)] = src[c][(size_t)j * g.nx + i];
  }

  void cons_of_state(const T st[4], T out[4]) const {
    out[0] = st[0];
    out[1] = st[0] * st[1];
    out[2] = st[0] * st[2];
    out[3] = energy(st[0], st[1], st[2], st[3], P.gamma);
  }

  // immersed boundary: ghost states from image-point interpolation of fluid cells
  void ib_fill() {
    const size_t ng = ib.gcell.size();
    for (size_t k = 0; k < ng; ++k) {
      T q[4] = {T(0.0), T(0.0), T(0.0), T(0.0)};
      for (int m = 0; m < 4; ++m) {
        const int cell = ib.icell[4 * k + m];
        const double w = ib.w[4 * k + m];
        if (w == 0.0) continue;
        const int i = cell % g.nx, j = cell / g.nx;
        const long id = L.idx(i, j);
        const T r = U[0][id], u = U[1][id] / r, v = U[2][id] / r;
        const T p = pressure(r, u, v, U[3][id], P.gamma);
        q[0] = q[0] + w * r; q[1] = q[1] + w * u; q[2] = q[2] + w * v; q[3] = q[3] + w * p;
      }
      const double nxv = ib.nrm[2 * k], nyv = ib.nrm[2 * k + 1];
      T ug, vg;
      if (g.wall == 0) {  // slip: reverse the normal component, keep the tangential one
        const T vn = q[1] * nxv + q[2] * nyv;
        ug = q[1] - 2.0 * vn * nxv;
        vg = q[2] - 2.0 * vn * nyv;
      } else {            // no-slip
        ug = -q[1];
        vg = -q[2];
      }
      const T st[4] = {q[0], ug, vg, q[3]};
      T out[4];
      cons_of_state(st, out);
      const int i = ib.gcell[k] % g.nx, j = ib.gcell[k] / g.nx;
      for (int c = 0; c < 4; ++c) U[c][L.idx(i, j)] = out[c];
    }
  }

  // domain halo: x sides on interior rows, then y sides on the full padded width
  void bc_fill() {
    const int nx = g.nx, ny = g.ny;
    T inflow_cons[4][4];
    for (int s = 0; s < 4; ++s) cons_of_state(P.inflow[s], inflow_cons[s]);
    for (int j = 0; j < ny; ++j) {
      for (int k = 1; k <= NG; ++k) {
        // x-low ghost i = -k
        {
          const long dst = L.idx(-k, j);
          switch (g.bc[0]) {
            case BC_TRANSMISSIVE: for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(0, j)]; break;
            case BC_REFLECTIVE:
              for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(k - 1, j)];
              U[1][dst] = -U[1][dst]; break;
            case BC_PERIODIC: for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(nx - k, j)]; break;
            default: for (int c = 0; c < 4; ++c) U[c][dst] = inflow_cons[0][c]; break;
          }
        }
        // x-high ghost i = nx-1+k
        {
          const long dst = L.idx(nx - 1 + k, j);
          switch (g.bc[1]) {
            case BC_TRANSMISSIVE: for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(nx - 1, j)]; break;
            case BC_REFLECTIVE:
              for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(nx - k, j)];
              U[1][dst] = -U[1][dst]; break;
            case BC_PERIODIC: for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(k - 1, j)]; break;
            default: for (int c = 0; c < 4; ++c) U[c][dst] = inflow_cons[1][c]; break;
          }
        }
      }
    }
    if (ny == 1) return;
    for (int i = -NG; i < nx + NG; ++i) {
      for (int k = 1; k <= NG; ++k) {
        {
          const long dst = L.idx(i, -k);
          switch (g.bc[2]) {
            case BC_TRANSMISSIVE: for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(i, 0)]; break;
            case BC_REFLECTIVE:
              for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(i, k - 1)];
              U[2][dst] = -U[2][dst]; break;
            case BC_PERIODIC: for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(i, ny - k)]; break;
            default: for (int c = 0; c < 4; ++c) U[c][dst] = inflow_cons[2][c]; break;
          }
        }
        {
          const long dst = L.idx(i, ny - 1 + k);
          switch (g.bc[3]) {
            case BC_TRANSMISSIVE: for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(i, ny - 1)]; break;
            case BC_REFLECTIVE:
              for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(i, ny - k)];
              U[2][dst] = -U[2][dst]; break;
            case BC_PERIODIC: for (int c = 0; c < 4; ++c) U[c][dst] = U[c][L.idx(i, k - 1)]; break;
            default: for (int c = 0; c < 4; ++c) U[c][dst] = inflow_cons[3][c]; break;
          }
        }
      }
    }
  }

  bool fluid(int i, int j) const { return ib.tag.empty() || ib.tag[(size_t)j * g.nx + i] == 0; }

  // cons -> prim on the whole padded array; returns false if a fluid cell is non-physical
  bool primitives() {
    const long n = L.size();
    for (long id = 0; id < n; ++id) {
      const T r = U[0][id];
      const T u = U[1][id] / r, v = U[2][id] / r;
      Q[0][id] = r; Q[1][id] = u; Q[2][id] = v;
      Q[3][id] = pressure(r, u, v, U[3][id], P.gamma);
    }
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        if (!fluid(i, j)) continue;
        const long id = L.idx(i, j);
        const double r = val(Q[0][id]), p = val(Q[3][id]);
        if (!(r > 0.0) || !(p > 0.0) || !std::isfinite(r) || !std::isfinite(p)) return false;
      }
    return true;
  }

  // numerical + viscous flux through the face between padded ids il (left/low) and ir
  // (right/high).  dir 0: x face, stride 1; dir 1: y face, stride W.
  // wL, wR (optional): the WENO5 face states (primitive) before the positivity fallback
  void face_flux(long il, long ir, long stride, long tstride, int dir, T out[4], T* wL = nullptr, T* wR = nullptr) {
    T qL[4], qR[4];
    for (int c = 0; c < 4; ++c) {
      const std::vector<T>& q = Q[c];
      qL[c] = weno5(q[il - 2 * stride], q[il - stride], q[il], q[il + stride], q[il + 2 * stride]);
      qR[c] = weno5(q[ir + 2 * stride], q[ir + stride], q[ir], q[ir - stride], q[ir - 2 * stride]);
    }
    if (wL) for (int c = 0; c < 4; ++c) { wL[c] = qL[c]; wR[c] = qR[c]; }
    if (!(qL[0] > 0.0) || !(qL[3] > 0.0) || !(qR[0] > 0.0) || !(qR[3] > 0.0)) {
      // positivity fallback: first-order (cell) states at this face
      for (int c = 0; c < 4; ++c) { qL[c] = Q[c][il]; qR[c] = Q[c][ir]; }
#pragma omp atomic
      ++g_fallback_faces;
    }
    const int n = (dir == 0) ? 1 : 2, t = (dir == 0) ? 2 : 1;  // normal / tangential velocity
    T F[4];
    hllc(qL[0], qL[n], qL[t], qL[3], qR[0], qR[n], qR[t], qR[3], P.gamma, g.hllc_literal, F);
    out[0] = F[0]; out[n] = F[1]; out[t] = F[2]; out[3] = F[3];
    if (is_off(P.mu)) return;
    // viscous and heat fluxes (constant mu, Stokes hypothesis, T = p / rho)
    const double hn = (dir == 0) ? g.dx : g.dy;  // spacing normal to the face
    const double ht = (dir == 0) ? g.dy : g.dx;  // spacing along the face
    const bool has_t = (g.ny > 1);               // tangential derivatives exist in 2D only
    const T un_n = (Q[n][ir] - Q[n][il]) / hn;   // d(normal velocity)/dn
    const T ut_n = (Q[t][ir] - Q[t][il]) / hn;   // d(tangential velocity)/dn
    const T TL = Q[3][il] / Q[0][il], TR = Q[3][ir] / Q[0][ir];
    const T T_n = (TR - TL) / hn;
    T un_t(0.0), ut_t(0.0);
    if (has_t) {
      un_t = ((Q[n][il + tstride] - Q[n][il - tstride]) + (Q[n][ir + tstride] - Q[n][ir - tstride])) / (4.0 * ht);
      ut_t = ((Q[t][il + tstride] - Q[t][il - tstride]) + (Q[t][ir + tstride] - Q[t][ir - tstride])) / (4.0 * ht);
    }
    const T tau_nn = P.mu * ((4.0 / 3.0) * un_n - (2.0 / 3.0) * ut_t);
    const T tau_nt = P.mu * (ut_n + un_t);
    const T unb = 0.5 * (Q[n][il] + Q[n][ir]);
    const T utb = 0.5 * (Q[t][il] + Q[t][ir]);
    const T kappa = P.mu * P.gamma / ((P.gamma - 1.0) * P.Pr);
    out[n] = out[n] - tau_nn;
    out[t] = out[t] - tau_nt;
    out[3] = out[3] - (unb * tau_nn + utb * tau_nt + kappa * T_n);
  }

  // L(U) for the padded state U (filled in place); Lout: nx*ny per component
  int rhs(std::vector<T> Lout[4]) {
    ib_fill();
    bc_fill();
    if (!primitives()) return ERR_NONPHYSICAL;
    const int nx = g.nx, ny = g.ny;
    const long W = L.W;
    const bool nn = g_nn.on;
    // network input images, frame channels (rho, normal momentum, tangential momentum, E):
    // x faces as [4][ny][nx+1]; y faces transposed, [4][nx][ny+1], so that the second image
    // axis is always the face-normal one
    std::vector<T> Xx, Xy;
    if (nn) {
      Xx.assign((size_t)4 * ny * (nx + 1), T(0.0));
      if (ny > 1) Xy.assign((size_t)4 * nx * (ny + 1), T(0.0));
    }
    auto image_value = [&](const T wL[4], const T wR[4], int dir, T x[4]) {
      const int n = (dir == 0) ? 1 : 2, t = (dir == 0) ? 2 : 1;
      const T EL = energy(wL[0], wL[1], wL[2], wL[3], P.gamma), ER = energy(wR[0], wR[1], wR[2], wR[3], P.gamma);
      const T m[4] = {0.5 * (wL[0] + wR[0]), 0.5 * (wL[0] * wL[n] + wR[0] * wR[n]),
                      0.5 * (wL[0] * wL[t] + wR[0] * wR[t]), 0.5 * (EL + ER)};
      for (int c = 0; c < 4; ++c) x[c] = (m[c] - g_nn.mean[c]) / g_nn.sd[c];
    };
#pragma omp parallel for schedule(static) if (parallel)
    for (int j = 0; j < ny; ++j)
      for (int f = 0; f <= nx; ++f) {
        T out[4], wL[4], wR[4];
        face_flux(L.idx(f - 1, j), L.idx(f, j), 1, W, 0, out, nn ? wL : nullptr, nn ? wR : nullptr);
        for (int c = 0; c < 4; ++c) Fx[c][(size_t)j * (nx + 1) + f] = out[c];
        if (nn) {
          T x[4];
          image_value(wL, wR, 0, x);
          for (int c = 0; c < 4; ++c) Xx[((size_t)c * ny + j) * (nx + 1) + f] = x[c];
        }
      }
    if (ny > 1) {
#pragma omp parallel for schedule(static) if (parallel)
      for (int f = 0; f <= ny; ++f)
        for (int i = 0; i < nx; ++i) {
          T out[4], wL[4], wR[4];
          face_flux(L.idx(i, f - 1), L.idx(i, f), W, 1, 1, out, nn ? wL : nullptr, nn ? wR : nullptr);
          for (int c = 0; c < 4; ++c) Gy[c][(size_t)f * nx + i] = out[c];
          if (nn) {
            T x[4];
            image_value(wL, wR, 1, x);
            for (int c = 0; c < 4; ++c) Xy[((size_t)c * nx + i) * (ny + 1) + f] = x[c];
          }
        }
    }
    if (nn) {
      // neural flux added to the numerical flux of every face (same network both ways)
      const std::vector<T> Pn = nn_params<T>();
      std::vector<T> Y;
      nn_forward(Xx, ny, nx + 1, Pn, Y);
      const int fx[4] = {0, 1, 2, 3};  // conserved component of each frame channel, x faces
      for (int c = 0; c < 4; ++c)
        for (int j = 0; j < ny; ++j)
          for (int f = 0; f <= nx; ++f) {
            T& F = Fx[fx[c]][(size_t)j * (nx + 1) + f];
            F = F + Y[((size_t)c * ny + j) * (nx + 1) + f];
          }
      if (ny > 1) {
        nn_forward(Xy, nx, ny + 1, Pn, Y);
        const int fy[4] = {0, 2, 1, 3};  // y faces: normal momentum is rho v
        for (int c = 0; c < 4; ++c)
          for (int i = 0; i < nx; ++i)
            for (int f = 0; f <= ny; ++f) {
              T& G = Gy[fy[c]][(size_t)f * nx + i];
              G = G + Y[((size_t)c * nx + i) * (ny + 1) + f];
            }
      }
    }
    const bool av = !is_off(P.nu);
#pragma omp parallel for schedule(static) if (parallel)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t o = (size_t)j * nx + i;
        if (!fluid(i, j)) {
          for (int c = 0; c < 4; ++c) Lout[c][o] = T(0.0);
          continue;
        }
        const long id = L.idx(i, j);
        for (int c = 0; c < 4; ++c) {
          T r = -(Fx[c][(size_t)j * (nx + 1) + i + 1] - Fx[c][(size_t)j * (nx + 1) + i]) / g.dx;
          if (ny > 1) r = r - (Gy[c][(size_t)(j + 1) * nx + i] - Gy[c][(size_t)j * nx + i]) / g.dy;
          if (av) {
            T lap = (U[c][id + 1] - 2.0 * U[c][id] + U[c][id - 1]) / (g.dx * g.dx);
            if (ny > 1) lap = lap + (U[c][id + W] - 2.0 * U[c][id] + U[c][id - W]) / (g.dy * g.dy);
            r = r + P.nu * lap;
          }
          Lout[c][o] = r;
        }
      }
    return OK;
  }

  // maximum admissible dt on the unpadded state src (fluid cells only)
  T max_dt(const std::vector<T> src[4], double cfl) const {
    T rate(0.0), rmin(0.0);
    bool first = true;
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        if (!fluid(i, j)) continue;
        const size_t o = (size_t)j * g.nx + i;
        const T r = src[0][o], u = src[1][o] / r, v = src[2][o] / r;
        const T p = pressure(r, u, v, src[3][o], P.gamma);
        const T a = sqrt(P.gamma * p / r);
        T s = (tabs(u) + a) / g.dx;
        if (g.ny > 1) s = s + (tabs(v) + a) / g.dy;
        rate = first ? s : tmax(rate, s);
        rmin = first ? r : tmin(rmin, r);
        first = false;
      }
    T dt = cfl / rate;
    if (!is_off(P.mu)) {
      const double h = (g.ny > 1) ? (g.dx < g.dy ? g.dx : g.dy) : g.dx;
      const T dtv = cfl * h * h * rmin / (2.0 * P.mu * tmax(T(4.0 / 3.0), P.gamma / P.Pr));
      dt = tmin(dt, dtv);
    }
    return dt;
  }
};

// One SSP-RK3 step of the unpadded state Uc (nx*ny per component), in place.
template <class T>
int rk3_step(Solver<T>& S, std::vector<T> Uc[4], double dt) {
  const or_grid& g = S.g;
  const size_t n = (size_t)g.nx * g.ny;
  std::vector<T> U0[4], Us[4], Lv[4];
  for (int c = 0; c < 4; ++c) { U0[c] = Uc[c]; Us[c].resize(n); Lv[c].resize(n); }
  const double a[3] = {0.0, 0.75, 1.0 / 3.0};
  const double b[3] = {1.0, 0.25, 2.0 / 3.0};
  std::vector<T>* cur = U0;
  for (int s = 0; s < 3; ++s) {
    S.load(cur);
    const int rc = S.rhs(Lv);
    if (rc) return rc;
    // stage input after the immersed-boundary fill (non-fluid cells are carried over)
    std::vector<T> filled[4];
    for (int c = 0; c < 4; ++c) {
      filled[c].resize(n);
      for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) filled[c][(size_t)j * g.nx + i] = S.U[c][S.L.idx(i, j)];
    }
    for (int c = 0; c < 4; ++c)
      for (size_t o = 0; o < n; ++o) {
        const int i = (int)(o % g.nx), j = (int)(o / g.nx);
        if (!S.fluid(i, j)) { Us[c][o] = filled[c][o]; continue; }
        const T adv = filled[c][o] + dt * Lv[c][o];
        if (s == 0) Us[c][o] = adv;
        else Us[c][o] = a[s] * U0[c][o] + b[s] * adv;
      }
    for (int c = 0; c < 4; ++c) Uc[c] = Us[c];
    cur = Uc;
  }
  return OK;
}

template <class T>
void to_vec(const double* U, int nx, int ny, std::vector<T> out[4]) {
  const size_t n = (size_t)nx * ny;
  for (int c = 0; c < 4; ++c) {
    out[c].resize(n);
    for (size_t o = 0; o < n; ++o) out[c][o] = T(U[c * n + o]);
  }
}

bool grid_ok(const or_grid* g) {
  if (!g || g->nx < 6 || g->ny < 1) return false;
  if (g->ny > 1 && g->ny < 6) return false;
  if (!(g->dx > 0.0) || !(g->dy > 0.0)) return false;
  for (int s = 0; s < 4; ++s) if (g->bc[s] < 0 || g->bc[s] > 3) return false;
  return true;
}

int g_threads = 0;
void apply_threads() {
#ifdef _OPENMP
  if (g_threads > 0) omp_set_num_threads(g_threads);
#endif
}

}  // namespace

// =======================================================================================
// C ABI
// =======================================================================================
extern "C" {

void or_set_threads(int n) { g_threads = n; }

int or_get_threads(void) {
#ifdef _OPENMP
  apply_threads();
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int or_prim_to_cons(const or_grid* g, const double* theta, const double* W, double* U) {
  if (!grid_ok(g)) return ERR_ARG;
  const size_t n = (size_t)g->nx * g->ny;
  const double gamma = theta[0];
  for (size_t o = 0; o < n; ++o) {
    const double r = W[o], u = W[n + o], v = W[2 * n + o], p = W[3 * n + o];
    U[o] = r; U[n + o] = r * u; U[2 * n + o] = r * v; U[3 * n + o] = energy(r, u, v, p, gamma);
  }
  return OK;
}

int or_cons_to_prim(const or_grid* g, const double* theta, const double* U, double* W) {
  if (!grid_ok(g)) return ERR_ARG;
  const size_t n = (size_t)g->nx * g->ny;
  const double gamma = theta[0];
  for (size_t o = 0; o < n; ++o) {
    const double r = U[o], u = U[n + o] / r, v = U[2 * n + o] / r;
    W[o] = r; W[n + o] = u; W[2 * n + o] = v; W[3 * n + o] = pressure(r, u, v, U[3 * n + o], gamma);
  }
  return OK;
}

int or_ib_tables(const or_grid* g, const double* sdf, unsigned char* tag, int* nghost, int cap,
                 int* gcell, int* icell, double* w, double* nrm) {
  if (!grid_ok(g)) return ERR_ARG;
  IbTable ib;
  const int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  const size_t n = (size_t)g->nx * g->ny;
  if (tag) for (size_t o = 0; o < n; ++o) tag[o] = ib.tag.empty() ? 0 : ib.tag[o];
  const int ng = (int)ib.gcell.size();
  *nghost = ng;
  if (ng > cap) return OK;
  for (int k = 0; k < ng; ++k) {
    if (gcell) gcell[k] = ib.gcell[k];
    for (int m = 0; m < 4; ++m) {
      if (icell) icell[4 * k + m] = ib.icell[4 * k + m];
      if (w) w[4 * k + m] = ib.w[4 * k + m];
    }
    if (nrm) { nrm[2 * k] = ib.nrm[2 * k]; nrm[2 * k + 1] = ib.nrm[2 * k + 1]; }
  }
  return OK;
}

int or_rhs(const or_grid* g, const double* theta, const double* sdf, const double* U, double* Lout) {
  if (!grid_ok(g)) return ERR_ARG;
  apply_threads();
  IbTable ib;
  int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  Solver<double> S(*g, make_par<double>(theta), ib, true);
  std::vector<double> Uc[4], Lv[4];
  to_vec<double>(U, g->nx, g->ny, Uc);
  const size_t n = (size_t)g->nx * g->ny;
  for (int c = 0; c < 4; ++c) Lv[c].resize(n);
  S.load(Uc);
  rc = S.rhs(Lv);
  if (rc) return rc;
  for (int c = 0; c < 4; ++c) std::memcpy(Lout + c * n, Lv[c].data(), n * sizeof(double));
  return OK;
}

int or_step(const or_grid* g, const double* theta, const double* sdf, double* U, const double* dts,
            int nsteps) {
  if (!grid_ok(g) || nsteps < 0) return ERR_ARG;
  apply_threads();
  IbTable ib;
  int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  Solver<double> S(*g, make_par<double>(theta), ib, true);
  std::vector<double> Uc[4];
  to_vec<double>(U, g->nx, g->ny, Uc);
  for (int k = 0; k < nsteps; ++k) {
    rc = rk3_step(S, Uc, dts[k]);
    if (rc) return rc;
  }
  const size_t n = (size_t)g->nx * g->ny;
  for (int c = 0; c < 4; ++c) std::memcpy(U + c * n, Uc[c].data(), n * sizeof(double));
  return OK;
}

int or_max_dt(const or_grid* g, const double* theta, const double* sdf, const double* U, double cfl,
              double* dt) {
  if (!grid_ok(g)) return ERR_ARG;
  IbTable ib;
  int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  Solver<double> S(*g, make_par<double>(theta), ib, false);
  std::vector<double> Uc[4];
  to_vec<double>(U, g->nx, g->ny, Uc);
  *dt = S.max_dt(Uc, cfl);
  return OK;
}

// CFL-driven run to t_end, last step clipped; dts_out (capacity max_steps) receives the dt
// sequence actually used.
int or_run_to(const or_grid* g, const double* theta, const double* sdf, double* U, double cfl,
              double t_end, int max_steps, double* dts_out, int* nsteps_out) {
  if (!grid_ok(g)) return ERR_ARG;
  apply_threads();
  IbTable ib;
  int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  Solver<double> S(*g, make_par<double>(theta), ib, true);
  std::vector<double> Uc[4];
  to_vec<double>(U, g->nx, g->ny, Uc);
  double t = 0.0;
  int k = 0;
  while (t < t_end && k < max_steps) {
    double dt = S.max_dt(Uc, cfl);
    if (t + dt > t_end) dt = t_end - t;
    rc = rk3_step(S, Uc, dt);
    if (rc) return rc;
    if (dts_out) dts_out[k] = dt;
    t = t + dt;
    ++k;
  }
  *nsteps_out = k;
  const size_t n = (size_t)g->nx * g->ny;
  for (int c = 0; c < 4; ++c) std::memcpy(U + c * n, Uc[c].data(), n * sizeof(double));
  return OK;
}

// Forward-mode derivative of the RHS: tangent dU of the state and dtheta of the parameters.
int or_rhs_tangent(const or_grid* g, const double* theta, const double* dtheta, const double* sdf,
                   const double* U, const double* dU, double* Lout, double* dLout) {
  if (!grid_ok(g)) return ERR_ARG;
  apply_threads();
  typedef Dual<1> D;
  IbTable ib;
  int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  Par<D> P = make_par<D>(theta);
  P.gamma.d[0] = dtheta[0]; P.mu.d[0] = dtheta[1]; P.Pr.d[0] = dtheta[2]; P.nu.d[0] = dtheta[3];
  for (int s = 0; s < 4; ++s) for (int c = 0; c < 4; ++c) P.inflow[s][c].d[0] = dtheta[4 + 4 * s + c];
  Solver<D> S(*g, P, ib, true);
  const size_t n = (size_t)g->nx * g->ny;
  std::vector<D> Uc[4], Lv[4];
  for (int c = 0; c < 4; ++c) {
    Uc[c].resize(n); Lv[c].resize(n);
    for (size_t o = 0; o < n; ++o) { Uc[c][o] = D(U[c * n + o]); Uc[c][o].d[0] = dU[c * n + o]; }
  }
  S.load(Uc);
  rc = S.rhs(Lv);
  if (rc) return rc;
  for (int c = 0; c < 4; ++c)
    for (size_t o = 0; o < n; ++o) { Lout[c * n + o] = Lv[c][o].v; dLout[c * n + o] = Lv[c][o].d[0]; }
  return OK;
}

// Forward-mode derivative of nsteps SSP-RK3 steps with fixed dts; U and dU updated in place.
int or_step_tangent(const or_grid* g, const double* theta, const double* dtheta, const double* sdf,
                    double* U, double* dU, const double* dts, int nsteps) {
  if (!grid_ok(g) || nsteps < 0) return ERR_ARG;
  apply_threads();
  typedef Dual<1> D;
  IbTable ib;
  int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  Par<D> P = make_par<D>(theta);
  P.gamma.d[0] = dtheta[0]; P.mu.d[0] = dtheta[1]; P.Pr.d[0] = dtheta[2]; P.nu.d[0] = dtheta[3];
  for (int s = 0; s < 4; ++s) for (int c = 0; c < 4; ++c) P.inflow[s][c].d[0] = dtheta[4 + 4 * s + c];
  Solver<D> S(*g, P, ib, true);
  const size_t n = (size_t)g->nx * g->ny;
  std::vector<D> Uc[4];
  for (int c = 0; c < 4; ++c) {
    Uc[c].resize(n);
    for (size_t o = 0; o < n; ++o) { Uc[c][o] = D(U[c * n + o]); Uc[c][o].d[0] = dU[c * n + o]; }
  }
  for (int k = 0; k < nsteps; ++k) {
    rc = rk3_step(S, Uc, dts[k]);
    if (rc) return rc;
  }
  for (int c = 0; c < 4; ++c)
    for (size_t o = 0; o < n; ++o) { U[c * n + o] = Uc[c][o].v; dU[c * n + o] = Uc[c][o].d[0]; }
  return OK;
}

// Neural flux: w = NN_NPARAM parameters (NULL switches the network off), dw = their tangent
// for the *_tangent calls (NULL: zero), norm = mean[4], sd[4], scale[4] of the frame channels.
// The setting applies to every later call.
int or_nn_set(const double* w, const double* dw, const double* norm) {
  if (!w) { g_nn.on = false; g_nn.w.clear(); g_nn.dw.clear(); return OK; }
  if (!norm) return ERR_ARG;
  for (int c = 0; c < 4; ++c) if (!(norm[4 + c] > 0.0)) return ERR_ARG;
  g_nn.w.assign(w, w + NN_NPARAM);
  if (dw) g_nn.dw.assign(dw, dw + NN_NPARAM); else g_nn.dw.clear();
  for (int c = 0; c < 4; ++c) { g_nn.mean[c] = norm[c]; g_nn.sd[c] = norm[4 + c]; g_nn.scale[c] = norm[8 + c]; }
  g_nn.on = true;
  return OK;
}

int or_nn_nparam(void) { return NN_NPARAM; }

// The network alone on one image X[4][H][W] -> Y[4][H][W] (uses the parameters of or_nn_set).
int or_nn_eval(const double* X, int H, int Wd, double* Y) {
  if (!g_nn.on || H < 1 || Wd < 1) return ERR_ARG;
  std::vector<double> x(X, X + (size_t)4 * H * Wd), y;
  nn_forward(x, H, Wd, nn_params<double>(), y);
  std::copy(y.begin(), y.end(), Y);
  return OK;
}

// Operation tally of one RHS evaluation: out = [add, mul, div, sqrt, cmp] (add includes sub).
int or_count_rhs(const or_grid* g, const double* theta, const double* sdf, const double* U,
                 long long* out) {
  if (!grid_ok(g)) return ERR_ARG;
  IbTable ib;
  int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  Solver<Cnt> S(*g, make_par<Cnt>(theta), ib, false);
  const size_t n = (size_t)g->nx * g->ny;
  std::vector<Cnt> Uc[4], Lv[4];
  for (int c = 0; c < 4; ++c) {
    Uc[c].resize(n); Lv[c].resize(n);
    for (size_t o = 0; o < n; ++o) Uc[c][o] = Cnt(U[c * n + o]);
  }
  S.load(Uc);
  g_tally = OpTally{0, 0, 0, 0, 0};
  rc = S.rhs(Lv);
  out[0] = g_tally.add; out[1] = g_tally.mul; out[2] = g_tally.div; out[3] = g_tally.sqrt; out[4] = g_tally.cmp;
  return rc;
}

// Number of faces at which the positivity fallback was taken since the last call (every RHS
// evaluation of every entry point counts); resets the count.
long long or_fallback_faces(void) {
  const long long n = g_fallback_faces;
  g_fallback_faces = 0;
  return n;
}

// The immersed-boundary ghost fill alone (Sec. 2, Fig. 1(c)): U (unpadded [4][ny][nx]) with
// every ghost cell replaced by the slip-wall (or no-slip) mirror of the interpolated image-point
// state, written to out; other cells are copied.
int or_ib_fill(const or_grid* g, const double* theta, const double* sdf, const double* U, double* out) {
  if (!grid_ok(g)) return ERR_ARG;
  IbTable ib;
  int rc = build_ib(*g, sdf, ib);
  if (rc) return rc;
  Solver<double> S(*g, make_par<double>(theta), ib, false);
  std::vector<double> Uc[4];
  to_vec<double>(U, g->nx, g->ny, Uc);
  S.load(Uc);
  S.ib_fill();
  const size_t n = (size_t)g->nx * g->ny;
  for (int c = 0; c < 4; ++c)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) out[c * n + (size_t)j * g->nx + i] = S.U[c][S.L.idx(i, j)];
  return OK;
}

// ---- building blocks exposed for the pins -------------------------------------------------
void or_weno5(const double* q, int linear, double* out) {
  *out = weno5(q[0], q[1], q[2], q[3], q[4], linear != 0);
}
void or_weno5_beta(const double* q, double* beta) {
  double p[3];
  weno5_parts(q[0], q[1], q[2], q[3], q[4], beta, p);
}
// diag (27): sL, sR, s*, U*L[4], U*R[4], UL[4], UR[4], FL[4], FR[4]
void or_hllc(const double* qL, const double* qR, double gamma, int literal, double* F, double* diag) {
  HllcDiag<double> d;
  hllc(qL[0], qL[1], qL[2], qL[3], qR[0], qR[1], qR[2], qR[3], gamma, literal, F, diag ? &d : nullptr);
  if (diag) {
    diag[0] = d.sL; diag[1] = d.sR; diag[2] = d.ss;
    for (int c = 0; c < 4; ++c) {
      diag[3 + c] = d.UsL[c]; diag[7 + c] = d.UsR[c]; diag[11 + c] = d.UL[c]; diag[15 + c] = d.UR[c];
      diag[19 + c] = d.FL[c]; diag[23 + c] = d.FR[c];
    }
  }
}

// ---- exact Riemann solver for the 1D Euler equations (textbook: Newton on the pressure
// function, then self-similar sampling).  Used to pin the Sod shock tube of Sec. 3. ---------
static void pfun(double p, double rk, double pk, double ak, double gamma, double* f, double* df) {
  if (p > pk) {
    const double A = 2.0 / ((gamma + 1.0) * rk), B = (gamma - 1.0) / (gamma + 1.0) * pk;
    const double q = std::sqrt(A / (p + B));
    *f = (p - pk) * q;
    *df = q * (1.0 - 0.5 * (p - pk) / (B + p));
  } else {
    const double pr = p / pk;
    *f = 2.0 * ak / (gamma - 1.0) * (std::pow(pr, (gamma - 1.0) / (2.0 * gamma)) - 1.0);
    *df = 1.0 / (rk * ak) * std::pow(pr, -(gamma + 1.0) / (2.0 * gamma));
  }
}

int or_exact_riemann(double rl, double ul, double pl, double rr, double ur, double pr, double gamma,
                     double xdisc, double t, const double* x, int n, double* ro, double* uo, double* po,
                     double* star) {
  const double al = std::sqrt(gamma * pl / rl), ar = std::sqrt(gamma * pr / rr);
  if (2.0 * al / (gamma - 1.0) + 2.0 * ar / (gamma - 1.0) <= ur - ul) return ERR_ARG;  // vacuum
  double p = 0.5 * (pl + pr);
  for (int it = 0; it < 200; ++it) {
    double fl, dfl, fr, dfr;
    pfun(p, rl, pl, al, gamma, &fl, &dfl);
    pfun(p, rr, pr, ar, gamma, &fr, &dfr);
    double pn = p - (fl + fr + ur - ul) / (dfl + dfr);
    if (pn < 1e-14) pn = 1e-14;
    const double change = std::fabs(pn - p) / (0.5 * (pn + p));
    p = pn;
    if (change < 1e-15) break;
  }
  double fl, dfl, fr, dfr;
  pfun(p, rl, pl, al, gamma, &fl, &dfl);
  pfun(p, rr, pr, ar, gamma, &fr, &dfr);
  const double us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  const double g1 = (gamma - 1.0) / (gamma + 1.0);
  const double rsl = (p > pl) ? rl * ((p / pl + g1) / (g1 * p / pl + 1.0)) : rl * std::pow(p / pl, 1.0 / gamma);
  const double rsr = (p > pr) ? rr * ((p / pr + g1) / (g1 * p / pr + 1.0)) : rr * std::pow(p / pr, 1.0 / gamma);
  if (star) { star[0] = p; star[1] = us; star[2] = rsl; star[3] = rsr; }
  for (int k = 0; k < n; ++k) {
    const double S = (t > 0.0) ? (x[k] - xdisc) / t : ((x[k] < xdisc) ? -1e300 : 1e300);
    double r, u, pp;
    if (S <= us) {  // left of the contact
      if (p > pl) {  // left shock
        const double sl = ul - al * std::sqrt((gamma + 1.0) / (2.0 * gamma) * p / pl + (gamma - 1.0) / (2.0 * gamma));
        if (S <= sl) { r = rl; u = ul; pp = pl; } else { r = rsl; u = us; pp = p; }
      } else {       // left rarefaction
        const double shl = ul - al, asl = al * std::pow(p / pl, (gamma - 1.0) / (2.0 * gamma)), stl = us - asl;
        if (S <= shl) { r = rl; u = ul; pp = pl; }
        else if (S > stl) { r = rsl; u = us; pp = p; }
        else {
          u = 2.0 / (gamma + 1.0) * (al + 0.5 * (gamma - 1.0) * ul + S);
          const double c = 2.0 / (gamma + 1.0) + (gamma - 1.0) / ((gamma + 1.0) * al) * (ul - S);
          r = rl * std::pow(c, 2.0 / (gamma - 1.0));
          pp = pl * std::pow(c, 2.0 * gamma / (gamma - 1.0));
        }
      }
    } else {         // right of the contact
      if (p > pr) {  // right shock
        const double sr = ur + ar * std::sqrt((gamma + 1.0) / (2.0 * gamma) * p / pr + (gamma - 1.0) / (2.0 * gamma));
        if (S >= sr) { r = rr; u = ur; pp = pr; } else { r = rsr; u = us; pp = p; }
      } else {       // right rarefaction
        const double shr = ur + ar, asr = ar * std::pow(p / pr, (gamma - 1.0) / (2.0 * gamma)), str = us + asr;
        if (S >= shr) { r = rr; u = ur; pp = pr; }
        else if (S <= str) { r = rsr; u = us; pp = p; }
        else {
          u = 2.0 / (gamma + 1.0) * (-ar + 0.5 * (gamma - 1.0) * ur + S);
          const double c = 2.0 / (gamma + 1.0) - (gamma - 1.0) / ((gamma + 1.0) * ar) * (ur - S);
          r = rr * std::pow(c, 2.0 / (gamma - 1.0));
          pp = pr * std::pow(c, 2.0 * gamma / (gamma - 1.0));
        }
      }
    }
    ro[k] = r; uo[k] = u; po[k] = pp;
  }
  return OK;
}

}  // extern "C"
