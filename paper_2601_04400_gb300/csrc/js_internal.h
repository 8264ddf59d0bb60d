// Internal launch arguments shared by the kernels and the host side of libjaxshock.so.
#pragma once
#include <cuda_runtime.h>

#include "js_device.cuh"

namespace js {

struct StageArgs {
  const double* Uin;         // padded stage input (halo and IB ghosts filled)
  const double* Un;          // padded U^n (RK combination), may alias Uout
  double* Uout;              // padded stage output, or [4][ny][nx] in RHS mode
  const unsigned char* tag;  // [ny][nx] cell tags (0 fluid) or nullptr
  double* acc;               // [4][ny][nx] scratch: x-flux differences of the stage
  double* acc2;              // [4][ny][nx] scratch: y-flux differences (concurrent sweeps)
  int* err;                  // device error flag
  Lay lay;
  double gamma, gm1, g1;
  double cx, cy;             // dt/dx, dt/dy (stage) or 1/dx, 1/dy (RHS)
  double rk_a, rk_b;         // out = rk_a U^n + rk_b (U_s + dt L(U_s))
  double avx, avy;           // (dt) nu / dx^2, (dt) nu / dy^2
  ViscC vx, vy;              // viscous constants of x and y faces
  int use_un, has_av;
  // WENO5 internals for the reverse pass (kernels instantiated with SAVE): 56 planes of
  // `splane` doubles, x lines transposed (row pitch tpitch), y lines in the padded layout
  double* wsave;
  long long splane;
  int tpitch;
  // device-resident step size (js_step_cfl): when set, cx, cy, avx, avy are read from
  // dtc[0..3] at kernel start, and dtc[4] == 0 means the step is inactive (skip the stage)
  const double* dtc;
  // neural flux (kernels instantiated with IMG): the face images of the stage input, FP32
  // [4][ny][nx+1] (x faces) then [4][nx][ny+1] (y faces), normalised by img_mean / img_isd
  float* img;
  float img_mean[4], img_isd[4], img_g1;
};

// the per-step constants of a device step size dt: dtc = {dt/dx, dt/dy, dt nu/dx^2,
// dt nu/dy^2, active, dt}
constexpr int DTC_N = 6;

struct BcArgs {
  int kind[4];
  double inflow_cons[4][4];  // conserved inflow states per side
};

struct IbArgs {
  int n;                     // ghost cells
  const long long* dst;      // padded index of each ghost cell
  const long long* src;      // 4 padded indices of the interpolation cells
  const double* w;           // 4 weights (0 for non-fluid cells)
  const double* nrm;         // unit normal (2)
};

// transposed IB fill: for each fluid source cell, the ghosts that interpolate from it
struct IbTArgs {
  int nsrc;
  const long long* cell;     // padded index of each source cell
  const int* ptr;            // nsrc + 1 offsets into ghost / w
  const int* ghost;          // ghost number
  const double* w;           // its weight
};

// reverse-mode launch arguments (js_adjoint.cu)
struct AdjArgs {
  Lay lay;
  const double* X;           // padded filled stage state (4 planes)
  double* Q;                 // padded primitives rho, u, v, p, T (5 planes)
  double* lam;               // padded lambda' (4 planes), zero outside fluid cells
  double* Ub;                // padded conserved adjoints of X (4 planes)
  double* wsave;             // WENO internals [dir][var][7] planes of splane doubles
  double* fadj;              // face-state adjoints [dir][left/right][var] planes of splane
  long long splane;          // plane size of wsave / fadj (>= both layouts below)
  int tpitch;                // x-direction planes are stored transposed: (i+3)*tpitch + j+gy
  double* pbar;              // parameter gradient (JS_NPARAM) or nullptr
  const unsigned char* tag;
  Gas gas;
  double inv_dx, inv_dy;     // 1/dx, 1/dy
  double nu_x, nu_y;         // nu/dx^2, nu/dy^2
  double nu_x1, nu_y1;       // 1/dx^2, 1/dy^2
  ViscC vx, vy;
  double inv_mu, kg, kp;     // 1/mu, -1/(gamma (gamma-1)), -1/Pr
  int visc, has_av, two_d;
  int weno_saved;            // wsave already holds the stage's WENO internals (forward SAVE)
  // deterministic reverse (no floating-point atomics: every sum in a fixed order)
  double* fcell;             // per face [dir][12] planes of splane: adjoints that go straight to
                             //   the two cells of the face (positivity fallback, viscous terms:
                             //   left cell rho,u,v,p,T at 0-4, right cell at 5-9, tangential
                             //   derivative terms at 10-11)
  double* wrev;              // pass-2 output slots [dir][4][seg][SL][line] (WENO5 reverse)
  double* pp;                // block partials of pbar[0..3] of the current launch (4 per block)
};

// pass-2 segment length (cells per thread along a line) and slot length of wrev
constexpr int ADJ_SEG2 = 8, ADJ_SEG2_1D = 4;
// doubles of the wrev slots of a grid, and of the parameter-gradient block partials of one
// reverse stage (bounds; nn_blocks = blocks of the neural image reverse, 0 without it)
long long adj_wrev_doubles(const Lay& lay);
long long adj_ppart_doubles(const Lay& lay, int n_ghost, int n_src, long long nn_blocks);
// blocks of the neural image-reverse kernel for a grid (one partial each)
long long nn_image_vjp_blocks(const Lay& lay);

// ---------------------------------------------------------------------------------------
// neural flux (Sec. 2.3): three 3x3 convolution layers 4 -> 16 -> 32 -> 4 (ReLU, ReLU, tanh)
// over the face images of each direction (x faces [C][ny][nx+1]; y faces transposed,
// [C][nx][ny+1]); parameter blocks (weights [co][ci][3][3] then biases) at NN_OFF*
// ---------------------------------------------------------------------------------------
constexpr int NN_NPARAM = 6388;
constexpr int NN_OFF1 = 0, NN_OFF2 = 592, NN_OFF3 = 5232;

struct NnArgs {
  Lay lay;
  int fp32;                   // network arithmetic: 0 FP64, 1 FP32
  int nimg;                   // face images: 1 (1D: x faces only) or 2
  int H[2], W[2];             // image extents (lines x faces per line)
  long long pix0;             // H[0] * W[0]: image 1 starts at C * pix0 in a C-channel buffer
  const double* w;            // parameters (device, NN_NPARAM)
  double* w_bar;              // accumulated parameter gradient or nullptr
  double mean[4], inv_sd[4], scale[4];  // frame channels (rho, normal mom., tangential mom., E)
  double g1;                  // 1/(gamma - 1)
  void* X;                    // 4-channel network input
  void* A1;                   // 16-channel activations of layer 1
  void* A2;                   // 32-channel activations of layer 2
  void* T3;                   // 4-channel tanh outputs (unscaled)
  void* G4;                   // 4-channel gradient scratch
  void* G16;                  // 16-channel gradient scratch
  void* G32;                  // 32-channel gradient scratch
  double* partial;            // weight-gradient partial sums [nwblk][NN_NPARAM]
  int nwblk;
  // WENO5 internals of the stage (2D, layout of StageArgs::wsave) to form the face states
  // from, or nullptr: the image kernels then recompute WENO5
  const double* wsave;
  long long splane;
  int tpitch;
  int bf16;                   // layers 2 and 3 on the tensor cores (BF16 operands, FP32 accumulate)
  void* A1h;                  // BF16 copies of the activations of layers 1 and 2, pixel-major with
  void* A2h;                  //   the channels contiguous ([image][H][W][C]), tensor-core inputs
  int* err;                   // device error flag (bounded waits of the tensor-core layers)
  int keep;                   // 1: the FP32 activations A1, A2 are written (a reverse pass reads
                              //   them); 0: BF16 forward-only stages skip them
  int fwd_ready;              // reverse: X, A1, A2, T3 of this stage's forward are in place
  int fused;                  // BF16 forward-only stages: the whole network in one launch
};

// forward: images of the stage input (primitives Q, plane qplane) and the network, into T3
cudaError_t nn_forward(const NnArgs& n, const double* Q, long long qplane, cudaStream_t s);
// primitive variables of every padded cell of U into Q (4 planes)
cudaError_t nn_prims(const double* U, double* Q, const Lay& lay, double gamma, cudaStream_t s);
// the network alone on the face images already in n.X, into T3 (forward)
cudaError_t nn_layers(const NnArgs& n, cudaStream_t s);
// stage output (or RHS) minus the divergence of the neural flux held in T3
cudaError_t nn_apply(const NnArgs& n, const StageArgs& a, bool rhs, cudaStream_t s);
// reverse: recompute the network on a.Q, seed with the face-flux adjoints of a.lam, back-
// propagate (parameter gradient into n.w_bar), add the face-state adjoints to a.fadj
cudaError_t nn_reverse(const NnArgs& n, const AdjArgs& a, cudaStream_t s);
// the network alone on one image X[4][H][W] (FP64, device) -> scaled output Y[4][H][W]
cudaError_t nn_eval(const NnArgs& n, const double* X, int H, int W, double* Y, cudaStream_t s);
cudaError_t nn_eval_vjp(const NnArgs& n, const double* X, int H, int W, const double* GY, double* GX,
                        cudaStream_t s);
// out[4][ny/fy][nx/fx] = means of fx x fy blocks of U[4][ny][nx]
cudaError_t launch_block_average(const double* U, int nx, int ny, int fx, int fy, double* out, cudaStream_t s);

// nn: the neural flux's reverse (run between pass 1 and pass 2) or nullptr
// inflow_part: [4 sides][max(nx + 6, ny)][4] partial sums of the inflow halo adjoints
cudaError_t launch_adj_stage(const AdjArgs& a, const BcArgs& bc, const IbArgs& ib, const IbTArgs& ibt, int wall,
                             const double* Unext, double* Uacc, double ra, double rb, double dt, bool rhs_mode,
                             double* inflow_part, const double* inflow_prim, double* qIb, cudaStream_t s,
                             long long* launches, const NnArgs* nn = nullptr);
cudaError_t launch_adj_unpack(const double* P, const double* P2, double* U, const Lay& lay, cudaStream_t s);

// one instance of the batched kernel (js_batch.cu), filled from a context by js_internal_desc
struct InstDesc {
  Lay lay;
  double* N;
  double* A;
  double* B;
  double* U;                 // user state [4][ny][nx]
  double* acc;               // stage scratch [4][ny][nx]
  double* acc2;
  const unsigned char* tag;
  IbArgs ib;
  BcArgs bc;
  double gamma, mu, Pr, nu, dx, dy;
  double hmin, lim;          // viscous dt cap: cfl hmin^2 rho_min / (2 mu lim)
  ViscC vx, vy;
  int wall, visc, has_av, ntx, nty;
};

// reverse-pass description of one instance for the persistent batched reverse kernel
// (js_batch.cu): the context's adjoint arguments and workspace (js_internal_rev_desc) and the
// instance's work-item counts and parameter-gradient slot offsets (set by js_batch.cu)
struct InstRev {
  AdjArgs a;                 // X, Ub, pbar, pp, wsave, weno_saved are set per phase
  IbTArgs ibt;
  double* P0;                // adjoint ping-pong states (4 padded planes each)
  double* P1;
  double* Uacc;              // U^n part of the step's adjoint (4 padded planes)
  double* wsave_own;         // WENO5 internals recomputed by pass 1 (stage 2)
  double* wfwd;              // internals stored by the forward stages 0 and 1 (2 x 56 planes)
  double* inflow_part;
  const double* inflow_prim;
  double* qIb;
  double* ppart;             // warp partials of the parameter gradient
  int tmax;                  // max(nx + 6, ny): inflow_part row length
  int seg1_re, seg1_sv, seg2;  // pass-1 segment lengths (recompute / stored internals), pass 2
  long long xpad_re, xpad_sv, xpad_p2;  // x-line items of passes 1 and 2, rounded up to 32
  long long w1_re, w1_sv;    // warp slots of pass 1 (both directions)
  long long off_prim, w_prim, off_g, w_g, off_s, w_s;  // slots of primvjp, IB ghost, IB source
};

// opaque 128-byte, 64-byte aligned tensor map (CUtensorMap) for TMA copies
struct alignas(64) TensorMap128 {
  unsigned long long opaque[16];
};

// box of the TMA-staged stage tile (32x32 cells + 3-cell halo, 4 planes)
constexpr int TMA_TX = 32, TMA_TY = 32;

// IEEE-order arithmetic mode (js_ieee.cu): padded primitives Q (4 planes of lay.plane),
// x-face fluxes F [4][ny][nx+1], y-face fluxes G [4][ny+1][nx]
struct IeeeBufs {
  double* Q;
  double* F;
  double* G;
};
cudaError_t launch_ieee_ib_fill(double* U, const Lay& lay, const IbArgs& ib, double gamma, int wall, cudaStream_t s);
// one stage (RHS mode: a.Uout = L(a.Uin) in [4][ny][nx]) from the filled padded input a.Uin
cudaError_t launch_ieee_stage(const StageArgs& a, const IeeeBufs& b, double dt, int stage, bool rhs, double mu,
                              double Pr, double nu, double dx, double dy, cudaStream_t s);
// (a.dtc set: dt = a.dtc[5], and the stage does nothing when a.dtc[4] == 0)

constexpr int STAGE_VARIANTS = 5;
cudaError_t launch_stage(const StageArgs& a, bool visc, bool rhs, int variant, const TensorMap128* tmap,
                         cudaStream_t s);
// stage update (not RHS mode) that also stores the WENO5 internals to a.wsave (2D only;
// 32x32 concurrent tile, TMA-staged when tmap is given)
cudaError_t launch_stage_save(const StageArgs& a, bool visc, const TensorMap128* tmap, cudaStream_t s);
// stage update that also writes the neural flux's face images of its input to a.img (2D)
cudaError_t launch_stage_img(const StageArgs& a, bool visc, const TensorMap128* tmap, cudaStream_t s);
cudaError_t launch_bc_fill(double* U, const Lay& lay, const BcArgs& bc, cudaStream_t s);
cudaError_t launch_ib_fill(double* U, const Lay& lay, const IbArgs& ib, double gamma, int wall, cudaStream_t s);
cudaError_t launch_pack(const double* U, double* P, const Lay& lay, cudaStream_t s);
cudaError_t launch_unpack(const double* P, double* U, const Lay& lay, cudaStream_t s);
cudaError_t launch_prim_to_cons(const double* W, double* U, long long n, double gamma, cudaStream_t s);
// rows [row0, row0 + nrows) of the 4 planes of a [4][ny][nx] array <-> a [4][nrows][nx] buffer
// (pack: zero != 0 also clears those rows of U; unpack: add != 0 adds instead of copying)
cudaError_t launch_rows_pack(double* U, int nx, int ny, int row0, int nrows, double* buf, int zero, cudaStream_t s);
cudaError_t launch_rows_unpack(double* U, int nx, int ny, int row0, int nrows, const double* buf, int add,
                               cudaStream_t s);
// CFL reduction of U (user layout): red[0] = bits of the largest rate, red[1] = bits of the
// smallest density over fluid cells (red: 3 words; bmax: CFL_MAX_BLOCKS doubles of scratch)
constexpr int CFL_MAX_BLOCKS = 152 * 8;
// the step size of the reduction in red on the device (js_max_dt's arithmetic; viscous cap when
// mu > 0 with lim = max(4/3, gamma/Pr), hmin = min(dx, dy) in 2D), clipped to t_end with the
// running time t (or t == nullptr), into the stage constants dtc[DTC_N] and dt_log[k]
cudaError_t launch_cfl_dt(const unsigned long long* red, double cfl, double dx, double dy, double nu, double mu,
                          double lim, double hmin, double* t, double t_end, double* dtc, double* dt_log, int k,
                          int* err, cudaStream_t s);
// (padded: U is a context's padded buffer, e.g. the state N between the steps of js_step_cfl)
cudaError_t launch_cfl(const double* U, const Lay& lay, const unsigned char* tag, double gamma, double dx,
                       double dy, unsigned long long* red, double* bmax, cudaStream_t s, bool padded = false);

}  // namespace js
