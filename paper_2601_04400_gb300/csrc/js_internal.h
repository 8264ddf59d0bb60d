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
  int* err;                  // device error flag
  Lay lay;
  double gamma, gm1, g1;
  double cx, cy;             // dt/dx, dt/dy (stage) or 1/dx, 1/dy (RHS)
  double rk_a, rk_b;         // out = rk_a U^n + rk_b (U_s + dt L(U_s))
  double avx, avy;           // (dt) nu / dx^2, (dt) nu / dy^2
  ViscC vx, vy;              // viscous constants of x and y faces
  int use_un, has_av;
};

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

cudaError_t launch_stage(const StageArgs& a, bool visc, bool rhs, cudaStream_t s);
cudaError_t launch_bc_fill(double* U, const Lay& lay, const BcArgs& bc, cudaStream_t s);
cudaError_t launch_ib_fill(double* U, const Lay& lay, const IbArgs& ib, double gamma, int wall, cudaStream_t s);
cudaError_t launch_pack(const double* U, double* P, const Lay& lay, cudaStream_t s);
cudaError_t launch_unpack(const double* P, double* U, const Lay& lay, cudaStream_t s);
cudaError_t launch_prim_to_cons(const double* W, double* U, long long n, double gamma, cudaStream_t s);
cudaError_t launch_cfl(const double* U, const Lay& lay, const unsigned char* tag, double gamma, double dx,
                       double dy, unsigned long long* red, cudaStream_t s);

}  // namespace js
