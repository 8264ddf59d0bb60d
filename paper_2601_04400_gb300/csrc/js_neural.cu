// Neural flux (arXiv 2601.04400, Sec. 2.3): a fully convolutional network of three 3x3
// layers with zero ("SAME") padding, 4 -> 16 -> 32 -> 4 channels, ReLU, ReLU, tanh (6388
// parameters), evaluated on the face images of each direction and added to the HLLC flux;
// the update of Sec. 2.3 then takes the divergence of F_HLLC + F_neural.
//
// Face image of direction d (d = 0: x faces as [C][ny][nx+1]; d = 1: y faces transposed,
// [C][nx][ny+1], so that the second axis is always the face-normal one and both directions
// share the network): pixel (line h, face f) holds the normalised mean of the two WENO5 face
// states of face f in conserved variables of the face frame (rho, normal momentum,
// tangential momentum, E).  The network's output channel k, times scale[k], is the neural
// flux of frame component k through that face.
//
// Forward per stage: primitives -> images -> three convolution launches (T3 = tanh output)
// -> the fused stage kernel (HLLC part) -> nn_apply subtracts the neural flux divergence.
// Reverse per stage: the images and activations are recomputed from the stage state; the
// seed is the face-flux adjoint (lambda'_right - lambda'_left)/h (the same as for the HLLC
// flux); three data-gradient launches (ReLU masks fused), three weight-gradient launches
// (per-block partial sums, reduced in a fixed order, so the parameter gradient is
// reproducible) and the image reverse, which adds the face-state adjoints to the WENO5
// reverse's inputs and d/dgamma of the face energies to the parameter gradient.
//
// Arithmetic type T: double (FP64, the oracle's precision) or float (FP32 on the CUDA
// cores; the network is a dense contraction of 6336 multiply-adds per face, which FP64
// would make about 20x the cost of the FP64 solver it corrects).  BF16 precision (float
// buffers): the forward's three layers on the tensor cores, BF16 operands, FP32 accumulation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "js_device.cuh"
#include "js_internal.h"
#include "js_stage.cuh"  // smem_u32, mbar_init, mbar_wait

namespace js {

namespace {

constexpr int TILE = 16;            // pixels per tile side; one thread per pixel
constexpr int TH = TILE + 2;        // tile with its 1-pixel halo
constexpr int NTHR = TILE * TILE;

template <class T>
__device__ __forceinline__ T* chan_img(void* base, int C, int d, long long pix0) {
  return static_cast<T*>(base) + (d == 0 ? 0LL : (long long)C * pix0);
}
template <class T>
__device__ __forceinline__ const T* chan_img(const void* base, int C, int d, long long pix0) {
  return static_cast<const T*>(base) + (d == 0 ? 0LL : (long long)C * pix0);
}

__device__ __forceinline__ double act_tanh(double x) { return tanh(x); }
__device__ __forceinline__ float act_tanh(float x) { return tanhf(x); }

// two floats rounded to BF16 (to nearest even) and packed, lo in the low half; eight of them as
// one 16-byte value (built in registers, not through a local array)
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}
__device__ __forceinline__ uint4 pack_bf16x8(const float v[8]) {
  return make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                    pack_bf16x2(v[6], v[7]));
}

// WENO5 face states (primitive, before any positivity fallback) of face f of line h in
// direction d: left-biased from cell f-1, right-biased from cell f (the stage kernel's
// formulation, so the same values)
__device__ __forceinline__ void face_states(const Lay& L, const double* Q, long long qplane, int d, int h, int f,
                                            double wl[4], double wr[4]) {
  const long long st = (d == 0) ? 1 : L.pitch;
  const long long cf = (d == 0) ? L.idx(f, h) : L.idx(h, f);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double* q = Q + c * qplane + cf;
    const double qm3 = q[-3 * st], qm2 = q[-2 * st], qm1 = q[-st], q0 = q[0], qp1 = q[st], qp2 = q[2 * st];
    double dummy;
    Win a;
    a.init(qm3, qm2, qm1, q0);
    a.step<true, false>(qp1, wl[c], dummy);
    Win b;
    b.init(qm2, qm1, q0, qp1);
    b.step<false, true>(qp2, dummy, wr[c]);
  }
}

// the same face states from the stage's stored WENO5 internals: state = q_cell + q/6 with the
// quotient q saved for the left-biased state of cell f-1 and the right-biased one of cell f
__device__ __forceinline__ void face_states_saved(const NnArgs& n, const Lay& L, const double* Q, long long qplane,
                                                  int d, int h, int f, double wl[4], double wr[4]) {
  const long long ca = (d == 0) ? L.idx(f - 1, h) : L.idx(h, f - 1);
  const long long cb = (d == 0) ? L.idx(f, h) : L.idx(h, f);
  const long long sa = (d == 0) ? (long long)(f + 2) * n.tpitch + (h + L.gy) : ca;
  const long long sb = (d == 0) ? (long long)(f + 3) * n.tpitch + (h + L.gy) : cb;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double* sv = n.wsave + (long long)(d * 28 + c * 7) * n.splane;
    wl[c] = fma(sv[3 * n.splane + sa], SIXTH, Q[c * qplane + ca]);
    wr[c] = fma(sv[5 * n.splane + sb], SIXTH, Q[c * qplane + cb]);
  }
}

__device__ __forceinline__ void face_states_any(const NnArgs& n, const Lay& L, const double* Q, long long qplane,
                                                int d, int h, int f, double wl[4], double wr[4]) {
  if (n.wsave) face_states_saved(n, L, Q, qplane, d, h, f, wl, wr);
  else face_states(L, Q, qplane, d, h, f, wl, wr);
}

// ---------------------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------------------
__global__ void nn_prims_kernel(const double* __restrict__ U, double* __restrict__ Q, Lay L, Gas g) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.plane) return;
  const int col = (int)(t % L.pitch), row = (int)(t / L.pitch);
  if (col >= L.nx + 6 || row >= L.H) return;
  double u, v, p, T;
  const double r = U[t];
  cons_to_prim(r, U[L.plane + t], U[2 * L.plane + t], U[3 * L.plane + t], g, u, v, p, T);
  Q[t] = r;
  Q[L.plane + t] = u;
  Q[2 * L.plane + t] = v;
  Q[3 * L.plane + t] = p;
}

// The image kernels work on 32 x 32 tiles of (line h, face f) pixels: the FP64 face-state
// arithmetic runs with consecutive threads on consecutive lines, the direction along which the
// stage's stored WENO5 internals and the face adjoints are contiguous in both directions, and the
// image values (contiguous along f) pass through a shared-memory tile.
constexpr int IT = 32;

template <class T>
__global__ void __launch_bounds__(256) nn_image_kernel(NnArgs n, const double* __restrict__ Q, long long qplane) {
  __shared__ T sx[4][IT][IT + 1];
  const int d = blockIdx.z;
  const int H = n.H[d], Wd = n.W[d];
  const int f0 = blockIdx.x * IT, h0 = blockIdx.y * IT;
  if (f0 >= Wd || h0 >= H) return;  // uniform per block
  const long long pix = (long long)H * Wd;
  const int hl = threadIdx.x % IT;
  const int un = (d == 0) ? 1 : 2, ut = (d == 0) ? 2 : 1;
  T mean[4], isd[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    mean[k] = (T)n.mean[k];
    isd[k] = (T)n.inv_sd[k];
  }
  for (int fl = threadIdx.x / IT; fl < IT; fl += 256 / IT) {
    const int h = h0 + hl, f = f0 + fl;
    if (h >= H || f >= Wd) continue;
    double wl[4], wr[4];
    T m[4];
    face_states_any(n, n.lay, Q, qplane, d, h, f, wl, wr);
    face_image<T>(wl, wr, un, ut, (T)n.g1, mean, isd, m);
#pragma unroll
    for (int k = 0; k < 4; ++k) sx[k][hl][fl] = m[k];
  }
  __syncthreads();
  T* X = chan_img<T>(n.X, 4, d, n.pix0);
  for (int e = threadIdx.x; e < 4 * IT * IT; e += 256) {
    const int k = e / (IT * IT), r = e % (IT * IT), h = h0 + r / IT, f = f0 + r % IT;
    if (h < H && f < Wd) X[k * pix + (long long)h * Wd + f] = sx[k][r / IT][r % IT];
  }
}

// one 3x3 layer on a 16x16 pixel tile per block; ACT 0: ReLU, 1: tanh
template <class T, int CIN, int COUT, int ACT>
__global__ void __launch_bounds__(NTHR) nn_conv_kernel(NnArgs n, const void* in, void* out, int woff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = COUT * CIN * 9 + COUT;
  T* sw = reinterpret_cast<T*>(smem_raw);
  T* sx = sw + ((NW + 1) & ~1);
  const int d = blockIdx.z;
  const int H = n.H[d], Wd = n.W[d];
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
  if (x0 >= Wd || y0 >= H) return;  // the grid covers the larger image
  const long long pix = (long long)H * Wd;
  const T* X = chan_img<T>(in, CIN, d, n.pix0);
  T* Y = chan_img<T>(out, COUT, d, n.pix0);
  for (int k = threadIdx.x; k < NW; k += NTHR) sw[k] = (T)n.w[woff + k];
  for (int k = threadIdx.x; k < CIN * TH * TH; k += NTHR) {
    const int ci = k / (TH * TH), r = k % (TH * TH);
    const int gy = y0 + r / TH - 1, gx = x0 + r % TH - 1;
    sx[k] = (gy >= 0 && gy < H && gx >= 0 && gx < Wd) ? X[ci * pix + (long long)gy * Wd + gx] : (T)0;
  }
  __syncthreads();
  const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
  T acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = sw[COUT * CIN * 9 + co];
  for (int ci = 0; ci < CIN; ++ci)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const T v = sx[ci * TH * TH + (ty + ky) * TH + tx + kx];
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fma(sw[((co * CIN + ci) * 3 + ky) * 3 + kx], v, acc[co]);
      }
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < Wd && gy < H) {
    const long long o = (long long)gy * Wd + gx;
#pragma unroll
    for (int co = 0; co < COUT; ++co) Y[co * pix + o] = (ACT == 0) ? (acc[co] > (T)0 ? acc[co] : (T)0) : act_tanh(acc[co]);
  }
}

// FP32 layer with register blocking: 128 threads per 16x16 tile, each computing 2 adjacent
// pixels for all output channels; weights tap-major with the output channels contiguous, so
// one 16-byte shared load feeds 8 fused multiply-adds
constexpr int PB = 2;                 // pixels per thread (along the tile row)
constexpr int NTHR_F = NTHR / PB;     // 128

template <int CIN, int COUT, int ACT>
__global__ void __launch_bounds__(NTHR_F) nn_conv_f32_kernel(NnArgs n, const void* in, void* out, int woff,
                                                             void* outh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  static_assert(COUT % 4 == 0, "output channels in groups of 4");
  float* sw = reinterpret_cast<float*>(smem_raw);  // [CIN*9][COUT]
  float* sb = sw + CIN * 9 * COUT;                  // [COUT]
  float* sx = sb + COUT;                            // [CIN][18][18]
  const int d = blockIdx.z;
  const int H = n.H[d], Wd = n.W[d];
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
  if (x0 >= Wd || y0 >= H) return;
  const long long pix = (long long)H * Wd;
  const float* X = chan_img<float>(in, CIN, d, n.pix0);
  float* Y = out ? chan_img<float>(out, COUT, d, n.pix0) : nullptr;  // FP32 output (optional)
  for (int k = threadIdx.x; k < COUT * CIN * 9; k += NTHR_F) {
    const int co = k / (CIN * 9), r = k % (CIN * 9);
    sw[r * COUT + co] = (float)n.w[woff + k];
  }
  for (int k = threadIdx.x; k < COUT; k += NTHR_F) sb[k] = (float)n.w[woff + COUT * CIN * 9 + k];
  for (int k = threadIdx.x; k < CIN * TH * TH; k += NTHR_F) {
    const int ci = k / (TH * TH), r = k % (TH * TH);
    const int gy = y0 + r / TH - 1, gx = x0 + r % TH - 1;
    sx[k] = (gy >= 0 && gy < H && gx >= 0 && gx < Wd) ? X[ci * pix + (long long)gy * Wd + gx] : 0.0f;
  }
  __syncthreads();
  const int ty = threadIdx.x / (TILE / PB), tx0 = (threadIdx.x % (TILE / PB)) * PB;
  float acc[PB][COUT];
#pragma unroll
  for (int q = 0; q < PB; ++q)
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[q][co] = sb[co];
  for (int ci = 0; ci < CIN; ++ci)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const float* row = sx + ci * TH * TH + (ty + ky) * TH + tx0;
      float x[PB + 2];
#pragma unroll
      for (int j = 0; j < PB + 2; ++j) x[j] = row[j];
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const float4* w4 = reinterpret_cast<const float4*>(sw + ((ci * 3 + ky) * 3 + kx) * COUT);
#pragma unroll
        for (int c4 = 0; c4 < COUT / 4; ++c4) {
          const float4 wv = w4[c4];
#pragma unroll
          for (int q = 0; q < PB; ++q) {
            const float v = x[q + kx];
            acc[q][4 * c4 + 0] = fmaf(wv.x, v, acc[q][4 * c4 + 0]);
            acc[q][4 * c4 + 1] = fmaf(wv.y, v, acc[q][4 * c4 + 1]);
            acc[q][4 * c4 + 2] = fmaf(wv.z, v, acc[q][4 * c4 + 2]);
            acc[q][4 * c4 + 3] = fmaf(wv.w, v, acc[q][4 * c4 + 3]);
          }
        }
      }
    }
  const int gy = y0 + ty;
#pragma unroll
  for (int q = 0; q < PB; ++q) {
    const int gx = x0 + tx0 + q;
    if (gx < Wd && gy < H) {
      const long long o = (long long)gy * Wd + gx;
#pragma unroll
      for (int co = 0; co < COUT; ++co) {
        const float v = acc[q][co];
        acc[q][co] = (ACT == 0) ? (v > 0.0f ? v : 0.0f) : tanhf(v);
        if (Y) Y[co * pix + o] = acc[q][co];
      }
      if (outh) {
        // BF16 pixel-major copy (the tensor-core layer's input), 8 channels per 16-byte store
        __nv_bfloat16* Yh = static_cast<__nv_bfloat16*>(outh) + (d == 0 ? 0LL : (long long)COUT * n.pix0);
#pragma unroll
        for (int c8 = 0; c8 < COUT / 8; ++c8) {
          *reinterpret_cast<uint4*>(Yh + o * COUT + 8 * c8) = pack_bf16x8(&acc[q][8 * c8]);
        }
      }
    }
  }
}

// FP32 data gradient with the same blocking: weights [co][ky][kx][ci], input channels
// contiguous; the ReLU mask of the layer below is applied when MASK
template <int CIN, int COUT, bool MASK>
__global__ void __launch_bounds__(NTHR_F) nn_dgrad_f32_kernel(NnArgs n, const void* gout, const void* aprev, void* gin,
                                                              int woff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  static_assert(CIN % 4 == 0, "input channels in groups of 4");
  float* sw = reinterpret_cast<float*>(smem_raw);  // [COUT*9][CIN]
  float* sg = sw + COUT * 9 * CIN;                  // [COUT][18][18]
  const int d = blockIdx.z;
  const int H = n.H[d], Wd = n.W[d];
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
  if (x0 >= Wd || y0 >= H) return;
  const long long pix = (long long)H * Wd;
  const float* G = chan_img<float>(gout, COUT, d, n.pix0);
  float* D = chan_img<float>(gin, CIN, d, n.pix0);
  for (int k = threadIdx.x; k < COUT * CIN * 9; k += NTHR_F) {
    const int co = k / (CIN * 9), r = k % (CIN * 9), ci = r / 9, t = r % 9;
    sw[(co * 9 + t) * CIN + ci] = (float)n.w[woff + k];
  }
  for (int k = threadIdx.x; k < COUT * TH * TH; k += NTHR_F) {
    const int co = k / (TH * TH), r = k % (TH * TH);
    const int gy = y0 + r / TH - 1, gx = x0 + r % TH - 1;
    sg[k] = (gy >= 0 && gy < H && gx >= 0 && gx < Wd) ? G[co * pix + (long long)gy * Wd + gx] : 0.0f;
  }
  __syncthreads();
  const int ty = threadIdx.x / (TILE / PB), tx0 = (threadIdx.x % (TILE / PB)) * PB;
  float acc[PB][CIN];
#pragma unroll
  for (int q = 0; q < PB; ++q)
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[q][ci] = 0.0f;
  for (int co = 0; co < COUT; ++co)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      // gout at (ty - ky + 1, tx - kx + 1): tile row ty - ky + 2, columns tx0 .. tx0 + 5
      const float* row = sg + co * TH * TH + (ty - ky + 2) * TH + tx0;
      float x[PB + 2];
#pragma unroll
      for (int j = 0; j < PB + 2; ++j) x[j] = row[j];
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const float4* w4 = reinterpret_cast<const float4*>(sw + ((co * 3 + ky) * 3 + kx) * CIN);
#pragma unroll
        for (int c4 = 0; c4 < CIN / 4; ++c4) {
          const float4 wv = w4[c4];
#pragma unroll
          for (int q = 0; q < PB; ++q) {
            const float v = x[q + 2 - kx];
            acc[q][4 * c4 + 0] = fmaf(wv.x, v, acc[q][4 * c4 + 0]);
            acc[q][4 * c4 + 1] = fmaf(wv.y, v, acc[q][4 * c4 + 1]);
            acc[q][4 * c4 + 2] = fmaf(wv.z, v, acc[q][4 * c4 + 2]);
            acc[q][4 * c4 + 3] = fmaf(wv.w, v, acc[q][4 * c4 + 3]);
          }
        }
      }
    }
  const int gy = y0 + ty;
  const float* A = MASK ? chan_img<float>(aprev, CIN, d, n.pix0) : nullptr;
#pragma unroll
  for (int q = 0; q < PB; ++q) {
    const int gx = x0 + tx0 + q;
    if (gx < Wd && gy < H) {
      const long long o = (long long)gy * Wd + gx;
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) {
        float v = acc[q][ci];
        if (MASK && !(A[ci * pix + o] > 0.0f)) v = 0.0f;
        D[ci * pix + o] = v;
      }
    }
  }
}

// FP32 weight gradient: a work item is (group of 4 output channels, input channel, kernel
// row) with 4 x 3 sums (the three kernel columns); per pixel one 16-byte load of the output
// gradient and one input value slid along the row.  The tile's 16 rows are split into R
// parts so that every thread carries exactly 3 (item, part) units (NI * R = 768 for the three
// layers); the parts, and the bias sums (every thread sums a strided subset of the tile's
// pixels for one channel), are added in shared memory in a fixed order at the end.
constexpr int WG_UNITS = 3 * NTHR;

// 4-byte asynchronous global -> shared copy (zero-filled, nothing read, when !valid; src must
// still be a valid address), and its group commit / wait
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int CIN, int COUT>
__host__ __device__ constexpr int wgrad_tile_floats() {
  return NTHR * COUT + CIN * TH * TH;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(NTHR) nn_wgrad_f32_kernel(NnArgs n, const void* gout, const void* ain, int woff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NI = (COUT / 4) * CIN * 3;          // work items
  constexpr int R = WG_UNITS / NI;                  // row parts per item
  static_assert(NI * R == WG_UNITS && TILE % R == 0 && NTHR % COUT == 0, "work split");
  constexpr int RROWS = TILE / R;
  constexpr int TF = wgrad_tile_floats<CIN, COUT>();
  // two tile buffers, each [256 pixels][COUT] output gradient + [CIN][18][18] input: the next
  // tile is copied asynchronously while the current one is summed
  float* const buf0 = reinterpret_cast<float*>(smem_raw);
  float acc[3][12];
  float bacc = 0.0f;                                // bias: channel tid % COUT, pixels tid / COUT + k * (NTHR / COUT)
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[u][k] = 0.0f;
  int ntx[2], nty[2];
  for (int d = 0; d < 2; ++d) {
    ntx[d] = (d < n.nimg) ? (n.W[d] + TILE - 1) / TILE : 0;
    nty[d] = (d < n.nimg) ? (n.H[d] + TILE - 1) / TILE : 0;
  }
  const int t0 = ntx[0] * nty[0], total = t0 + ntx[1] * nty[1];
  // output gradient tile, pixel-major: pixel r's channel group c4 (4 channels, 16 bytes) at
  // group slot c4 ^ (r mod COUT/4), which spreads a warp's accesses of one group over the banks
  auto fetch = [&](int t, float* sg) {
    float* sa = sg + NTHR * COUT;
    const int d = (t < t0) ? 0 : 1;
    const int tl = (d == 0) ? t : t - t0;
    const int x0 = (tl % ntx[d]) * TILE, y0 = (tl / ntx[d]) * TILE;
    const int H = n.H[d], Wd = n.W[d];
    const long long pix = (long long)H * Wd;
    const float* G = chan_img<float>(gout, COUT, d, n.pix0);
    const float* A = chan_img<float>(ain, CIN, d, n.pix0);
    for (int k = threadIdx.x; k < (COUT / 4) * NTHR; k += NTHR) {
      const int c4 = k / NTHR, r = k % NTHR;
      const int gy = y0 + r / TILE, gx = x0 + r % TILE;
      const bool in = gy < H && gx < Wd;
      const long long o = in ? (long long)gy * Wd + gx : 0;
      float* dst = sg + 4 * (r * (COUT / 4) + (c4 ^ (r % (COUT / 4))));
#pragma unroll
      for (int j = 0; j < 4; ++j) cp_async4(dst + j, G + (4 * c4 + j) * pix + o, in);
    }
    for (int k = threadIdx.x; k < CIN * TH * TH; k += NTHR) {
      const int ci = k / (TH * TH), r = k % (TH * TH);
      const int gy = y0 + r / TH - 1, gx = x0 + r % TH - 1;
      const bool in = gy >= 0 && gy < H && gx >= 0 && gx < Wd;
      cp_async4(sa + k, A + ci * pix + (in ? (long long)gy * Wd + gx : 0), in);
    }
  };
  int cur = 0;
  if ((int)blockIdx.x < total) fetch(blockIdx.x, buf0);
  cp_async_commit();
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int tn = t + gridDim.x;
    if (tn < total) fetch(tn, buf0 + (cur ^ 1) * TF);
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of tile t are done
    __syncthreads();     // and everyone's
    const float* sg = buf0 + cur * TF;
    const float* sa = sg + NTHR * COUT;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int unit = threadIdx.x + u * NTHR;
      const int item = unit % NI, part = unit / NI;
      const int c4 = item / (CIN * 3), rem = item % (CIN * 3), ci = rem / 3, ky = rem % 3;
      for (int py = part * RROWS; py < (part + 1) * RROWS; ++py) {
        const float* arow = sa + ci * TH * TH + (py + ky) * TH;
        const float4* g4 = reinterpret_cast<const float4*>(sg + py * TILE * COUT);
        float a0 = arow[0], a1 = arow[1];
#pragma unroll
        for (int px = 0; px < TILE; ++px) {
          const float a2 = arow[px + 2];
          const float4 g = g4[px * (COUT / 4) + (c4 ^ ((py * TILE + px) % (COUT / 4)))];
          acc[u][0] = fmaf(g.x, a0, acc[u][0]);
          acc[u][1] = fmaf(g.y, a0, acc[u][1]);
          acc[u][2] = fmaf(g.z, a0, acc[u][2]);
          acc[u][3] = fmaf(g.w, a0, acc[u][3]);
          acc[u][4] = fmaf(g.x, a1, acc[u][4]);
          acc[u][5] = fmaf(g.y, a1, acc[u][5]);
          acc[u][6] = fmaf(g.z, a1, acc[u][6]);
          acc[u][7] = fmaf(g.w, a1, acc[u][7]);
          acc[u][8] = fmaf(g.x, a2, acc[u][8]);
          acc[u][9] = fmaf(g.y, a2, acc[u][9]);
          acc[u][10] = fmaf(g.z, a2, acc[u][10]);
          acc[u][11] = fmaf(g.w, a2, acc[u][11]);
          a0 = a1;
          a1 = a2;
        }
      }
    }
    {
      const int co = threadIdx.x % COUT, c4 = co / 4, j = co % 4;
      for (int q = threadIdx.x / COUT; q < NTHR; q += NTHR / COUT)
        bacc += sg[(q * (COUT / 4) + (c4 ^ (q % (COUT / 4)))) * 4 + j];
    }
    __syncthreads();  // tile t is read: its buffer takes tile t + 2 gridDim.x next
    cur ^= 1;
  }
  cp_async_wait<0>();
  // block sums: (item, part) units and bias partials through shared memory, added in part order
  __syncthreads();
  float* red = reinterpret_cast<float*>(smem_raw);  // [WG_UNITS][12], then [NTHR] bias partials
  float* bred = red + WG_UNITS * 12;
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int k = 0; k < 12; ++k) red[(threadIdx.x + u * NTHR) * 12 + k] = acc[u][k];
  bred[threadIdx.x] = bacc;
  __syncthreads();
  double* part = n.partial + (long long)blockIdx.x * NN_NPARAM + woff;
  for (int e = threadIdx.x; e < NI * 12; e += NTHR) {
    const int item = e / 12, k = e % 12;
    float sum = 0.0f;
    for (int pr = 0; pr < R; ++pr) sum += red[(pr * NI + item) * 12 + k];
    const int c4 = item / (CIN * 3), rem = item % (CIN * 3), ci = rem / 3, ky = rem % 3;
    const int kx = k / 4, jj = k % 4;
    part[(((4 * c4 + jj) * CIN + ci) * 3 + ky) * 3 + kx] = (double)sum;
  }
  if (threadIdx.x < COUT) {
    float sum = 0.0f;
    for (int q = 0; q < NTHR / COUT; ++q) sum += bred[q * COUT + threadIdx.x];
    part[COUT * CIN * 9 + threadIdx.x] = (double)sum;
  }
}

// ---------------------------------------------------------------------------------------
// BF16 tensor-core layer (tcgen05): a 3x3 convolution as an implicit GEMM
//   D[pixel][co] = sum over taps (ky, kx) and input channels ci of
//                  A_tap[pixel][ci] * W_tap[co][ci],   A_tap[pixel] = input[pixel + (ky-1, kx-1)]
// A block computes M = 128 consecutive pixels of one image row.  The haloed input rows (3 x 130
// pixels) sit in shared memory as BF16 in the no-swizzle K-major core-matrix layout
// [channel group of 8][row][column][8 channels] (a core matrix = 8 consecutive pixels x 16 bytes),
// so every tap's A operand is the same buffer at a shifted start address; the weights per tap as
// [channel group][co][8 channels].  One thread issues, per tap and group of 16 channels, a
// tcgen05.mma (kind::f16, M = 128, N = output channels rounded up to 16, K = 16) accumulating in
// FP32 in tensor memory; tcgen05.commit signals an mbarrier (bounded wait); each warp then reads
// its 32 accumulator lanes with tcgen05.ld and applies bias and activation.
// ---------------------------------------------------------------------------------------
constexpr int TC_M = 128;                 // pixels per block
constexpr int TC_COLS = TC_M + 2;         // with the halo
// shared bytes of the input row ring of a layer with CIN input channels: 4 rows x 130 pixels x
// CIN channels, BF16 (sized per layer, so that the narrower layers fit more blocks per SM)
constexpr int TC_NSLOT = 4;
__host__ __device__ constexpr int tc_aregion(int cin) { return TC_NSLOT * (cin / 8) * TC_COLS * 16; }

// 16-byte asynchronous global -> shared copy (zero-filled, nothing read, when !valid)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;   // leading (K-direction) core-matrix offset
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;   // stride (M/N-direction) 8-row-group offset
  d |= (uint64_t)1 << 46;                        // descriptor version of tcgen05; no swizzle
  return d;
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// A block owns work items of one 128-pixel-wide column strip and TC_ROWS output rows.  It loads
// the weights and allocates tensor memory once, then walks its rows keeping its input rows in a
// ring of four row slots: while the MMAs of output row h (input rows h-1, h, h+1) run and its
// epilogue stores it, the asynchronous 16-byte copies of input row h+2 (8 channels of a pixel
// each) fill the slot of row h-2.
constexpr int TC_ROWS = 16;

// MODE 0: a layer's forward (bias, then ReLU for ACT 0, tanh for ACT 1).  MODE 1: a layer's data
// gradient, the same implicit GEMM over the output gradient with the weights transposed and
// flipped, gin[ci] = sum over taps and co of w[co][ci][2-ky][2-kx] gout[co](pixel + (ky-1, kx-1)),
// times the ReLU mask (aprev > 0) of the layer below for ACT 1.  CINR <= CIN: channels present
// in the input (the rest are zero padding up to the MMA's K of 16; the first layer's 4).
template <int CIN, int COUT, int ACT, int MODE = 0, int CINR = CIN>
__global__ void __launch_bounds__(128) nn_conv_tc_kernel(NnArgs n, const void* inh, void* out, int woff,
                                                         void* outh, const void* aprev) {
  static_assert(CIN % 16 == 0, "input channels in groups of 16 (K of one MMA)");
  static_assert(CINR <= CIN, "present channels within the padded ones");
  constexpr int N = (COUT + 15) / 16 * 16;   // MMA N (multiple of 16 for M = 128)
  constexpr int KG = CIN / 8;                // 8-channel groups
  constexpr int GSTRIDE = TC_COLS * 16;      // bytes of one channel group of one row slot
  constexpr int SLOT = KG * GSTRIDE;         // bytes of one input row slot
  constexpr int BTAP = KG * N * 16;          // bytes of one tap of the weights
  constexpr int AREGION = tc_aregion(CIN);
  static_assert(TC_NSLOT * SLOT <= AREGION, "row slots");
  extern __shared__ __align__(16) unsigned char smem_raw[];  // 16-byte rows: no swizzle
  unsigned char* sA = smem_raw;
  unsigned char* sB = smem_raw + AREGION;
  float* sbias = reinterpret_cast<float*>(sB + 9 * BTAP);
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tmem_base;
  int nxs[2], nys[2];
  for (int d = 0; d < 2; ++d) {
    nxs[d] = (d < n.nimg) ? (n.W[d] + TC_M - 1) / TC_M : 0;
    nys[d] = (d < n.nimg) ? (n.H[d] + TC_ROWS - 1) / TC_ROWS : 0;
  }
  const int items0 = nxs[0] * nys[0], items = items0 + nxs[1] * nys[1];
  if ((int)blockIdx.x >= items) return;  // uniform per block, before any allocation
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
  }
  __nv_bfloat16* B16 = reinterpret_cast<__nv_bfloat16*>(sB);
  for (int k = tid; k < 9 * CIN * N; k += 128) {
    const int tap = k / (CIN * N), r = k % (CIN * N), ci = r / N, co = r % N;
    float v = 0.0f;
    if (co < COUT && ci < CINR)
      v = (MODE == 0) ? (float)n.w[woff + (co * CINR + ci) * 9 + tap] : (float)n.w[woff + (ci * COUT + co) * 9 + 8 - tap];
    B16[tap * (BTAP / 2) + ((ci >> 3) * N + co) * 8 + (ci & 7)] = __float2bfloat16_rn(v);
  }
  if (MODE == 0)
    for (int k = tid; k < COUT; k += 128) sbias[k] = (float)n.w[woff + COUT * CINR * 9 + k];
  __syncthreads();
  const uint32_t tmem = tmem_base;
  const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
  constexpr uint32_t idesc = umma_idesc_bf16(TC_M, N);
  constexpr long long kBudget = 2000000000LL;  // about one second of SM clock
  unsigned phase0 = 0u, phase1 = 0u;  // mbarrier phases of bar[0], bar[1] (scalars: no local memory)
  bool ok = true;
  for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
    const int d = (it < items0) ? 0 : 1;
    const int il = (d == 0) ? it : it - items0;
    const int x0 = (il % nxs[d]) * TC_M, h0 = (il / nxs[d]) * TC_ROWS;
    const int H = n.H[d], Wd = n.W[d];
    const int h1 = (h0 + TC_ROWS < H) ? h0 + TC_ROWS : H;
    const long long pix = (long long)H * Wd;
    const uint4* Xh = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(inh) +
                                                     (d == 0 ? 0LL : (long long)CIN * n.pix0));
    float* Y = out ? chan_img<float>(out, COUT, d, n.pix0) : nullptr;  // FP32 output (optional)
    __nv_bfloat16* Yh = outh ? static_cast<__nv_bfloat16*>(outh) + (d == 0 ? 0LL : (long long)COUT * n.pix0)
                             : nullptr;
    const float* Ap = (MODE == 1 && ACT == 1) ? chan_img<float>(aprev, COUT, d, n.pix0) : nullptr;
    // input row r (zeros outside the image) into its ring slot: asynchronous 16-byte copies of 8
    // channels of a pixel from the BF16 pixel-major input (consecutive threads: consecutive 16 bytes)
    auto load_row = [&](int r) {
      unsigned char* slot = sA + ((r + TC_NSLOT) % TC_NSLOT) * SLOT;
      for (int k = tid; k < KG * TC_COLS; k += 128) {
        const int col = k / KG, g = k % KG, gx = x0 + col - 1;
        const bool inside = r >= 0 && r < H && gx >= 0 && gx < Wd;
        cp_async16(slot + g * GSTRIDE + col * 16, inside ? Xh + (((long long)r * Wd + gx) * KG + g) : Xh, inside);
      }
      cp_async_commit();
    };
    // MMAs of output row r (input rows r-1 .. r+1 in their ring slots) into accumulator ai
    // (tensor-memory columns 32 ai ..), completion signalled on bar[ai]
    auto issue = [&](int r, int ai) {
      cp_async_wait<0>();  // this thread's copies of the rows issued so far (up to r + 1) have landed
      // shared stores of the generic proxy must be visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        int acc = 0;
        for (int tap = 0; tap < 9; ++tap) {
          const int ky = tap / 3, kx = tap % 3;
          const uint32_t slot = a0 + ((r + ky - 1 + TC_NSLOT) % TC_NSLOT) * SLOT;
          for (int kc = 0; kc < KG / 2; ++kc) {
            const uint64_t ad = umma_smem_desc(slot + 2 * kc * GSTRIDE + kx * 16, GSTRIDE, 128);
            const uint64_t bd = umma_smem_desc(b0 + tap * BTAP + 2 * kc * N * 16, N * 16, 128);
            umma_bf16(tmem + (uint32_t)(ai * 32), ad, bd, idesc, acc);
            acc = 1;
          }
        }
        umma_commit(&bar[ai]);
      }
    };
    // two accumulators: the MMAs of row h + 1 run while row h's epilogue reads the other one
    load_row(h0 - 1);
    load_row(h0);
    load_row(h0 + 1);
    if (h0 + 2 <= h1) load_row(h0 + 2);
    issue(h0, 0);
    for (int h = h0; h < h1; ++h) {
      const int ai = (h - h0) & 1;
      const bool next = h + 1 < h1;
      if (next) issue(h + 1, ai ^ 1);  // rows h .. h + 2 are in their slots
      // every thread waits (bounded) for row h's MMAs; the outcome is made uniform so that the
      // block leaves the loop together on a timeout
      const unsigned ph = ai ? phase1 : phase0;
      ok = __syncthreads_and(mbar_wait(&bar[ai], ph, kBudget) ? 1 : 0) != 0;
      if (!ok) {
        if (tid == 0) atomicOr(n.err, ERR_TIMEOUT_BIT);
        mbar_wait(&bar[ai], ph, kBudget);  // drain before the accumulators are released
        if (next) mbar_wait(&bar[ai ^ 1], ai ? phase0 : phase1, kBudget);
        break;
      }
      if (ai) phase1 ^= 1u; else phase0 ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // row h + 3 into the slot of row h - 1, whose last reader (row h's MMAs) has completed
      if (h + 3 <= h1) load_row(h + 3);
      const uint32_t taddr = tmem + (uint32_t)(ai * 32) + ((uint32_t)(warp * 32) << 16);
      const int gx = x0 + warp * 32 + lane;
      const long long o = (long long)h * Wd + gx;
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(taddr + c0, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (gx < Wd) {
          float v[16];
          if (MODE == 1 && ACT == 1) {
            // the 16 mask values are loaded before any store, so that they are in flight together
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = (c0 + j < COUT) ? __ldg(Ap + (c0 + j) * pix + o) : 0.0f;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int co = c0 + j;
            if (co < COUT) {
              if (MODE == 0) {
                const float z = __uint_as_float(r[j]) + sbias[co];
                v[j] = (ACT == 0) ? (z > 0.0f ? z : 0.0f) : tanhf(z);
              } else {
                v[j] = (ACT == 1 && !(v[j] > 0.0f)) ? 0.0f : __uint_as_float(r[j]);
              }
              if (Y) Y[co * pix + o] = v[j];
            }
          }
          if (Yh && c0 + 16 <= COUT) {
#pragma unroll
            for (int c8 = 0; c8 < 2; ++c8) {
              *reinterpret_cast<uint4*>(Yh + o * COUT + c0 + 8 * c8) = pack_bf16x8(&v[8 * c8]);
            }
          }
        }
      }
      // the accumulator is read and the oldest row slot may be refilled
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  cp_async_wait<0>();  // no copy of this block may land after it leaves (a timeout breaks early)
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// ---------------------------------------------------------------------------------------
// The whole network in one launch for forward-only BF16 stages: all three layers as tcgen05
// implicit GEMMs with the MMA sequences of nn_conv_tc_kernel (layer 1's 4 input channels padded
// to the MMA's K of 16), so the results equal the three separate launches bit for bit, while the
// 16- and 32-channel activations never leave shared memory.
//
// A block owns a 128-pixel-wide strip (local pixel p at x = x0 - 2 + p; layer 1 is exact on all
// 128 pixels, layer 2 on 1..126, layer 3 on 2..125, so a strip yields 124 outputs) and a band of
// output rows.  Step s of the band computes layer 3 on row s, layer 2 on row s + 2 and layer 1 on
// row s + 4: each layer reads only rows the step before produced, so one thread issues the 36
// MMAs of the step at its start, one bounded mbarrier wait later the epilogues write the new
// rows.  Rings (a slot is rewritten only after the MMAs that read it have completed):
//   FP32 input rows, 2 staging slots (row s + 6 to convert, row s + 7 in flight);
//   BF16 input rows s + 3 .. s + 5 (3 slots, 8-channel core matrices: 4 channels and 4 zeros;
//   the MMA's second K group points at a zero region), layer-1 and layer-2 rows (3 slots each).
// ---------------------------------------------------------------------------------------
constexpr int NF_OUT = TC_M - 4;                 // output pixels per strip
constexpr int NF_AS = 3;                         // ring slots
constexpr int NF_G = TC_COLS * 16;               // one 8-channel group of a BF16 row (core matrices)
constexpr int NF_A1SLOT = 2 * NF_G;              // 16 channels
constexpr int NF_A2SLOT = 4 * NF_G;              // 32 channels
constexpr int NF_XF = 4 * TC_COLS;               // floats of an FP32 input row: 4 channels x 130 pixels
constexpr int NF_B1TAP = 2 * 16 * 16;            // layer-1 weights of one tap: [group 2][co 16][8]
constexpr int NF_B2TAP = 2 * 32 * 16;            // layer-2 weights of one tap: [group 2][co 32][8]
constexpr int NF_B3TAP = 4 * 16 * 16;            // layer-3 weights of one tap: [group 4][co 16][8]
constexpr int NF_OFF_A2 = NF_AS * NF_A1SLOT;
constexpr int NF_OFF_X = NF_OFF_A2 + NF_AS * NF_A2SLOT;   // BF16 input rows, then the zero group
constexpr int NF_OFF_Z = NF_OFF_X + NF_AS * NF_G;
constexpr int NF_OFF_B1 = NF_OFF_Z + NF_G;
constexpr int NF_OFF_B2 = NF_OFF_B1 + 9 * NF_B1TAP;
constexpr int NF_OFF_B3 = NF_OFF_B2 + 9 * NF_B2TAP;
constexpr int NF_OFF_XF = NF_OFF_B3 + 9 * NF_B3TAP;
constexpr int NF_OFF_BIAS = NF_OFF_XF + 2 * NF_XF * 4;
constexpr int NF_SMEM = NF_OFF_BIAS + (16 + 32 + 4) * 4;
__host__ __device__ constexpr int nf_slot3(int r) { return (r + 15) % 3; }   // rows >= -15

__global__ void __launch_bounds__(128) nn_net_tc_kernel(NnArgs n, int band) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sA1 = smem_raw;
  unsigned char* sA2 = smem_raw + NF_OFF_A2;
  unsigned char* sX = smem_raw + NF_OFF_X;
  float* sXf = reinterpret_cast<float*>(smem_raw + NF_OFF_XF);
  float* sb1 = reinterpret_cast<float*>(smem_raw + NF_OFF_BIAS);
  float* sb2 = sb1 + 16;
  float* sb3 = sb2 + 32;
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tmem_base;
  int nxs[2], nys[2];
  for (int d = 0; d < 2; ++d) {
    nxs[d] = (d < n.nimg) ? (n.W[d] + NF_OUT - 1) / NF_OUT : 0;
    nys[d] = (d < n.nimg) ? (n.H[d] + band - 1) / band : 0;
  }
  const int items0 = nxs[0] * nys[0];
  if ((int)blockIdx.x >= items0 + nxs[1] * nys[1]) return;  // uniform per block, before any allocation
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    // three arrivals per phase: the threads issuing layer 1, 2 and 3 each commit to it
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 3;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights per tap as [group][co][8 channels], converted FP64 -> FP32 -> BF16 as the separate
  // layers do (zeros beyond the real channels); biases FP32
  __nv_bfloat16* B1 = reinterpret_cast<__nv_bfloat16*>(smem_raw + NF_OFF_B1);
  for (int k = tid; k < 9 * 16 * 16; k += 128) {
    const int tap = k / (16 * 16), r = k % (16 * 16), ci = r / 16, co = r % 16;
    B1[tap * (NF_B1TAP / 2) + ((ci >> 3) * 16 + co) * 8 + (ci & 7)] =
        __float2bfloat16_rn(ci < 4 ? (float)n.w[NN_OFF1 + (co * 4 + ci) * 9 + tap] : 0.0f);
  }
  __nv_bfloat16* B2 = reinterpret_cast<__nv_bfloat16*>(smem_raw + NF_OFF_B2);
  for (int k = tid; k < 9 * 16 * 32; k += 128) {
    const int tap = k / (16 * 32), r = k % (16 * 32), ci = r / 32, co = r % 32;
    B2[tap * (NF_B2TAP / 2) + ((ci >> 3) * 32 + co) * 8 + (ci & 7)] =
        __float2bfloat16_rn((float)n.w[NN_OFF2 + (co * 16 + ci) * 9 + tap]);
  }
  __nv_bfloat16* B3 = reinterpret_cast<__nv_bfloat16*>(smem_raw + NF_OFF_B3);
  for (int k = tid; k < 9 * 32 * 16; k += 128) {
    const int tap = k / (32 * 16), r = k % (32 * 16), ci = r / 16, co = r % 16;
    B3[tap * (NF_B3TAP / 2) + ((ci >> 3) * 16 + co) * 8 + (ci & 7)] =
        __float2bfloat16_rn(co < 4 ? (float)n.w[NN_OFF3 + (co * 32 + ci) * 9 + tap] : 0.0f);
  }
  for (int k = tid; k < 16; k += 128) sb1[k] = (float)n.w[NN_OFF1 + 16 * 36 + k];
  for (int k = tid; k < 32; k += 128) sb2[k] = (float)n.w[NN_OFF2 + 32 * 144 + k];
  for (int k = tid; k < 4; k += 128) sb3[k] = (float)n.w[NN_OFF3 + 4 * 288 + k];
  // the rings and the zero group start zeroed (rows before the band's first valid ones are read
  // only by outputs that are never stored)
  for (int k = tid; k < NF_OFF_B1 / 16; k += 128) reinterpret_cast<uint4*>(smem_raw)[k] = make_uint4(0, 0, 0, 0);

  const int it = blockIdx.x;
  const int d = (it < items0) ? 0 : 1;
  const int il = (d == 0) ? it : it - items0;
  const int H = n.H[d], Wd = n.W[d];
  const int x0 = (il % nxs[d]) * NF_OUT, h0 = (il / nxs[d]) * band;
  const int h1 = (h0 + band < H) ? h0 + band : H;
  const int xs = x0 - 2;  // image column of local pixel 0
  const long long pix = (long long)H * Wd;
  const float* X = chan_img<float>(n.X, 4, d, n.pix0);
  float* T3 = chan_img<float>(n.T3, 4, d, n.pix0);
  const int p = tid, xp = xs + p;
  const bool col_in = xp >= 0 && xp < Wd;
  // FP32 input row r (zeros outside the image): 4 channels x 130 pixels (local -1 .. 128), 4-byte
  // copies into staging slot r & 1; element tid + 128 i of a slot is channel / column xofs[i]
  constexpr int NXL = (NF_XF + 127) / 128;
  long long xofs[NXL];
  bool xok[NXL];
#pragma unroll
  for (int i = 0; i < NXL; ++i) {
    const int k = tid + 128 * i, ch = k / TC_COLS, gx = xs - 1 + k % TC_COLS;
    xok[i] = k < NF_XF && gx >= 0 && gx < Wd;
    xofs[i] = ch * pix + gx;
  }
  auto load_x = [&](int r) {
    float* slot = sXf + (r & 1) * NF_XF + tid;
    const bool row_in = r >= 0 && r < H;
    const float* Xr = X + (long long)r * Wd;
#pragma unroll
    for (int i = 0; i < NXL; ++i)
      if (tid + 128 * i < NF_XF) cp_async4(slot + 128 * i, row_in && xok[i] ? Xr + xofs[i] : X, row_in && xok[i]);
    cp_async_commit();
  };
  // staged FP32 row r to its BF16 ring slot: per pixel one 16-byte core-matrix row (4 channels
  // rounded to BF16, 4 zeros)
  auto convert_x = [&](int r) {
    const float* src = sXf + (r & 1) * NF_XF;
    unsigned char* dst = sX + nf_slot3(r) * NF_G;
    for (int c = tid; c < TC_COLS; c += 128)
      *reinterpret_cast<uint4*>(dst + c * 16) =
          make_uint4(pack_bf16x2(src[c], src[TC_COLS + c]), pack_bf16x2(src[2 * TC_COLS + c], src[3 * TC_COLS + c]),
                     0u, 0u);
  };
  const int s0 = h0 - 6;
  // prologue: input rows s0 + 3 .. s0 + 5 into the BF16 ring, row s0 + 6 staged
  for (int r = s0 + 3; r <= s0 + 5; ++r) {
    load_x(r);
    cp_async_wait<0>();
    __syncthreads();
    convert_x(r);
    __syncthreads();
  }
  load_x(s0 + 6);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // shared-memory descriptors of the ring slots and weights; a byte offset o (a multiple of 16)
  // adds o / 16 to a descriptor
  uint64_t ds0, ds1, ds2, db;  // the three ring slots of the layer this thread issues, its weights
  if (tid == 64) {  // layer 1: input rows (second K group: the zero region), weights [tap][2][16][8]
    const uint32_t b = smem_u32(sX);
    ds0 = umma_smem_desc(b, 3 * NF_G, 128);
    ds1 = umma_smem_desc(b + NF_G, 2 * NF_G, 128);
    ds2 = umma_smem_desc(b + 2 * NF_G, NF_G, 128);
    db = umma_smem_desc(smem_u32(smem_raw + NF_OFF_B1), 16 * 16, 128);
  } else if (tid == 32) {  // layer 2: layer-1 rows, weights [tap][2][32][8]
    const uint32_t b = smem_u32(sA1);
    ds0 = umma_smem_desc(b, NF_G, 128);
    ds1 = umma_smem_desc(b + NF_A1SLOT, NF_G, 128);
    ds2 = umma_smem_desc(b + 2 * NF_A1SLOT, NF_G, 128);
    db = umma_smem_desc(smem_u32(smem_raw + NF_OFF_B2), 32 * 16, 128);
  } else {  // layer 3: layer-2 rows, weights [tap][4][16][8]
    const uint32_t b = smem_u32(sA2);
    ds0 = umma_smem_desc(b, NF_G, 128);
    ds1 = umma_smem_desc(b + NF_A2SLOT, NF_G, 128);
    ds2 = umma_smem_desc(b + 2 * NF_A2SLOT, NF_G, 128);
    db = umma_smem_desc(smem_u32(smem_raw + NF_OFF_B3), 16 * 16, 128);
  }
  auto dsl = [&](int r) {  // descriptor of the slot of row r
    const int sl = nf_slot3(r);
    return sl == 0 ? ds0 : (sl == 1 ? ds1 : ds2);
  };
  constexpr uint32_t idesc16 = umma_idesc_bf16(TC_M, 16), idesc32 = umma_idesc_bf16(TC_M, 32);
  constexpr long long kBudget = 2000000000LL;  // about one second of SM clock
  unsigned phase = 0u;
  bool ok = true;
  for (int s = s0; s < h1; ++s) {
    load_x(s + 7);  // into the staging slot of row s + 5, converted in the step before
    // one thread per layer issues its MMAs (into its own accumulator) and commits to the barrier
    if (tid == 64) {
      // layer 1 of row s + 4 from input rows s + 3 .. s + 5, accumulator columns 48 .. 63
      for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        umma_bf16(tmem + 48, dsl(s + 3 + ky) + kx, db + tap * (NF_B1TAP / 16), idesc16, tap > 0 ? 1 : 0);
      }
      umma_commit(&bar);
    } else if (tid == 32) {
      // layer 2 of row s + 2 from layer-1 rows s + 1 .. s + 3, accumulator columns 0 .. 31
      for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        umma_bf16(tmem, dsl(s + 1 + ky) + kx, db + tap * (NF_B2TAP / 16), idesc32, tap > 0 ? 1 : 0);
      }
      umma_commit(&bar);
    } else if (tid == 0) {
      // layer 3 of row s from layer-2 rows s - 1 .. s + 1, accumulator columns 32 .. 47
      for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
        for (int kc = 0; kc < 2; ++kc)
          umma_bf16(tmem + 32, dsl(s - 1 + ky) + (2 * kc * NF_G) / 16 + kx,
                    db + tap * (NF_B3TAP / 16) + kc * (2 * 16 * 16 / 16), idesc16, (tap > 0 || kc > 0) ? 1 : 0);
      }
      umma_commit(&bar);
    }
    cp_async_wait<1>();  // this thread's copies of input row s + 6 have landed
    // every thread waits (bounded) for the step's MMAs; the outcome is made uniform (and the
    // barrier makes every thread's staged copies visible)
    ok = __syncthreads_and(mbar_wait(&bar, phase, kBudget) ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) atomicOr(n.err, ERR_TIMEOUT_BIT);
      mbar_wait(&bar, phase, kBudget);  // drain before the accumulators are released
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    convert_x(s + 6);  // into the slot of row s + 3, whose last reader (layer 1 of row s + 4) is done
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    // layer 1 of row s + 4 (bias, ReLU, zero outside the image) into the slot of row s + 1
    {
      const int r1 = s + 4;
      const bool in = col_in && r1 >= 0 && r1 < H;
      uint32_t r[16];
      tmem_ld16(tl + 48, r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      unsigned char* dst = sA1 + nf_slot3(r1) * NF_A1SLOT + (p + 1) * 16;
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        float v8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float z = __uint_as_float(r[8 * g + e]) + sb1[8 * g + e];
          v8[e] = in ? (z > 0.0f ? z : 0.0f) : 0.0f;
        }
        *reinterpret_cast<uint4*>(dst + g * NF_G) = pack_bf16x8(v8);
      }
    }
    // layer 2 of row s + 2 (bias, ReLU, zero outside the image) into the slot of row s - 1
    {
      const int r2 = s + 2;
      const bool in = col_in && r2 >= 0 && r2 < H;
      uint32_t r[32];
      tmem_ld16(tl, r);
      tmem_ld16(tl + 16, r + 16);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      unsigned char* dst = sA2 + nf_slot3(r2) * NF_A2SLOT + (p + 1) * 16;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float v8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float z = __uint_as_float(r[8 * g + e]) + sb2[8 * g + e];
          v8[e] = in ? (z > 0.0f ? z : 0.0f) : 0.0f;
        }
        *reinterpret_cast<uint4*>(dst + g * NF_G) = pack_bf16x8(v8);
      }
    }
    // layer 3 of row s (bias, tanh) to the FP32 output
    {
      uint32_t r[16];
      tmem_ld16(tl + 32, r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (s >= h0 && p >= 2 && p < 2 + NF_OUT && xp < Wd) {
        const long long o = (long long)s * Wd + xp;
#pragma unroll
        for (int co = 0; co < 4; ++co) T3[co * pix + o] = tanhf(__uint_as_float(r[co]) + sb3[co]);
      }
    }
    // the new rows must be visible to the tensor core (async proxy) before the next step's MMAs
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  cp_async_wait<0>();  // no copy of this block may land after it leaves
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// ---------------------------------------------------------------------------------------
// BF16 weight gradient of one layer on the tensor cores (the BF16 reverse):
//   dW[co][ci][ky][kx] = sum over pixels q of G[co](q) A[ci](q + (ky-1, kx-1)),  db[co] = sum G[co]
// with G (the layer's output gradient) and A (its input) rounded to BF16, FP32 accumulation.
// Per chunk of WC = 64 pixels of image row y (x0 .. x0+63), one implicit GEMM with K = the chunk's
// pixels:  D[(ky, co)][(kx, ci)] += sum_x G[co](y+1-ky, x) A[ci](y, x+kx-1)  — which is dW once
// summed over every row y, the shift of a tap split between the two operands: the A operand holds
// the three G rows y+1, y, y-1 (channels padded to 8), the B operand three x-shifted copies of A's
// row y and a row of ones (D's ones column on the unshifted G rows is db).  M = 128 (rows beyond
// 3 x COUTP ignored), N = NB = 3 CIN + 1 rounded up to 16, one tcgen05.mma per 16 pixels into a
// TMEM accumulator that holds the block's sum over all its chunks.
// A block walks work items of a 64-pixel column strip and a band of rows; the FP32 rows arrive by
// 4-byte cp.async into rings (G rows y-1 .. y+1 read, y+2 in flight; A row y read, y+1 in flight;
// channel strides padded against shared-memory bank conflicts),
// and each chunk's BF16 operands are built from them into one of two buffers, the next chunk's
// while the MMAs read the current one.  Each block writes its sums to partial[block] (all the
// layer's parameters; zeros when it had no chunk), reduced in a fixed order afterwards.
// ---------------------------------------------------------------------------------------
constexpr int WC = 64;            // pixels per chunk (the GEMM's K per chunk)
constexpr int WKG = WC / 8;       // 8-pixel core-matrix columns per chunk
constexpr int WBAND = 16;         // rows per work item
constexpr int WNT = 256;          // threads per block
constexpr int WGS = WC + 4;       // floats per channel of a staged G row (padded: no bank conflicts)
constexpr int WAS = WC + 3;       // floats per channel of a staged A row (1-pixel halo, odd stride)
template <int CIN, int COUT>
struct WgTc {
  static constexpr int COUTP = (COUT + 7) / 8 * 8;          // G channels per row, padded
  static constexpr int NB = (3 * CIN + 1 + 15) / 16 * 16;   // MMA N
  static constexpr int ABYTES = 128 * WC * 2;               // A operand: 128 rows x WC pixels, BF16
  static constexpr int BBYTES = NB * WC * 2;
  static constexpr int BUF = ABYTES + BBYTES;
  static constexpr int GROW = COUT * WGS;                   // floats of a staged G row
  static constexpr int AROW = CIN * WAS;                    // floats of a staged A row
  static constexpr int OFF_G = 2 * BUF;                     // G ring (4 rows), then A ring (2 rows)
  static constexpr int OFF_A = OFF_G + 4 * GROW * 4;
  static constexpr int SMEM = OFF_A + 2 * AROW * 4;
  static_assert(3 * COUTP <= 128 && NB <= 256, "one MMA tile");
};

// 8 floats -> one 16-byte core-matrix row of 8 BF16 values
__device__ __forceinline__ uint4 bf16x8(const float v[8]) { return pack_bf16x8(v); }

template <int CIN, int COUT>
__global__ void __launch_bounds__(WNT) nn_wgrad_tc_kernel(NnArgs n, const float* __restrict__ gout,
                                                          const float* __restrict__ ain, int woff) {
  using P = WgTc<CIN, COUT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
  }
  // both operand buffers zeroed, then the constant rows of B: the ones row (n = 3 CIN); the
  // padding rows and the A rows beyond 3 COUTP stay zero
  for (int k = tid; k < 2 * P::BUF / 16; k += WNT) reinterpret_cast<uint4*>(smem_raw)[k] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int u = tid; u < 2 * WKG; u += WNT) {
    const int buf = u / WKG, kg = u % WKG, nrow = 3 * CIN;
    const float one[8] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
    *reinterpret_cast<uint4*>(smem_raw + buf * P::BUF + P::ABYTES + ((nrow >> 3) * WKG + kg) * 128 + (nrow & 7) * 16) =
        bf16x8(one);
  }
  float* sG = reinterpret_cast<float*>(smem_raw + P::OFF_G);
  float* sAr = reinterpret_cast<float*>(smem_raw + P::OFF_A);
  // work items: image d, 64-pixel column strip, band of WBAND rows
  int nsx[2], nit[2];
  for (int d = 0; d < 2; ++d) {
    nsx[d] = (d < n.nimg) ? (n.W[d] + WC - 1) / WC : 0;
    nit[d] = (d < n.nimg) ? nsx[d] * ((n.H[d] + WBAND - 1) / WBAND) : 0;
  }
  const int items = nit[0] + nit[1];
  // FP32 rows of the item's strip into the rings (zeros outside the image), 4-byte copies: G row
  // rg as [co][64] (element: channel, pixel x0 + tid % 64), A row ra as [ci][66] (pixels x0 - 1 ..
  // x0 + 64)
  auto load_g = [&](int d, int x0, int rg) {
    const int H = n.H[d], Wd = n.W[d];
    const long long pix = (long long)H * Wd;
    const float* G = gout + (d == 0 ? 0LL : (long long)COUT * n.pix0);
    float* dst = sG + ((rg + 8) & 3) * P::GROW;
    const int x = x0 + (tid & 63);
    const bool in = rg >= 0 && rg < H && x < Wd;
    for (int co = tid >> 6; co < COUT; co += WNT / 64)
      cp_async4(dst + co * WGS + (tid & 63), in ? G + co * pix + (long long)rg * Wd + x : G, in);
  };
  auto load_a = [&](int d, int x0, int ra) {
    const int H = n.H[d], Wd = n.W[d];
    const long long pix = (long long)H * Wd;
    const float* A = ain + (d == 0 ? 0LL : (long long)CIN * n.pix0);
    float* dst = sAr + (ra & 1) * P::AROW;
    for (int k = tid; k < CIN * (WC + 2); k += WNT) {
      const int ci = k / (WC + 2), xx = k % (WC + 2), x = x0 - 1 + xx;
      const bool in = ra < H && x >= 0 && x < Wd;
      cp_async4(dst + ci * WAS + xx, in ? A + ci * pix + (long long)ra * Wd + x : A, in);
    }
  };
  // the BF16 operands of chunk (row y) into buffer b; unit u = (8-row group, pixel column, row
  // in group) at shared-memory offset 16 u (consecutive threads: consecutive 16-byte rows)
  auto build = [&](int y, int b) {
    unsigned char* sA = smem_raw + b * P::BUF;
    unsigned char* sB = sA + P::ABYTES;
    constexpr int AU = 3 * P::COUTP * WKG;
    for (int u = tid; u < AU; u += WNT) {
      const int kg = (u >> 3) % WKG, m = ((u >> 3) / WKG) * 8 + (u & 7);
      const int ky = m / P::COUTP, co = m % P::COUTP;
      if (co >= COUT) continue;  // padding rows stay zero
      const float4* src = reinterpret_cast<const float4*>(sG + ((y + 1 - ky + 8) & 3) * P::GROW + co * WGS + kg * 8);
      const float4 p = src[0], q = src[1];
      const float v[8] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
      *reinterpret_cast<uint4*>(sA + 16 * u) = bf16x8(v);
    }
    constexpr int BU = (3 * CIN + 7) / 8 * 8 * WKG;
    for (int u = tid; u < BU; u += WNT) {
      const int kg = (u >> 3) % WKG, nr = ((u >> 3) / WKG) * 8 + (u & 7);
      if (nr >= 3 * CIN) continue;  // the ones row and padding are constant
      const int kx = nr / CIN, ci = nr % CIN;
      const float* src = sAr + (y & 1) * P::AROW + ci * WAS + kg * 8 + kx;
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = src[e];
      *reinterpret_cast<uint4*>(sB + 16 * u) = bf16x8(v);
    }
  };
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = umma_idesc_bf16(128, P::NB);
  constexpr long long kBudget = 2000000000LL;  // about one second of SM clock
  unsigned phase0 = 0u, phase1 = 0u;
  bool pend0 = false, pend1 = false;  // MMAs committed to bar[b] and not yet waited for
  bool ok = true;
  int nmma = 0, chunk = 0;
  // a bounded wait, uniform across the block, for the MMAs committed to bar[b]
  auto wait_buf = [&](int b) {
    const unsigned ph = b ? phase1 : phase0;
    ok = __syncthreads_and(mbar_wait(&bar[b], ph, kBudget) ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) atomicOr(n.err, ERR_TIMEOUT_BIT);
      mbar_wait(&bar[b], ph, kBudget);  // drain before the accumulator is released
    }
    if (b) {
      phase1 ^= 1u;
      pend1 = false;
    } else {
      phase0 ^= 1u;
      pend0 = false;
    }
  };
  for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
    const int d = (it < nit[0]) ? 0 : 1;
    const int il = (d == 0) ? it : it - nit[0];
    const int H = n.H[d];
    const int x0 = (il % nsx[d]) * WC, h0 = (il / nsx[d]) * WBAND;
    const int h1 = (h0 + WBAND < H) ? h0 + WBAND : H;
    // prologue: G rows h0 - 1 .. h0 + 1 and A row h0
    load_g(d, x0, h0 - 1);
    load_g(d, x0, h0);
    load_g(d, x0, h0 + 1);
    load_a(d, x0, h0);
    cp_async_commit();
    for (int y = h0; y < h1; ++y, ++chunk) {
      const int b = chunk & 1;
      // the next row's copies: G row y + 2 into the slot of row y - 2, A row y + 1 into the slot of
      // row y - 1, whose last readers (the chunk of row y - 1) passed the barrier before its MMAs
      load_g(d, x0, y + 2);
      load_a(d, x0, y + 1);
      cp_async_commit();
      if (b ? pend1 : pend0) {
        wait_buf(b);  // the MMAs of two chunks ago read this buffer
        if (!ok) break;
      }
      cp_async_wait<1>();  // this thread's copies of G rows up to y + 1 and A row y have landed
      __syncthreads();
      build(y, b);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        const uint32_t a0 = smem_u32(smem_raw + b * P::BUF), b0 = a0 + P::ABYTES;
        for (int j = 0; j < WKG / 2; ++j)  // 16 pixels (two core-matrix columns) per MMA
          umma_bf16(tmem, umma_smem_desc(a0 + 2 * j * 128, 128, WKG * 128),
                    umma_smem_desc(b0 + 2 * j * 128, 128, WKG * 128), idesc, (nmma + j) > 0 ? 1 : 0);
        umma_commit(&bar[b]);
      }
      nmma += WKG / 2;  // every thread counts the MMAs issued
      if (b) pend1 = true; else pend0 = true;
    }
    // the item's last copies (rows past the band) land before the rings are refilled
    cp_async_wait<0>();
    __syncthreads();
  }
  cp_async_wait<0>();
  if (ok && pend0) wait_buf(0);
  if (ok && pend1) wait_buf(1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue (warps 0-3, one accumulator lane each): lane m = row (ky, co); columns (kx, ci) and
  // the ones column
  const int m = tid;
  const int ky = m / P::COUTP, co = m % P::COUTP;
  const bool real = warp < 4 && ky < 3 && co < COUT;
  double* part = n.partial + (long long)blockIdx.x * NN_NPARAM + woff;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
  for (int c0 = 0; c0 < P::NB; c0 += 16) {
    if (warp >= 4) break;  // warp-uniform
    uint32_t r[16];
    tmem_ld16(tl + c0, r);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (real && ok) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int nc = c0 + e;
        const double v = (nmma > 0) ? (double)__uint_as_float(r[e]) : 0.0;
        if (nc < 3 * CIN) {
          const int kx = nc / CIN, ci = nc % CIN;
          part[(co * CIN + ci) * 9 + ky * 3 + kx] = v;
        } else if (nc == 3 * CIN && ky == 1) {
          part[COUT * CIN * 9 + co] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

// the FP32 network input X (planar, 4 channels) as the first tensor-core layer's input: BF16
// pixel-major, 16 channels per pixel (4 and 12 zeros)
__global__ void nn_x16_kernel(NnArgs n, __nv_bfloat16* __restrict__ Xh) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long pix = n.pix0 + (n.nimg > 1 ? (long long)n.H[1] * n.W[1] : 0LL);
  if (t >= pix) return;
  const int d = (t < n.pix0) ? 0 : 1;
  const long long q = (d == 0) ? t : t - n.pix0, pd = (long long)n.H[d] * n.W[d];
  const float* X = chan_img<float>(n.X, 4, d, n.pix0);
  uint4* dst = reinterpret_cast<uint4*>(Xh + t * 16);
  dst[0] = make_uint4(pack_bf16x2(X[q], X[pd + q]), pack_bf16x2(X[2 * pd + q], X[3 * pd + q]), 0u, 0u);
  dst[1] = make_uint4(0u, 0u, 0u, 0u);
}

// network input from an FP64 image / scaled FP64 output (js_nn_eval)
template <class T>
__global__ void nn_load_kernel(const double* __restrict__ Xd, T* __restrict__ X, long long n4) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n4) X[t] = (T)Xd[t];
}
template <class T>
__global__ void nn_store_kernel(const T* __restrict__ T3, double* __restrict__ Y, long long pix, NnArgs n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 4 * pix) Y[t] = n.scale[t / pix] * (double)T3[t];
}

// reverse of js_nn_eval: seed G4 = GY * scale * (1 - T3^2) (the derivative of scale * tanh) with an
// optional BF16 pixel-major copy padded to 16 channels, and the input gradient back to FP64
template <class T>
__global__ void nn_seed_eval_kernel(NnArgs n, const double* __restrict__ GY, long long pix, __nv_bfloat16* gh) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pix) return;
  const T* t3 = static_cast<const T*>(n.T3);
  T* g = static_cast<T*>(n.G4);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double t = (double)t3[k * pix + p];
    g[k * pix + p] = (T)(GY[k * pix + p] * n.scale[k] * (1.0 - t * t));
  }
  if (gh) {
    float v8[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v8[e] = e < 4 ? (float)g[e * pix + p] : 0.0f;
    uint4* dst = reinterpret_cast<uint4*>(gh + p * 16);
    dst[0] = pack_bf16x8(v8);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}
template <class T>
__global__ void nn_unload_kernel(const T* __restrict__ G, double* __restrict__ GX, long long n4) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n4) GX[t] = (double)G[t];
}

// stage output (or RHS) minus the neural flux divergence on fluid cells
template <class T>
__global__ void __launch_bounds__(256) nn_apply_kernel(NnArgs n, StageArgs a, int rhs) {
  // 32 x 32 cells per block: the tile's y-face fluxes (image 1: line = column i, face = row j)
  // pass through shared memory, so both images are read along their contiguous axis
  __shared__ T sy[4][IT][IT + 2];
  const Lay& L = a.lay;
  const int i0 = blockIdx.x * IT, j0 = blockIdx.y * IT;
  const long long ncell = (long long)L.nx * L.ny;
  const bool two = n.nimg > 1;
  if (two) {
    const T* Fy = chan_img<T>(n.T3, 4, 1, n.pix0);
    const long long py = (long long)n.H[1] * n.W[1];
    for (int e = threadIdx.x; e < 4 * IT * (IT + 1); e += 256) {
      const int k = e / (IT * (IT + 1)), r = e % (IT * (IT + 1)), il = r / (IT + 1), jl = r % (IT + 1);
      const int i = i0 + il, j = j0 + jl;
      sy[k][il][jl] = (i < L.nx && j <= L.ny) ? Fy[k * py + (long long)i * n.W[1] + j] : (T)0;
    }
  }
  __syncthreads();
  const T* Fx = chan_img<T>(n.T3, 4, 0, n.pix0);
  const long long px = (long long)n.H[0] * n.W[0];
  const double fac = (!rhs && a.use_un) ? a.rk_b : 1.0;
  const int ky_of[4] = {0, 2, 1, 3};  // frame channel of each conserved component, y faces
  const float cxf = (float)a.cx, cyf = (float)a.cy;
  const float scf[4] = {(float)n.scale[0], (float)n.scale[1], (float)n.scale[2], (float)n.scale[3]};
  const int il = threadIdx.x % IT;
  for (int jl = threadIdx.x / IT; jl < IT; jl += 256 / IT) {
    const int i = i0 + il, j = j0 + jl;
    if (i >= L.nx || j >= L.ny) continue;
    const long long o = (long long)j * L.nx + i;
    if (a.tag && a.tag[o] != 0) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const long long ox = (long long)j * n.W[0] + i;
      double corr;
      if (std::is_same<T, float>::value) {
        // FP32 network: its flux divergence in FP32 (the FP64 pipe only adds it to the state)
        float cf = cxf * (scf[c] * (Fx[c * px + ox + 1] - Fx[c * px + ox]));
        if (two) {
          const int k = ky_of[c];
          cf = fmaf(cyf, scf[k] * (sy[k][il][jl + 1] - sy[k][il][jl]), cf);
        }
        corr = (double)cf;
      } else {
        corr = a.cx * (n.scale[c] * ((double)Fx[c * px + ox + 1] - (double)Fx[c * px + ox]));
        if (two) {
          const int k = ky_of[c];
          corr = fma(a.cy, n.scale[k] * ((double)sy[k][il][jl + 1] - (double)sy[k][il][jl]), corr);
        }
      }
      if (rhs) a.Uout[c * ncell + o] -= corr;
      else a.Uout[c * L.plane + L.idx(i, j)] -= fac * corr;
    }
  }
}

// ---------------------------------------------------------------------------------------
// reverse
// ---------------------------------------------------------------------------------------
// dZ3 = (face-flux adjoint in the frame) * scale * (1 - t^2)
// (gh: optional BF16 pixel-major copy, 16 channels per pixel with 12 zeros, the input of the
// tensor-core data gradient of the last layer)
template <class T>
__global__ void nn_seed_kernel(NnArgs n, AdjArgs a, __nv_bfloat16* gh) {
  const int d = blockIdx.y;
  const int Wd = n.W[d];
  const long long pix = (long long)n.H[d] * Wd;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pix) return;
  const int h = (int)(p / Wd), f = (int)(p % Wd);
  const Lay& L = a.lay;
  const long long ca = (d == 0) ? L.idx(f - 1, h) : L.idx(h, f - 1);
  const long long cb = (d == 0) ? L.idx(f, h) : L.idx(h, f);
  const double invh = (d == 0) ? a.inv_dx : a.inv_dy;
  const T* t3 = chan_img<T>(n.T3, 4, d, n.pix0);
  T* g = chan_img<T>(n.G4, 4, d, n.pix0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = (d == 0) ? k : (k == 1 ? 2 : (k == 2 ? 1 : k));
    const double Fb = (a.lam[c * L.plane + cb] - a.lam[c * L.plane + ca]) * invh;
    const double t = (double)t3[k * pix + p];
    g[k * pix + p] = (T)(Fb * n.scale[k] * (1.0 - t * t));
  }
  if (gh) {
    float v8[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v8[e] = e < 4 ? (float)g[e * pix + p] : 0.0f;
    uint4* dst = reinterpret_cast<uint4*>(gh + (d == 0 ? 0LL : 16LL * n.pix0) + p * 16);
    dst[0] = pack_bf16x8(v8);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// data gradient of one layer: gin[ci] = sum_co,ky,kx w[co][ci][ky][kx] gout[co][h-ky+1][x-kx+1],
// times the ReLU mask of the layer below when MASK
template <class T, int CIN, int COUT, bool MASK>
__global__ void __launch_bounds__(NTHR) nn_dgrad_kernel(NnArgs n, const void* gout, const void* aprev, void* gin,
                                                        int woff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NWW = COUT * CIN * 9;
  T* sw = reinterpret_cast<T*>(smem_raw);
  T* sg = sw + ((NWW + 1) & ~1);
  const int d = blockIdx.z;
  const int H = n.H[d], Wd = n.W[d];
  const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
  if (x0 >= Wd || y0 >= H) return;
  const long long pix = (long long)H * Wd;
  const T* G = chan_img<T>(gout, COUT, d, n.pix0);
  T* D = chan_img<T>(gin, CIN, d, n.pix0);
  for (int k = threadIdx.x; k < NWW; k += NTHR) sw[k] = (T)n.w[woff + k];
  for (int k = threadIdx.x; k < COUT * TH * TH; k += NTHR) {
    const int co = k / (TH * TH), r = k % (TH * TH);
    const int gy = y0 + r / TH - 1, gx = x0 + r % TH - 1;
    sg[k] = (gy >= 0 && gy < H && gx >= 0 && gx < Wd) ? G[co * pix + (long long)gy * Wd + gx] : (T)0;
  }
  __syncthreads();
  const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
  T acc[CIN];
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) acc[ci] = (T)0;
  for (int co = 0; co < COUT; ++co)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const T v = sg[co * TH * TH + (ty - ky + 2) * TH + tx - kx + 2];
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) acc[ci] = fma(sw[((co * CIN + ci) * 3 + ky) * 3 + kx], v, acc[ci]);
      }
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx < Wd && gy < H) {
    const long long o = (long long)gy * Wd + gx;
    const T* A = MASK ? chan_img<T>(aprev, CIN, d, n.pix0) : nullptr;
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      T v = acc[ci];
      if (MASK && !(A[ci * pix + o] > (T)0)) v = (T)0;
      D[ci * pix + o] = v;
    }
  }
}

// weight gradient of one layer: blocks stride over the tiles of both images and keep
// per-thread sums of the weights they own; each block writes its sums to partial[block]
template <class T, int CIN, int COUT>
__global__ void __launch_bounds__(NTHR) nn_wgrad_kernel(NnArgs n, const void* gout, const void* ain, int woff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = COUT * CIN * 9 + COUT;
  constexpr int PER = (NW + NTHR - 1) / NTHR;
  T* sg = reinterpret_cast<T*>(smem_raw);  // [COUT][256]
  T* sa = sg + COUT * NTHR;                // [CIN][18][18]
  T acc[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) acc[r] = (T)0;
  int ntx[2], nty[2];
  for (int d = 0; d < 2; ++d) {
    ntx[d] = (d < n.nimg) ? (n.W[d] + TILE - 1) / TILE : 0;
    nty[d] = (d < n.nimg) ? (n.H[d] + TILE - 1) / TILE : 0;
  }
  const int t0 = ntx[0] * nty[0], total = t0 + ntx[1] * nty[1];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int d = (t < t0) ? 0 : 1;
    const int tl = (d == 0) ? t : t - t0;
    const int x0 = (tl % ntx[d]) * TILE, y0 = (tl / ntx[d]) * TILE;
    const int H = n.H[d], Wd = n.W[d];
    const long long pix = (long long)H * Wd;
    const T* G = chan_img<T>(gout, COUT, d, n.pix0);
    const T* A = chan_img<T>(ain, CIN, d, n.pix0);
    __syncthreads();
    for (int k = threadIdx.x; k < COUT * NTHR; k += NTHR) {
      const int co = k / NTHR, r = k % NTHR;
      const int gy = y0 + r / TILE, gx = x0 + r % TILE;
      sg[k] = (gy < H && gx < Wd) ? G[co * pix + (long long)gy * Wd + gx] : (T)0;
    }
    for (int k = threadIdx.x; k < CIN * TH * TH; k += NTHR) {
      const int ci = k / (TH * TH), r = k % (TH * TH);
      const int gy = y0 + r / TH - 1, gx = x0 + r % TH - 1;
      sa[k] = (gy >= 0 && gy < H && gx >= 0 && gx < Wd) ? A[ci * pix + (long long)gy * Wd + gx] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int k = threadIdx.x + r * NTHR;
      if (k >= NW) continue;
      T s = (T)0;
      if (k < COUT * CIN * 9) {
        const int co = k / (CIN * 9), rem = k % (CIN * 9);
        const int ci = rem / 9, ky = (rem % 9) / 3, kx = rem % 3;
        const T* g = sg + co * NTHR;
        const T* a = sa + ci * TH * TH + ky * TH + kx;
        for (int py = 0; py < TILE; ++py)
#pragma unroll
          for (int px = 0; px < TILE; ++px) s = fma(g[py * TILE + px], a[py * TH + px], s);
      } else {
        const T* g = sg + (k - COUT * CIN * 9) * NTHR;
        for (int q = 0; q < NTHR; ++q) s += g[q];
      }
      acc[r] += s;
    }
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int k = threadIdx.x + r * NTHR;
    if (k < NW) n.partial[(long long)blockIdx.x * NN_NPARAM + woff + k] = (double)acc[r];
  }
}

__global__ void nn_wreduce_kernel(NnArgs n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NN_NPARAM) return;
  double s = 0.0;
  for (int b = 0; b < n.nwblk; ++b) s += n.partial[(long long)b * NN_NPARAM + k];
  n.w_bar[k] += s;
}

__device__ __forceinline__ double nn_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// image reverse: network-input adjoint -> WENO face-state adjoints (added to a.fadj) and
// d/dgamma of the face energies (added to pbar[0]); 32 x 32 pixel tiles as nn_image_kernel
template <class T>
__global__ void __launch_bounds__(256) nn_image_vjp_kernel(NnArgs n, AdjArgs a) {
  __shared__ T sx[4][IT][IT + 1];
  const int d = blockIdx.z;
  const int H = n.H[d], Wd = n.W[d];
  const int f0 = blockIdx.x * IT, h0 = blockIdx.y * IT;
  // per-warp partials of pbar[0] (gamma; the other three entries 0), summed with the other
  // partials of the stage in a fixed order: warp w of block b writes pp[4 (8 b + w) + k]
  const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
  const long long pw = 4 * (8 * blk + (threadIdx.x >> 5));
  if (f0 >= Wd || h0 >= H) {  // uniform per block
    if (a.pp && (threadIdx.x & 31) < 4) a.pp[pw + (threadIdx.x & 31)] = 0.0;
    return;
  }
  const long long pix = (long long)H * Wd;
  const T* dX = chan_img<T>(n.G4, 4, d, n.pix0);
  for (int e = threadIdx.x; e < 4 * IT * IT; e += 256) {
    const int k = e / (IT * IT), r = e % (IT * IT), h = h0 + r / IT, f = f0 + r % IT;
    sx[k][r / IT][r % IT] = (h < H && f < Wd) ? dX[k * pix + (long long)h * Wd + f] : (T)0;
  }
  __syncthreads();
  double gbar = 0.0;
  const int hl = threadIdx.x % IT;
  const int un = (d == 0) ? 1 : 2, ut = (d == 0) ? 2 : 1;
  const int fdir = d * 8;
  for (int fl = threadIdx.x / IT; fl < IT; fl += 256 / IT) {
    const int h = h0 + hl, f = f0 + fl;
    if (h >= H || f >= Wd) continue;
    double wl[4], wr[4];
    face_states_any(n, a.lay, a.Q, a.lay.plane, d, h, f, wl, wr);
    double gk[4];  // adjoint of each side's conserved frame state (the image is their mean)
#pragma unroll
    for (int k = 0; k < 4; ++k) gk[k] = 0.5 * n.inv_sd[k] * (double)sx[k][hl][fl];
    const long long si = (d == 0) ? (long long)(f + 3) * a.tpitch + (h + a.lay.gy) : a.lay.idx(h, f);
    for (int sd = 0; sd < 2; ++sd) {
      const double* w = (sd == 0) ? wl : wr;
      const double r = w[0], vn = w[un], vt = w[ut], pr = w[3];
      double b[4];
      b[0] = fma(0.5 * fma(vn, vn, vt * vt), gk[3], fma(vn, gk[1], fma(vt, gk[2], gk[0])));
      b[un] = r * fma(vn, gk[3], gk[1]);
      b[ut] = r * fma(vt, gk[3], gk[2]);
      b[3] = gk[3] * n.g1;
      gbar -= pr * n.g1 * n.g1 * gk[3];
#pragma unroll
      for (int c = 0; c < 4; ++c) a.fadj[(long long)(fdir + 4 * sd + c) * a.splane + si] += b[c];
    }
  }
  gbar = nn_warp_sum(gbar);
  const int lane = threadIdx.x & 31;
  if (a.pp && lane < 4) a.pp[pw + lane] = (lane == 0) ? gbar : 0.0;
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

long long max_pix(const NnArgs& n) {
  long long m = (long long)n.H[0] * n.W[0];
  if (n.nimg > 1 && (long long)n.H[1] * n.W[1] > m) m = (long long)n.H[1] * n.W[1];
  return m;
}

dim3 image_grid(const NnArgs& n) {
  int W = n.W[0], H = n.H[0];
  if (n.nimg > 1) {
    W = W > n.W[1] ? W : n.W[1];
    H = H > n.H[1] ? H : n.H[1];
  }
  return dim3(cdiv(W, IT), cdiv(H, IT), n.nimg);
}

dim3 tile_grid(const NnArgs& n) {
  int W = n.W[0], H = n.H[0];
  if (n.nimg > 1) {
    W = W > n.W[1] ? W : n.W[1];
    H = H > n.H[1] ? H : n.H[1];
  }
  return dim3(cdiv(W, TILE), cdiv(H, TILE), n.nimg);
}

template <class T, int CIN, int COUT, int ACT>
cudaError_t conv(const NnArgs& n, const void* in, void* out, int woff, cudaStream_t s, void* outh = nullptr) {
  if (std::is_same<T, float>::value) {
    const size_t sm = sizeof(float) * (CIN * 9 * COUT + COUT + CIN * TH * TH);
    auto k = nn_conv_f32_kernel<CIN, COUT, ACT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<tile_grid(n), NTHR_F, sm, s>>>(n, in, out, woff, outh);
    return cudaGetLastError();
  }
  constexpr int NW = COUT * CIN * 9 + COUT;
  const size_t sm = sizeof(T) * (((NW + 1) & ~1) + CIN * TH * TH);
  auto k = nn_conv_kernel<T, CIN, COUT, ACT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<tile_grid(n), NTHR, sm, s>>>(n, in, out, woff);
  return cudaGetLastError();
}

template <class T, int CIN, int COUT, bool MASK>
cudaError_t dgrad(const NnArgs& n, const void* gout, const void* aprev, void* gin, int woff, cudaStream_t s) {
  if (std::is_same<T, float>::value) {
    const size_t sm = sizeof(float) * (COUT * 9 * CIN + COUT * TH * TH);
    auto k = nn_dgrad_f32_kernel<CIN, COUT, MASK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<tile_grid(n), NTHR_F, sm, s>>>(n, gout, aprev, gin, woff);
    return cudaGetLastError();
  }
  constexpr int NWW = COUT * CIN * 9;
  const size_t sm = sizeof(T) * (((NWW + 1) & ~1) + COUT * TH * TH);
  auto k = nn_dgrad_kernel<T, CIN, COUT, MASK>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<tile_grid(n), NTHR, sm, s>>>(n, gout, aprev, gin, woff);
  return cudaGetLastError();
}

// BF16 weight gradient on the tensor cores: one block per weight-gradient partial sum
template <int CIN, int COUT>
cudaError_t wgrad_tc(const NnArgs& n, const void* gout, const void* ain, int woff, cudaStream_t s) {
  using P = WgTc<CIN, COUT>;
  auto k = nn_wgrad_tc_kernel<CIN, COUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM);
  if (e != cudaSuccess) return e;
  k<<<n.nwblk, WNT, P::SMEM, s>>>(n, static_cast<const float*>(gout), static_cast<const float*>(ain), woff);
  return cudaGetLastError();
}

template <class T, int CIN, int COUT>
cudaError_t wgrad(const NnArgs& n, const void* gout, const void* ain, int woff, cudaStream_t s) {
  // BF16 precision: layers 2 and 3 on the tensor cores (the first layer's 4 input channels leave
  // its tensor-core form slower than the FP32 kernel)
  if (std::is_same<T, float>::value && n.bf16 && CIN >= 16) return wgrad_tc<CIN, COUT>(n, gout, ain, woff, s);
  if (std::is_same<T, float>::value) {
    const size_t tiles = 2 * wgrad_tile_floats<CIN, COUT>(), sums = WG_UNITS * 12 + NTHR;
    const size_t sm = sizeof(float) * (tiles > sums ? tiles : sums);
    auto k = nn_wgrad_f32_kernel<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<n.nwblk, NTHR, sm, s>>>(n, gout, ain, woff);
    return cudaGetLastError();
  }
  const size_t sm = sizeof(T) * (COUT * NTHR + CIN * TH * TH);
  auto k = nn_wgrad_kernel<T, CIN, COUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<n.nwblk, NTHR, sm, s>>>(n, gout, ain, woff);
  return cudaGetLastError();
}

template <int CIN, int COUT, int ACT, int MODE = 0, int CINR = CIN>
cudaError_t conv_tc(const NnArgs& n, const void* inh, void* out, int woff, cudaStream_t s, void* outh = nullptr,
                    const void* aprev = nullptr) {
  constexpr int N = (COUT + 15) / 16 * 16;
  const size_t sm = tc_aregion(CIN) + 9 * (CIN / 8) * N * 16 + COUT * sizeof(float);
  auto k = nn_conv_tc_kernel<CIN, COUT, ACT, MODE, CINR>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // one block per work item: the occupancy query reports one block per SM for this kernel
  // (it allocates tensor memory), while shared memory admits several, which the hardware
  // co-schedules; each block allocates its 32 tensor-memory columns once and frees them
  long long items = 0;
  for (int d = 0; d < n.nimg; ++d) items += (long long)cdiv(n.W[d], TC_M) * cdiv(n.H[d], TC_ROWS);
  k<<<(unsigned)items, 128, sm, s>>>(n, inh, out, woff, outh, aprev);
  return cudaGetLastError();
}

// the fused network kernel: rows per band about one wave of co-resident blocks (shared memory
// admits three per SM), at least 16 (each band recomputes 6 rows of layers 1 and 2 at its top)
cudaError_t net_tc(const NnArgs& n, cudaStream_t s) {
  auto k = nn_net_tc_kernel;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, NF_SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  long long rows = 0;
  int hmax = 1;
  for (int d = 0; d < n.nimg; ++d) {
    rows += (long long)cdiv(n.W[d], NF_OUT) * n.H[d];
    hmax = n.H[d] > hmax ? n.H[d] : hmax;
  }
  long long band = (rows + 3LL * sms - 1) / (3LL * sms);
  band = band < 16 ? 16 : (band > hmax ? hmax : band);
  long long items = 0;
  for (int d = 0; d < n.nimg; ++d) items += (long long)cdiv(n.W[d], NF_OUT) * ((n.H[d] + band - 1) / band);
  k<<<(unsigned)items, 128, NF_SMEM, s>>>(n, (int)band);
  return cudaGetLastError();
}

// the three layers on n.X -> n.T3
template <class T>
cudaError_t layers_t(const NnArgs& n, cudaStream_t s) {
  cudaError_t e;
  const bool tc = std::is_same<T, float>::value && n.bf16;
  if (tc && !n.keep && n.fused) return net_tc(n, s);
  // (the tensor-core layers read BF16 pixel-major copies written by the step before them: the
  // input's into the G16 scratch; their FP32 activations are written only for a reverse pass)
  if (tc) {
    void* a1 = n.keep ? n.A1 : nullptr;
    void* a2 = n.keep ? n.A2 : nullptr;
    const long long pix = n.pix0 + (n.nimg > 1 ? (long long)n.H[1] * n.W[1] : 0LL);
    __nv_bfloat16* xh = static_cast<__nv_bfloat16*>(n.G16);
    nn_x16_kernel<<<(unsigned)((pix + 255) / 256), 256, 0, s>>>(n, xh);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = conv_tc<16, 16, 0, 0, 4>(n, xh, a1, NN_OFF1, s, n.A1h)) != cudaSuccess) return e;
    if ((e = conv_tc<16, 32, 0>(n, n.A1h, a2, NN_OFF2, s, n.A2h)) != cudaSuccess) return e;
    return conv_tc<32, 4, 1>(n, n.A2h, n.T3, NN_OFF3, s);
  }
  if ((e = conv<T, 4, 16, 0>(n, n.X, n.A1, NN_OFF1, s)) != cudaSuccess) return e;
  if ((e = conv<T, 16, 32, 0>(n, n.A1, n.A2, NN_OFF2, s)) != cudaSuccess) return e;
  return conv<T, 32, 4, 1>(n, n.A2, n.T3, NN_OFF3, s);
}

template <class T>
cudaError_t forward_t(const NnArgs& n, const double* Q, long long qplane, cudaStream_t s) {
  nn_image_kernel<T><<<image_grid(n), 256, 0, s>>>(n, Q, qplane);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return layers_t<T>(n, s);
}

template <class T>
cudaError_t eval_t(const NnArgs& n0, const double* X, int H, int W, double* Y, cudaStream_t s) {
  NnArgs n = n0;
  n.nimg = 1;
  n.H[0] = H;
  n.W[0] = W;
  n.pix0 = (long long)H * W;
  const long long pix = n.pix0;
  nn_load_kernel<T><<<cdiv(4 * pix, 256), 256, 0, s>>>(X, static_cast<T*>(n.X), 4 * pix);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = layers_t<T>(n, s)) != cudaSuccess) return e;
  nn_store_kernel<T><<<cdiv(4 * pix, 256), 256, 0, s>>>(static_cast<const T*>(n.T3), Y, pix, n);
  return cudaGetLastError();
}

// no more weight-gradient blocks than tiles (small images leave most blocks idle)
NnArgs capped_wblocks(const NnArgs& n0) {
  NnArgs n = n0;
  long long tiles = 0;
  for (int d = 0; d < n.nimg; ++d) tiles += (long long)cdiv(n.W[d], TILE) * cdiv(n.H[d], TILE);
  if (tiles < n.nwblk) n.nwblk = (int)tiles;
  return n;
}

// the layers' reverse from G4 = dZ3 (activations A1, A2 of the forward in place): data gradients
// down to G4 = dX, weight gradients added to w_bar when it is set.  BF16 mode: the data
// gradients of layers 3 and 2 run on the tensor cores, reading BF16 pixel-major copies of G4
// (written by the seed into the A1h buffer) and G32 (into A2h): the forward's BF16 activations
// are no longer needed there.
template <class T>
cudaError_t layers_vjp_t(const NnArgs& n, cudaStream_t s) {
  cudaError_t e;
  const bool tc = std::is_same<T, float>::value && n.bf16;
  if (tc) e = conv_tc<16, 32, 1, 1, 4>(n, n.A1h, n.G32, NN_OFF3, s, n.A2h, n.A2);                 // G32 = dZ2
  else e = dgrad<T, 32, 4, true>(n, n.G4, n.A2, n.G32, NN_OFF3, s);
  if (e != cudaSuccess) return e;
  if (n.w_bar && (e = wgrad<T, 32, 4>(n, n.G4, n.A2, NN_OFF3, s)) != cudaSuccess) return e;
  if (tc) e = conv_tc<32, 16, 1, 1>(n, n.A2h, n.G16, NN_OFF2, s, nullptr, n.A1);                   // G16 = dZ1
  else e = dgrad<T, 16, 32, true>(n, n.G32, n.A1, n.G16, NN_OFF2, s);
  if (e != cudaSuccess) return e;
  if (n.w_bar && (e = wgrad<T, 16, 32>(n, n.G32, n.A1, NN_OFF2, s)) != cudaSuccess) return e;
  if ((e = dgrad<T, 4, 16, false>(n, n.G16, nullptr, n.G4, NN_OFF1, s)) != cudaSuccess) return e;  // G4 = dX
  if (n.w_bar) {
    if ((e = wgrad<T, 4, 16>(n, n.G16, n.X, NN_OFF1, s)) != cudaSuccess) return e;
    nn_wreduce_kernel<<<cdiv(NN_NPARAM, 256), 256, 0, s>>>(n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t reverse_t(const NnArgs& n0, const AdjArgs& a, cudaStream_t s) {
  NnArgs n = capped_wblocks(n0);
  n.keep = 1;
  cudaError_t e = n.fwd_ready ? cudaSuccess : forward_t<T>(n, a.Q, a.lay.plane, s);  // else kept
  if (e != cudaSuccess) return e;
  const dim3 pg(cdiv(max_pix(n), 256), n.nimg);
  const bool tc = std::is_same<T, float>::value && n.bf16;
  nn_seed_kernel<T><<<pg, 256, 0, s>>>(n, a, tc ? static_cast<__nv_bfloat16*>(n.A1h) : nullptr);  // G4 = dZ3
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = layers_vjp_t<T>(n, s)) != cudaSuccess) return e;
  nn_image_vjp_kernel<T><<<image_grid(n), 256, 0, s>>>(n, a);
  return cudaGetLastError();
}

template <class T>
cudaError_t eval_vjp_t(const NnArgs& n0, const double* X, int H, int W, const double* GY, double* GX,
                       cudaStream_t s) {
  NnArgs n = n0;
  n.nimg = 1;
  n.H[0] = H;
  n.W[0] = W;
  n.pix0 = (long long)H * W;
  n = capped_wblocks(n);
  n.keep = 1;
  const long long pix = n.pix0;
  nn_load_kernel<T><<<cdiv(4 * pix, 256), 256, 0, s>>>(X, static_cast<T*>(n.X), 4 * pix);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = layers_t<T>(n, s)) != cudaSuccess) return e;
  const bool tc = std::is_same<T, float>::value && n.bf16;
  nn_seed_eval_kernel<T><<<cdiv(pix, 256), 256, 0, s>>>(n, GY, pix, tc ? static_cast<__nv_bfloat16*>(n.A1h) : nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = layers_vjp_t<T>(n, s)) != cudaSuccess) return e;
  nn_unload_kernel<T><<<cdiv(4 * pix, 256), 256, 0, s>>>(static_cast<const T*>(n.G4), GX, 4 * pix);
  return cudaGetLastError();
}

}  // namespace

cudaError_t nn_prims(const double* U, double* Q, const Lay& lay, double gamma, cudaStream_t s) {
  nn_prims_kernel<<<cdiv(lay.plane, 256), 256, 0, s>>>(U, Q, lay, Gas{gamma, gamma - 1.0, 1.0 / (gamma - 1.0)});
  return cudaGetLastError();
}

cudaError_t nn_forward(const NnArgs& n, const double* Q, long long qplane, cudaStream_t s) {
  return n.fp32 ? forward_t<float>(n, Q, qplane, s) : forward_t<double>(n, Q, qplane, s);
}

cudaError_t nn_layers(const NnArgs& n, cudaStream_t s) {
  return n.fp32 ? layers_t<float>(n, s) : layers_t<double>(n, s);
}

cudaError_t nn_eval(const NnArgs& n, const double* X, int H, int W, double* Y, cudaStream_t s) {
  return n.fp32 ? eval_t<float>(n, X, H, W, Y, s) : eval_t<double>(n, X, H, W, Y, s);
}

cudaError_t nn_eval_vjp(const NnArgs& n, const double* X, int H, int W, const double* GY, double* GX,
                        cudaStream_t s) {
  return n.fp32 ? eval_vjp_t<float>(n, X, H, W, GY, GX, s) : eval_vjp_t<double>(n, X, H, W, GY, GX, s);
}

cudaError_t nn_apply(const NnArgs& n, const StageArgs& a, bool rhs, cudaStream_t s) {
  const dim3 grid(cdiv(a.lay.nx, IT), cdiv(a.lay.ny, IT));
  if (n.fp32) nn_apply_kernel<float><<<grid, 256, 0, s>>>(n, a, rhs ? 1 : 0);
  else nn_apply_kernel<double><<<grid, 256, 0, s>>>(n, a, rhs ? 1 : 0);
  return cudaGetLastError();
}

long long nn_image_vjp_blocks(const Lay& lay) {
  NnArgs n;
  n.nimg = lay.ny > 1 ? 2 : 1;
  n.H[0] = lay.ny;
  n.W[0] = lay.nx + 1;
  n.H[1] = lay.nx;
  n.W[1] = lay.ny + 1;
  const dim3 g = image_grid(n);
  return (long long)g.x * g.y * g.z;
}

cudaError_t nn_reverse(const NnArgs& n, const AdjArgs& a, cudaStream_t s) {
  // pass 1 has run: on 2D grids a.wsave holds the stage's WENO5 internals
  NnArgs m = n;
  m.wsave = a.two_d ? a.wsave : nullptr;
  m.splane = a.splane;
  m.tpitch = a.tpitch;
  return m.fp32 ? reverse_t<float>(m, a, s) : reverse_t<double>(m, a, s);
}

// ---------------------------------------------------------------------------------------
// block averaging of a state (the downsampling d(U) that makes the training targets of
// Sec. 2.4 from high-resolution runs)
// ---------------------------------------------------------------------------------------
namespace {
__global__ void block_average_kernel(const double* __restrict__ U, int nx, int ny, int fx, int fy,
                                     double* __restrict__ out) {
  const int cx = nx / fx, cy = ny / fy;
  const long long n = (long long)cx * cy;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * n) return;
  const int c = (int)(t / n);
  const long long o = t % n;
  const int i = (int)(o % cx), j = (int)(o / cx);
  const double* u = U + (long long)c * nx * ny;
  double s = 0.0;
  for (int b = 0; b < fy; ++b)
    for (int a = 0; a < fx; ++a) s += u[(long long)(j * fy + b) * nx + i * fx + a];
  out[t] = s / (double)(fx * fy);
}
}  // namespace

cudaError_t launch_block_average(const double* U, int nx, int ny, int fx, int fy, double* out, cudaStream_t s) {
  const long long n = 4LL * (nx / fx) * (ny / fy);
  block_average_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(U, nx, ny, fx, fy, out);
  return cudaGetLastError();
}

}  // namespace js
