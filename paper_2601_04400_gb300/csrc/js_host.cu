// Host side of libjaxshock.so: solver contexts, immersed-boundary precomputation and the
// C ABI declared in include/jaxshock.h.
#include <cuda.h>  // tensor-map types only; the encoder is looked up at run time
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "jaxshock.h"
#include "js_internal.h"

using js::BcArgs;
using js::IbArgs;
using js::Lay;
using js::StageArgs;

struct js_ctx {
  js_grid g;
  js_params p;
  js_boundary b;
  Lay lay;
  cudaStream_t stream = nullptr;
  double* N = nullptr;  // padded U^n / step output
  double* A = nullptr;  // padded stage buffers
  double* B = nullptr;
  double* acc = nullptr;   // stage scratch [4][ny][nx]: x-flux differences
  double* acc2 = nullptr;  // y-flux differences
  unsigned char* tag = nullptr;       // device [ny][nx] or null (no immersed body)
  std::vector<unsigned char> tag_host;
  int n_ghost = 0;
  long long* ib_dst = nullptr;
  long long* ib_src = nullptr;
  double* ib_w = nullptr;
  double* ib_nrm = nullptr;
  int* err = nullptr;
  unsigned long long* red = nullptr;
  double* cfl_bmax = nullptr;  // per-block scratch of the CFL reduction
  double* dtc = nullptr;       // stage constants of the device step size (js_step_cfl)
  BcArgs bc;
  // transposed IB tables
  int n_src = 0;
  long long* ibt_cell = nullptr;
  int* ibt_ptr = nullptr;
  int* ibt_ghost = nullptr;
  double* ibt_w = nullptr;
  // adjoint workspace (allocated by the first vjp call)
  bool adj_ready = false;
  double* Q = nullptr;       // 5 planes
  double* fcell = nullptr;   // 24 saved planes: per-face adjoints for the cells of the face
  double* wrev = nullptr;    // pass-2 segment slots (js::adj_wrev_doubles)
  double* ppart = nullptr;   // block partials of the parameter gradient (js::adj_ppart_doubles)
  double* lam = nullptr;     // 4 planes
  double* P0 = nullptr;      // 4 planes (stage adjoint ping)
  double* P1 = nullptr;      // 4 planes (pong)
  double* Uacc = nullptr;    // 4 planes
  double* wsave = nullptr;   // 56 planes
  double* wsave_fwd = nullptr;  // 2 x 56 planes: internals stored by the forward stages 1, 2
  double* fadj = nullptr;    // 16 planes
  double* inflow_part = nullptr;  // [4 sides][max(nx + 6, ny)][4] inflow halo adjoint partials
  double* inflow_prim = nullptr;  // 16
  double* inflow_host = nullptr;  // 16, pinned
  bool inflow_dirty = true;       // inflow_prim to be uploaded
  double* qIb = nullptr;     // 4 per ghost
  // neural flux (js_set_neural)
  bool nn_on = false;
  js::NnArgs nn;
  double* nnQ = nullptr;        // primitives of the stage input (4 planes)
  double* nn_wsave = nullptr;   // WENO5 internals of the current stage (2D; 56 planes)
  void* nn_buf[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void* nn_bf16[2] = {nullptr, nullptr};  // BF16 pixel-major activations (16 and 32 channels)
  // network input and activations (X, A1, A2, T3: 56 channels) of the forward stages 0 and 1 of
  // js_step_vjp, kept for their reverse (allocated by the first js_step_vjp with the network on)
  void* nn_keep[2] = {nullptr, nullptr};
  bool nn_keep_failed = false;
  double* nn_partial = nullptr;
  int variant = 0;  // stage-kernel tile shape (js_set_tuning)
  int arith = JS_ARITH_FAST;  // js_set_arith
  js::IeeeBufs ieee = {nullptr, nullptr, nullptr};  // workspace of JS_ARITH_IEEE
  std::vector<std::pair<const double*, js::TensorMap128>> tmaps;  // TMA maps of stage inputs
  // tape: per slot the three filled stage states of one recorded step and, when recording
  // internals (2D), the WENO5 internals of its three stages
  std::vector<double*> tape;
  std::vector<double*> tape_w;     // 3 per slot (56 planes each) or nullptr
  std::vector<char> tape_w_ok;     // per slot: internals of the recorded step are present
  bool tape_weno = false;
  // y slab of a decomposed grid (js_create_slab): local row k is global row
  // (slab_lo + k) mod slab_nyg; rows [slab_own, slab_own + slab_nown) are owned; the y sides
  // in slab_xchg[0] (low) / [1] (high) border a neighbouring slab
  bool slab = false;
  int slab_nyg = 0, slab_lo = 0, slab_own = 0, slab_nown = 0;
  bool slab_xchg[2] = {false, false};
  int svjp_next = 2;  // stage expected by the next js_step_stage_vjp (2, 1, 0, 2, ...)
  bool stage_kept[2] = {false, false};  // js_step_stage stored stage 0 / 1 internals in wsave_fwd
  // instrumentation
  bool profiling = false;
  std::vector<cudaEvent_t> ev;  // 2 per timed stage launch
  int ev_used = 0;
  long long launches = 0;
};

namespace {

#define JS_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return JS_ERR_CUDA;              \
  } while (0)

bool grid_valid(const js_grid* g) {
  if (!g || g->nx < 6 || g->ny < 1 || (g->ny > 1 && g->ny < 6)) return false;
  if (!(g->dx > 0.0) || !(g->dy > 0.0)) return false;
  if ((long long)g->nx * g->ny > (1LL << 31)) return false;
  return true;
}

bool params_valid(const js_params* p, const js_boundary* b) {
  if (!p || !b) return false;
  if (!(p->gamma > 1.0) || !(p->mu >= 0.0) || !(p->nu >= 0.0)) return false;
  if (p->mu > 0.0 && !(p->Pr > 0.0)) return false;
  if (p->wall != 0 && p->wall != 1) return false;
  for (int s = 0; s < 4; ++s)
    if (b->kind[s] < JS_BC_TRANSMISSIVE || b->kind[s] > JS_BC_INFLOW) return false;
  return true;
}

void set_bc(js_ctx* c) {
  for (int s = 0; s < 4; ++s) {
    // a side bordering a neighbouring slab: transmissive ghost layers (they reach only overlap
    // rows, which the halo exchange overwrites)
    c->bc.kind[s] = (s >= 2 && c->slab_xchg[s - 2]) ? JS_BC_TRANSMISSIVE : c->b.kind[s];
    const double r = c->b.inflow[s][0], u = c->b.inflow[s][1], v = c->b.inflow[s][2], pr = c->b.inflow[s][3];
    c->bc.inflow_cons[s][0] = r;
    c->bc.inflow_cons[s][1] = r * u;
    c->bc.inflow_cons[s][2] = r * v;
    c->bc.inflow_cons[s][3] = pr / (c->p.gamma - 1.0) + 0.5 * r * (u * u + v * v);
  }
}

// Ghost-cell IB tables (Sec. 2, Fig. 1(c)): solid = sdf < 0; ghost = solid cell with a fluid
// cell in its 7x7 box; normal = normalised gradient of sdf (central differences, one-sided
// at grid edges); image point = ghost centre - 2 sdf n; bilinear weights over the 2x2 block
// of cell centres around it (clamped into the grid), restricted to fluid cells and
// renormalised.
// The tables cover the context's rows, a window of a grid of nyg rows (global y origin y0g):
// local row k is global row (row_lo + k) mod nyg, and every quantity above is evaluated on the
// global grid, so that the entries equal those of the whole grid.  A ghost cell whose
// interpolation cells leave the window is frozen (tagged plain solid, not filled) unless its
// row lies in [exact_lo, exact_hi), which is an error.
int build_ib(js_ctx* c, const double* sdf, int nyg, double y0g, int row_lo, int exact_lo, int exact_hi) {
  const int nx = c->g.nx, ny = c->g.ny;
  const double dx = c->g.dx, dy = c->g.dy, x0 = c->g.x0;
  std::vector<unsigned char>& tag = c->tag_host;
  tag.assign((size_t)nx * ny, 0);
  auto S = [&](int i, int jg) { return sdf[(size_t)jg * nx + i]; };
  auto glob = [&](int k) { return (row_lo + k) % nyg; };
  auto loc = [&](int jg) {
    const int k = ((jg - row_lo) % nyg + nyg) % nyg;
    return k < ny ? k : -1;
  };
  for (int k = 0; k < ny; ++k)
    for (int i = 0; i < nx; ++i) tag[(size_t)k * nx + i] = (S(i, glob(k)) < 0.0) ? 1 : 0;
  for (int k = 0; k < ny; ++k)
    for (int i = 0; i < nx; ++i) {
      if (tag[(size_t)k * nx + i] == 0) continue;
      const int j = glob(k);
      bool fluid_near = false;
      for (int jj = j - 3; jj <= j + 3 && !fluid_near; ++jj)
        for (int ii = i - 3; ii <= i + 3; ++ii) {
          if (ii < 0 || jj < 0 || ii >= nx || jj >= nyg) continue;
          if (!(S(ii, jj) < 0.0)) { fluid_near = true; break; }
        }
      if (fluid_near) tag[(size_t)k * nx + i] = 2;
    }
  std::vector<long long> dst, src;
  std::vector<double> w, nrm;
  for (int k = 0; k < ny; ++k)
    for (int i = 0; i < nx; ++i) {
      if (tag[(size_t)k * nx + i] != 2) continue;
      const int j = glob(k);
      const int il = i > 0 ? i - 1 : i, ir = i < nx - 1 ? i + 1 : i;
      const int jl = j > 0 ? j - 1 : j, jr = j < nyg - 1 ? j + 1 : j;
      const double gx = (S(ir, j) - S(il, j)) / ((ir - il) * dx);
      const double gy = (S(i, jr) - S(i, jl)) / ((jr - jl) * dy);
      const double gn = std::sqrt(gx * gx + gy * gy);
      if (!(gn > 0.0)) return JS_ERR_IB;
      const double nxv = gx / gn, nyv = gy / gn;
      const double phi = S(i, j);
      const double xg = x0 + (i + 0.5) * dx, yg = y0g + (j + 0.5) * dy;
      const double xi = xg - 2.0 * phi * nxv, yi = yg - 2.0 * phi * nyv;
      const double fx = (xi - x0) / dx - 0.5, fy = (yi - y0g) / dy - 0.5;
      if (!(fx >= -0.5 && fy >= -0.5 && fx <= nx - 0.5 && fy <= nyg - 0.5)) return JS_ERR_IB;
      int i0 = (int)std::floor(fx), j0 = (int)std::floor(fy);
      i0 = i0 < 0 ? 0 : (i0 > nx - 2 ? nx - 2 : i0);
      j0 = j0 < 0 ? 0 : (j0 > nyg - 2 ? nyg - 2 : j0);
      const int k0 = loc(j0), k1 = loc(j0 + 1);
      if (k0 < 0 || k1 < 0) {
        if (k >= exact_lo && k < exact_hi) return JS_ERR_IB;
        tag[(size_t)k * nx + i] = 1;
        continue;
      }
      const double tx = fx - i0, ty = fy - j0;
      const int ci[4] = {i0, i0 + 1, i0, i0 + 1}, ck[4] = {k0, k0, k1, k1};
      double wk[4] = {(1.0 - tx) * (1.0 - ty), tx * (1.0 - ty), (1.0 - tx) * ty, tx * ty};
      double sum = 0.0;
      for (int m = 0; m < 4; ++m) {
        if (tag[(size_t)ck[m] * nx + ci[m]] != 0) wk[m] = 0.0;
        sum = sum + wk[m];
      }
      if (!(sum > 0.0)) return JS_ERR_IB;
      dst.push_back(c->lay.idx(i, k));
      for (int m = 0; m < 4; ++m) {
        src.push_back(c->lay.idx(ci[m], ck[m]));
        w.push_back(wk[m] / sum);
      }
      nrm.push_back(nxv);
      nrm.push_back(nyv);
    }
  c->n_ghost = (int)dst.size();
  // transposed tables: fluid source cell -> (ghost, weight), grouped by cell
  {
    std::vector<std::pair<long long, std::pair<int, double>>> ent;
    for (int k = 0; k < c->n_ghost; ++k)
      for (int m = 0; m < 4; ++m)
        if (w[4 * k + m] != 0.0) ent.push_back({src[4 * k + m], {k, w[4 * k + m]}});
    std::stable_sort(ent.begin(), ent.end(),
                     [](const auto& x, const auto& y) { return x.first < y.first; });
    std::vector<long long> cell;
    std::vector<int> ptr, gh;
    std::vector<double> ww;
    for (size_t e = 0; e < ent.size(); ++e) {
      if (e == 0 || ent[e].first != ent[e - 1].first) {
        cell.push_back(ent[e].first);
        ptr.push_back((int)e);
      }
      gh.push_back(ent[e].second.first);
      ww.push_back(ent[e].second.second);
    }
    ptr.push_back((int)ent.size());
    c->n_src = (int)cell.size();
    if (c->n_src > 0) {
      if (cudaMalloc(&c->ibt_cell, cell.size() * sizeof(long long)) != cudaSuccess ||
          cudaMalloc(&c->ibt_ptr, ptr.size() * sizeof(int)) != cudaSuccess ||
          cudaMalloc(&c->ibt_ghost, gh.size() * sizeof(int)) != cudaSuccess ||
          cudaMalloc(&c->ibt_w, ww.size() * sizeof(double)) != cudaSuccess)
        return JS_ERR_NOMEM;
      JS_CUDA(cudaMemcpy(c->ibt_cell, cell.data(), cell.size() * sizeof(long long), cudaMemcpyHostToDevice));
      JS_CUDA(cudaMemcpy(c->ibt_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
      JS_CUDA(cudaMemcpy(c->ibt_ghost, gh.data(), gh.size() * sizeof(int), cudaMemcpyHostToDevice));
      JS_CUDA(cudaMemcpy(c->ibt_w, ww.data(), ww.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
  }
  if (cudaMalloc(&c->tag, tag.size()) != cudaSuccess) return JS_ERR_NOMEM;
  JS_CUDA(cudaMemcpy(c->tag, tag.data(), tag.size(), cudaMemcpyHostToDevice));
  if (c->n_ghost > 0) {
    const size_t ng = (size_t)c->n_ghost;
    if (cudaMalloc(&c->ib_dst, ng * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&c->ib_src, 4 * ng * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&c->ib_w, 4 * ng * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->ib_nrm, 2 * ng * sizeof(double)) != cudaSuccess)
      return JS_ERR_NOMEM;
    JS_CUDA(cudaMemcpy(c->ib_dst, dst.data(), ng * sizeof(long long), cudaMemcpyHostToDevice));
    JS_CUDA(cudaMemcpy(c->ib_src, src.data(), 4 * ng * sizeof(long long), cudaMemcpyHostToDevice));
    JS_CUDA(cudaMemcpy(c->ib_w, w.data(), 4 * ng * sizeof(double), cudaMemcpyHostToDevice));
    JS_CUDA(cudaMemcpy(c->ib_nrm, nrm.data(), 2 * ng * sizeof(double), cudaMemcpyHostToDevice));
  }
  return JS_OK;
}

IbArgs ib_args(const js_ctx* c) {
  IbArgs a;
  a.n = c->n_ghost;
  a.dst = c->ib_dst;
  a.src = c->ib_src;
  a.w = c->ib_w;
  a.nrm = c->ib_nrm;
  return a;
}

// stage arguments common to js_rhs and js_step; cx, cy, av* and rk_* set by the caller
StageArgs base_args(const js_ctx* c) {
  StageArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tag = c->tag;
  a.acc = c->acc;
  a.acc2 = c->acc2;
  a.err = c->err;
  a.lay = c->lay;
  a.gamma = c->p.gamma;
  a.gm1 = c->p.gamma - 1.0;
  a.g1 = 1.0 / (c->p.gamma - 1.0);
  const double mu = c->p.mu, dx = c->g.dx, dy = c->g.dy;
  const double kappa = (mu > 0.0) ? mu * c->p.gamma / ((c->p.gamma - 1.0) * c->p.Pr) : 0.0;
  a.vx = js::ViscC{(4.0 / 3.0) * mu / dx, (2.0 / 3.0) * mu / (4.0 * dy), mu / dx, mu / (4.0 * dy), kappa / dx};
  a.vy = js::ViscC{(4.0 / 3.0) * mu / dy, (2.0 / 3.0) * mu / (4.0 * dx), mu / dy, mu / (4.0 * dx), kappa / dy};
  a.has_av = c->p.nu > 0.0 ? 1 : 0;
  return a;
}

int fill_halos(js_ctx* c, double* X, bool ieee = false) {
  if (ieee)
    JS_CUDA(js::launch_ieee_ib_fill(X, c->lay, ib_args(c), c->p.gamma, c->p.wall, c->stream));
  else
    JS_CUDA(js::launch_ib_fill(X, c->lay, ib_args(c), c->p.gamma, c->p.wall, c->stream));
  JS_CUDA(js::launch_bc_fill(X, c->lay, c->bc, c->stream));
  c->launches += (c->n_ghost > 0) ? 2 : 1;
  return JS_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor map of a padded state buffer: 3D (column, row, plane) FP64 tensor, box of the
// 32x32 tile with its 3-cell halo and all 4 planes; reads past the array return zeros.
const js::TensorMap128* stage_tmap(js_ctx* c, const double* buf) {
  if (c->lay.ny == 1) return nullptr;
  for (auto& e : c->tmaps)
    if (e.first == buf) return &e.second;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return nullptr;
  static_assert(sizeof(CUtensorMap) == sizeof(js::TensorMap128), "tensor map size");
  js::TensorMap128 m;
  const cuuint64_t dims[3] = {(cuuint64_t)c->lay.pitch, (cuuint64_t)c->lay.H, 4};
  const cuuint64_t strides[2] = {(cuuint64_t)c->lay.pitch * sizeof(double), (cuuint64_t)c->lay.plane * sizeof(double)};
  const cuuint32_t box[3] = {js::TMA_TX + 6, js::TMA_TY + 6, 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(reinterpret_cast<CUtensorMap*>(&m), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)buf, dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return nullptr;
  c->tmaps.push_back({buf, m});
  return &c->tmaps.back().second;
}

// neural flux of the stage input a.Uin (before the stage kernel) and its divergence
// subtracted from the stage output (after it)
// (wsave: the stage's stored WENO5 internals, or nullptr to recompute the face states)
int nn_before(js_ctx* c, const StageArgs& a, const double* wsave = nullptr, long long splane = 0, int tpitch = 0) {
  if (!c->nn_on) return JS_OK;
  c->nn.g1 = 1.0 / (c->p.gamma - 1.0);
  js::NnArgs n = c->nn;
  n.wsave = wsave;
  n.splane = splane;
  n.tpitch = tpitch;
  JS_CUDA(js::nn_prims(a.Uin, c->nnQ, c->lay, c->p.gamma, c->stream));
  JS_CUDA(js::nn_forward(n, c->nnQ, c->lay.plane, c->stream));
  c->launches += 5;
  return JS_OK;
}
int nn_after(js_ctx* c, const StageArgs& a, bool rhs) {
  if (!c->nn_on) return JS_OK;
  JS_CUDA(js::nn_apply(c->nn, a, rhs, c->stream));
  ++c->launches;
  return JS_OK;
}

// saved-array layouts: y lines padded (pitch x H), x lines transposed ((nx+6) x tpitch)
int transposed_pitch(const js_ctx* c) { return (c->lay.H + 3) / 4 * 4; }
long long saved_plane(const js_ctx* c) {
  const long long t = (long long)(c->lay.nx + 6) * transposed_pitch(c);
  const long long m = t > c->lay.plane ? t : c->lay.plane;
  return (m + 31) / 32 * 32;
}

size_t internals_bytes(const js_ctx* c) { return sizeof(double) * 56 * (size_t)saved_plane(c); }

// stage update that also stores its WENO5 internals to `wsave` (2D), bracketed by events
// while profiling like stage()
int stage_save(js_ctx* c, StageArgs a, bool visc, double* wsave) {
  a.wsave = wsave;
  a.splane = saved_plane(c);
  a.tpitch = transposed_pitch(c);
  const bool timed = c->profiling && c->ev_used + 2 <= (int)c->ev.size();
  if (timed) JS_CUDA(cudaEventRecord(c->ev[c->ev_used], c->stream));
  JS_CUDA(js::launch_stage_save(a, visc, stage_tmap(c, a.Uin), c->stream));
  if (timed) {
    JS_CUDA(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
    c->ev_used += 2;
  }
  ++c->launches;
  int rc = nn_before(c, a, wsave, a.splane, a.tpitch);
  if (rc) return rc;
  return nn_after(c, a, false);
}

// fused stage kernel, bracketed by events while profiling
// stage update that also writes the FP32 face images of the neural flux (FP32 and BF16
// networks on 2D grids), then the network and its divergence
int stage_img(js_ctx* c, StageArgs a, bool visc) {
  a.img = static_cast<float*>(c->nn.X);
  for (int k = 0; k < 4; ++k) {
    a.img_mean[k] = (float)c->nn.mean[k];
    a.img_isd[k] = (float)c->nn.inv_sd[k];
  }
  a.img_g1 = (float)(1.0 / (c->p.gamma - 1.0));
  const bool timed = c->profiling && c->ev_used + 2 <= (int)c->ev.size();
  if (timed) JS_CUDA(cudaEventRecord(c->ev[c->ev_used], c->stream));
  JS_CUDA(js::launch_stage_img(a, visc, stage_tmap(c, a.Uin), c->stream));
  if (timed) {
    JS_CUDA(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
    c->ev_used += 2;
  }
  JS_CUDA(js::nn_layers(c->nn, c->stream));
  c->launches += 4;
  return nn_after(c, a, false);
}

int stage(js_ctx* c, const StageArgs& a, bool visc, bool rhs) {
  // with the neural flux on a 2D grid the stage kernel also forms the network's face images
  // (FP32 and BF16 networks) or stores the WENO5 internals they are formed from (FP64)
  if (c->nn_on && !rhs && c->g.ny > 1 && c->nn.fp32) return stage_img(c, a, visc);
  if (c->nn_on && c->nn_wsave && !rhs) return stage_save(c, a, visc, c->nn_wsave);
  int rc = nn_before(c, a);
  if (rc) return rc;
  const bool timed = c->profiling && c->ev_used + 2 <= (int)c->ev.size();
  if (timed) JS_CUDA(cudaEventRecord(c->ev[c->ev_used], c->stream));
  const js::TensorMap128* tm = (c->variant == 0) ? stage_tmap(c, a.Uin) : nullptr;
  JS_CUDA(js::launch_stage(a, visc, rhs, c->variant, tm, c->stream));
  if (timed) {
    JS_CUDA(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
    c->ev_used += 2;
  }
  ++c->launches;
  return nn_after(c, a, rhs);
}

// a forward stage (or the RHS) of js_rhs / js_step / js_step_stage in the context's arithmetic
// mode: the fused stage kernel, or the IEEE-order kernels (stage k of step size dt)
int stage_fwd(js_ctx* c, const StageArgs& a, bool rhs, double dt, int k) {
  if (c->arith != JS_ARITH_IEEE) return stage(c, a, c->p.mu > 0.0, rhs);
  if (c->nn_on) return JS_ERR_ARG;
  JS_CUDA(js::launch_ieee_stage(a, c->ieee, dt, k, rhs, c->p.mu, c->p.Pr, c->p.nu, c->g.dx, c->g.dy, c->stream));
  c->launches += (c->g.ny > 1) ? 4 : 3;
  return JS_OK;
}

}  // namespace

// batched kernel description of a context (used by js_batch.cu)
void js_internal_desc(js_ctx* c, js::InstDesc* d) {
  std::memset(d, 0, sizeof(*d));
  d->lay = c->lay;
  d->N = c->N;
  d->A = c->A;
  d->B = c->B;
  d->acc = c->acc;
  d->acc2 = c->acc2;
  d->tag = c->tag;
  d->ib = ib_args(c);
  d->bc = c->bc;
  d->gamma = c->p.gamma;
  d->mu = c->p.mu;
  d->Pr = c->p.Pr;
  d->nu = c->p.nu;
  d->dx = c->g.dx;
  d->dy = c->g.dy;
  d->hmin = (c->g.ny > 1) ? (c->g.dx < c->g.dy ? c->g.dx : c->g.dy) : c->g.dx;
  d->lim = (c->p.mu > 0.0) ? ((4.0 / 3.0 < c->p.gamma / c->p.Pr) ? c->p.gamma / c->p.Pr : 4.0 / 3.0) : 1.0;
  const StageArgs a = base_args(c);
  d->vx = a.vx;
  d->vy = a.vy;
  d->wall = c->p.wall;
  d->visc = c->p.mu > 0.0 ? 1 : 0;
  d->has_av = c->p.nu > 0.0 ? 1 : 0;
}

extern "C" {

const char* js_strerror(int code) {
  switch (code) {
    case JS_OK: return "ok";
    case JS_ERR_ARG: return "invalid argument";
    case JS_ERR_CUDA: return "CUDA runtime error";
    case JS_ERR_NONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or NaN in a fluid cell)";
    case JS_ERR_TIMEOUT: return "bounded device wait timed out";
    case JS_ERR_IB: return "immersed boundary: image point outside the domain or without fluid neighbour";
    case JS_ERR_NOMEM: return "device allocation failed";
    default: return "unknown error";
  }
}

void js_destroy(js_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  cudaFree(c->N); cudaFree(c->A); cudaFree(c->B); cudaFree(c->acc); cudaFree(c->acc2);
  cudaFree(c->tag);
  cudaFree(c->ib_dst); cudaFree(c->ib_src); cudaFree(c->ib_w); cudaFree(c->ib_nrm);
  cudaFree(c->err); cudaFree(c->red); cudaFree(c->cfl_bmax); cudaFree(c->dtc);
  cudaFree(c->ieee.Q); cudaFree(c->ieee.F); cudaFree(c->ieee.G);
  cudaFree(c->ibt_cell); cudaFree(c->ibt_ptr); cudaFree(c->ibt_ghost); cudaFree(c->ibt_w);
  cudaFree(c->Q); cudaFree(c->fcell); cudaFree(c->wrev); cudaFree(c->ppart); cudaFree(c->lam); cudaFree(c->P0); cudaFree(c->P1); cudaFree(c->Uacc);
  cudaFree(c->wsave); cudaFree(c->wsave_fwd); cudaFree(c->fadj);
  if (c->inflow_host) cudaFreeHost(c->inflow_host);
  cudaFree(c->nnQ); cudaFree(c->nn_partial); cudaFree(c->nn_wsave);
  for (void* b : c->nn_buf) cudaFree(b);
  for (void* b : c->nn_bf16) cudaFree(b);
  for (void* b : c->nn_keep) cudaFree(b);
  cudaFree(c->inflow_part); cudaFree(c->inflow_prim); cudaFree(c->qIb);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  for (double* t : c->tape) cudaFree(t);
  for (double* t : c->tape_w) cudaFree(t);
  delete c;
}

}  // extern "C"

namespace {

// a context over `grid` (a whole grid, or the window of a slab described by `slab`); the IB
// tables come from the sdf of the whole grid (nyg rows, y origin y0g)
struct SlabDesc {
  bool on;
  int nyg, lo, own, nown;
  bool xchg[2];
  double y0g;
};

int create_ctx(const js_grid* grid, const js_params* params, const js_boundary* bc, const double* sdf_host,
               void* stream, const SlabDesc& sd, js_ctx** out) {
  js_ctx* c = new (std::nothrow) js_ctx();
  if (!c) return JS_ERR_NOMEM;
  c->slab = sd.on;
  c->slab_nyg = sd.nyg;
  c->slab_lo = sd.lo;
  c->slab_own = sd.own;
  c->slab_nown = sd.nown;
  c->slab_xchg[0] = sd.xchg[0];
  c->slab_xchg[1] = sd.xchg[1];
  c->g = *grid;
  c->p = *params;
  c->b = *bc;
  c->stream = (cudaStream_t)stream;
  Lay& L = c->lay;
  L.nx = grid->nx;
  L.ny = grid->ny;
  L.gy = (grid->ny == 1) ? 0 : 3;
  L.pitch = ((grid->nx + 6) + 3) / 4 * 4;  // 32-byte aligned rows
  L.H = grid->ny + 2 * L.gy;
  L.plane = ((long long)L.pitch * L.H + 31) / 32 * 32;
  const size_t bytes = sizeof(double) * 4 * (size_t)L.plane;
  if (cudaMalloc(&c->N, bytes) != cudaSuccess || cudaMalloc(&c->A, bytes) != cudaSuccess ||
      cudaMalloc(&c->B, bytes) != cudaSuccess || cudaMalloc(&c->err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->acc, sizeof(double) * 4 * (size_t)grid->nx * grid->ny) != cudaSuccess ||
      cudaMalloc(&c->acc2, sizeof(double) * 4 * (size_t)grid->nx * grid->ny) != cudaSuccess ||
      cudaMalloc(&c->red, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&c->cfl_bmax, sizeof(double) * js::CFL_MAX_BLOCKS) != cudaSuccess ||
      cudaMalloc(&c->dtc, sizeof(double) * js::DTC_N) != cudaSuccess) {
    js_destroy(c);
    return JS_ERR_NOMEM;
  }
  // padding never holds NaN garbage
  // (a device-wide synchronisation: the context's stream may be a non-blocking one that does
  // not wait for work on the legacy default stream)
  if (cudaMemset(c->N, 0, bytes) != cudaSuccess || cudaMemset(c->A, 0, bytes) != cudaSuccess ||
      cudaMemset(c->B, 0, bytes) != cudaSuccess || cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    js_destroy(c);
    return JS_ERR_CUDA;
  }
  set_bc(c);
  if (sdf_host) {
    // ghost cells within 3 rows of the owned rows feed owned stage outputs: they must be exact
    const int lo = sd.on ? sd.own - 3 : 0, hi = sd.on ? sd.own + sd.nown + 3 : grid->ny;
    const int rc = build_ib(c, sdf_host, sd.nyg, sd.y0g, sd.lo, lo, hi);
    if (rc != JS_OK) {
      js_destroy(c);
      return rc;
    }
  }
  *out = c;
  return JS_OK;
}

}  // namespace

extern "C" {

int js_create(const js_grid* grid, const js_params* params, const js_boundary* bc, const double* sdf_host,
              void* stream, js_ctx** out) {
  if (!out) return JS_ERR_ARG;
  *out = nullptr;
  if (!grid_valid(grid) || !params_valid(params, bc)) return JS_ERR_ARG;
  if (sdf_host && grid->ny == 1) return JS_ERR_ARG;
  const SlabDesc sd{false, grid->ny, 0, 0, grid->ny, {false, false}, grid->y0};
  return create_ctx(grid, params, bc, sdf_host, stream, sd, out);
}

int js_create_slab(const js_grid* grid, const js_params* params, const js_boundary* bc, const double* sdf_host,
                   int row0, int nrows, int overlap, void* stream, js_ctx** out) {
  if (!out) return JS_ERR_ARG;
  *out = nullptr;
  if (!grid_valid(grid) || !params_valid(params, bc) || grid->ny == 1) return JS_ERR_ARG;
  const int ny = grid->ny;
  if (row0 < 0 || nrows < 1 || row0 + nrows > ny || overlap < 0) return JS_ERR_ARG;
  const bool py0 = bc->kind[2] == JS_BC_PERIODIC, py1 = bc->kind[3] == JS_BC_PERIODIC;
  SlabDesc sd{true, ny, 0, row0, nrows, {false, false}, grid->y0};
  int rows = ny;
  if (nrows < ny) {
    if (overlap < 3 || py0 != py1) return JS_ERR_ARG;
    if (py0) {
      if (nrows + 2 * overlap > ny) return JS_ERR_ARG;
      sd.lo = ((row0 - overlap) % ny + ny) % ny;
      rows = nrows + 2 * overlap;
      sd.xchg[0] = sd.xchg[1] = true;
    } else {
      sd.lo = row0 > overlap ? row0 - overlap : 0;
      const int hi = (row0 + nrows + overlap < ny) ? row0 + nrows + overlap : ny;
      rows = hi - sd.lo;
      sd.xchg[0] = row0 > 0;
      sd.xchg[1] = row0 + nrows < ny;
    }
  }
  sd.own = (nrows < ny) ? ((row0 - sd.lo) % ny + ny) % ny : 0;
  js_grid g = *grid;
  g.ny = rows;
  g.y0 = grid->y0 + sd.lo * grid->dy;
  if (!grid_valid(&g)) return JS_ERR_ARG;
  return create_ctx(&g, params, bc, sdf_host, stream, sd, out);
}

int js_slab_info(js_ctx* c, int* row_lo, int* rows, int* own_lo, int* own_rows) {
  if (!c) return JS_ERR_ARG;
  if (row_lo) *row_lo = c->slab ? c->slab_lo : 0;
  if (rows) *rows = c->g.ny;
  if (own_lo) *own_lo = c->slab ? c->slab_own : 0;
  if (own_rows) *own_rows = c->slab ? c->slab_nown : c->g.ny;
  return JS_OK;
}

int js_rows_pack(js_ctx* c, double* U, int row0, int nrows, double* buf, int zero) {
  if (!c || !U || !buf || row0 < 0 || nrows < 0 || row0 + nrows > c->g.ny) return JS_ERR_ARG;
  JS_CUDA(js::launch_rows_pack(U, c->g.nx, c->g.ny, row0, nrows, buf, zero, c->stream));
  ++c->launches;
  return JS_OK;
}

int js_rows_unpack(js_ctx* c, double* U, int row0, int nrows, const double* buf, int add) {
  if (!c || !U || !buf || row0 < 0 || nrows < 0 || row0 + nrows > c->g.ny) return JS_ERR_ARG;
  JS_CUDA(js::launch_rows_unpack(U, c->g.nx, c->g.ny, row0, nrows, buf, add, c->stream));
  ++c->launches;
  return JS_OK;
}

int js_block_average(const double* U, int nx, int ny, int fx, int fy, double* out, void* stream) {
  if (!U || !out || nx < 1 || ny < 1 || fx < 1 || fy < 1 || nx % fx != 0 || ny % fy != 0) return JS_ERR_ARG;
  JS_CUDA(js::launch_block_average(U, nx, ny, fx, fy, out, static_cast<cudaStream_t>(stream)));
  return JS_OK;
}

int js_set_params(js_ctx* c, const js_params* params, const js_boundary* bc) {
  if (!c || !params_valid(params, bc)) return JS_ERR_ARG;
  c->p = *params;
  c->b = *bc;
  c->inflow_dirty = true;
  set_bc(c);
  return JS_OK;
}

int js_set_stream(js_ctx* c, void* stream) {
  if (!c) return JS_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return JS_OK;
}

int js_prim_to_cons(js_ctx* c, const double* W, double* U) {
  if (!c || !W || !U) return JS_ERR_ARG;
  JS_CUDA(js::launch_prim_to_cons(W, U, (long long)c->g.nx * c->g.ny, c->p.gamma, c->stream));
  return JS_OK;
}

int js_rhs(js_ctx* c, const double* U, double* dUdt) {
  if (!c || !U || !dUdt || U == dUdt) return JS_ERR_ARG;
  JS_CUDA(js::launch_pack(U, c->N, c->lay, c->stream));
  ++c->launches;
  int rc = fill_halos(c, c->N, c->arith == JS_ARITH_IEEE);
  if (rc) return rc;
  StageArgs a = base_args(c);
  a.Uin = c->N;
  a.Un = nullptr;
  a.Uout = dUdt;
  a.cx = 1.0 / c->g.dx;
  a.cy = 1.0 / c->g.dy;
  a.avx = c->p.nu / (c->g.dx * c->g.dx);
  a.avy = c->p.nu / (c->g.dy * c->g.dy);
  a.rk_a = 0.0;
  a.rk_b = 1.0;
  a.use_un = 0;
  return stage_fwd(c, a, true, 0.0, 0);
}

int js_max_dt(js_ctx* c, const double* U, double cfl, double* dt_out) {
  if (!c || !U || !dt_out || !(cfl > 0.0)) return JS_ERR_ARG;
  JS_CUDA(js::launch_cfl(U, c->lay, c->tag, c->p.gamma, c->g.dx, c->g.dy, c->red, c->cfl_bmax, c->stream));
  c->launches += 3;
  unsigned long long h[2];
  JS_CUDA(cudaMemcpyAsync(h, c->red, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  JS_CUDA(cudaStreamSynchronize(c->stream));
  double rate, rmin;
  std::memcpy(&rate, &h[0], sizeof(double));
  std::memcpy(&rmin, &h[1], sizeof(double));
  double dt = cfl / rate;
  if (c->p.mu > 0.0) {
    const double h2 = (c->g.ny > 1) ? (c->g.dx < c->g.dy ? c->g.dx : c->g.dy) : c->g.dx;
    const double lim = (4.0 / 3.0 < c->p.gamma / c->p.Pr) ? c->p.gamma / c->p.Pr : 4.0 / 3.0;
    const double dtv = cfl * h2 * h2 * rmin / (2.0 * c->p.mu * lim);
    dt = (dtv < dt) ? dtv : dt;
  }
  *dt_out = dt;
  if (!std::isfinite(dt) || !(dt > 0.0)) return JS_ERR_NONPHYSICAL;
  return JS_OK;
}

int js_step(js_ctx* c, double* U, double dt, int n_steps) {
  if (!c || !U || n_steps < 0 || !(dt > 0.0)) return JS_ERR_ARG;
  if (n_steps == 0) return JS_OK;
  JS_CUDA(js::launch_pack(U, c->N, c->lay, c->stream));
  StageArgs a = base_args(c);
  a.cx = dt / c->g.dx;
  a.cy = dt / c->g.dy;
  a.avx = dt * c->p.nu / (c->g.dx * c->g.dx);
  a.avy = dt * c->p.nu / (c->g.dy * c->g.dy);
  const bool visc = c->p.mu > 0.0;
  double* in[3] = {c->N, c->A, c->B};
  double* outp[3] = {c->A, c->B, c->N};
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int k = 0; k < n_steps; ++k) {
    for (int s = 0; s < 3; ++s) {
      int rc = fill_halos(c, in[s], c->arith == JS_ARITH_IEEE);
      if (rc) return rc;
      a.Uin = in[s];
      a.Un = c->N;
      a.Uout = outp[s];
      a.rk_a = ra[s];
      a.rk_b = rb[s];
      a.use_un = (s > 0) ? 1 : 0;
      rc = (c->arith == JS_ARITH_IEEE) ? stage_fwd(c, a, false, dt, s) : stage(c, a, visc, false);
      if (rc) return rc;
    }
  }
  JS_CUDA(js::launch_unpack(c->N, U, c->lay, c->stream));
  c->launches += 2;  // pack + unpack
  return JS_OK;
}

int js_step_cfl(js_ctx* c, double* U, double cfl, int n_steps, double* t_dev, double t_end, double* dt_log) {
  if (!c || !U || n_steps < 0 || !(cfl > 0.0) || c->nn_on) return JS_ERR_ARG;
  const bool ieee = c->arith == JS_ARITH_IEEE;
  const bool visc = c->p.mu > 0.0;
  const double hmin = (c->g.ny > 1) ? (c->g.dx < c->g.dy ? c->g.dx : c->g.dy) : c->g.dx;
  const double lim = visc ? ((4.0 / 3.0 < c->p.gamma / c->p.Pr) ? c->p.gamma / c->p.Pr : 4.0 / 3.0) : 0.0;
  double* in[3] = {c->N, c->A, c->B};
  double* outp[3] = {c->A, c->B, c->N};
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  StageArgs a = base_args(c);
  a.dtc = c->dtc;
  if (n_steps == 0) return JS_OK;
  // the state stays in the padded buffer N from the first step to the last
  JS_CUDA(js::launch_pack(U, c->N, c->lay, c->stream));
  ++c->launches;
  for (int k = 0; k < n_steps; ++k) {
    JS_CUDA(js::launch_cfl(c->N, c->lay, c->tag, c->p.gamma, c->g.dx, c->g.dy, c->red, c->cfl_bmax, c->stream,
                           true));
    JS_CUDA(js::launch_cfl_dt(c->red, cfl, c->g.dx, c->g.dy, c->p.nu, c->p.mu, lim, hmin, t_dev, t_end, c->dtc,
                              dt_log, k, c->err, c->stream));
    c->launches += 4;
    for (int s = 0; s < 3; ++s) {
      int rc = fill_halos(c, in[s], ieee);
      if (rc) return rc;
      a.Uin = in[s];
      a.Un = c->N;
      a.Uout = outp[s];
      a.rk_a = ra[s];
      a.rk_b = rb[s];
      a.use_un = (s > 0) ? 1 : 0;
      rc = ieee ? stage_fwd(c, a, false, 0.0, s) : stage(c, a, visc, false);
      if (rc) return rc;
    }
  }
  JS_CUDA(js::launch_unpack(c->N, U, c->lay, c->stream));
  ++c->launches;
  return JS_OK;
}

namespace {
int adj_reserve(js_ctx* c);  // defined with the reverse-pass entry points below
}  // namespace

int js_step_stage(js_ctx* c, const double* U_n, const double* U_in, double* U_out, double dt, int stage_flags) {
  const int stage_k = stage_flags & ~JS_STAGE_INTERNALS;
  if (!c || !U_in || !U_out || stage_k < 0 || stage_k > 2 || !(dt > 0.0) || (stage_k > 0 && !U_n))
    return JS_ERR_ARG;
  // stages 0 and 1 of a 2D grid may store their WENO5 internals for js_step_stage_vjp
  const bool keep = (stage_flags & JS_STAGE_INTERNALS) && stage_k < 2 && c->g.ny > 1;
  if (keep) {
    const int rc = adj_reserve(c);
    if (rc) return rc;
    if (!c->wsave_fwd) return JS_ERR_NOMEM;
  }
  double* X = (stage_k == 0) ? c->N : c->A;
  JS_CUDA(js::launch_pack(U_in, X, c->lay, c->stream));
  ++c->launches;
  if (stage_k > 0) {
    JS_CUDA(js::launch_pack(U_n, c->N, c->lay, c->stream));
    ++c->launches;
  }
  StageArgs a = base_args(c);
  a.cx = dt / c->g.dx;
  a.cy = dt / c->g.dy;
  a.avx = dt * c->p.nu / (c->g.dx * c->g.dx);
  a.avy = dt * c->p.nu / (c->g.dy * c->g.dy);
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  int rc = fill_halos(c, X, !keep && c->arith == JS_ARITH_IEEE);
  if (rc) return rc;
  a.Uin = X;
  a.Un = c->N;
  a.Uout = c->B;
  a.rk_a = ra[stage_k];
  a.rk_b = rb[stage_k];
  a.use_un = (stage_k > 0) ? 1 : 0;
  if (keep) rc = stage_save(c, a, c->p.mu > 0.0, c->wsave_fwd + 56 * (size_t)saved_plane(c) * stage_k);
  else rc = stage_fwd(c, a, false, dt, stage_k);
  if (rc) return rc;
  if (stage_k < 2) c->stage_kept[stage_k] = keep;
  JS_CUDA(js::launch_unpack(c->B, U_out, c->lay, c->stream));
  ++c->launches;
  return JS_OK;
}

namespace {

int adj_reserve(js_ctx* c) {
  if (c->adj_ready) return JS_OK;
  const size_t pl = sizeof(double) * (size_t)c->lay.plane;
  struct { double** p; size_t planes; } bufs[] = {
      {&c->Q, 5}, {&c->lam, 4}, {&c->P0, 4}, {&c->P1, 4}, {&c->Uacc, 4}};
  for (auto& b : bufs) {
    if (cudaMalloc(b.p, b.planes * pl) != cudaSuccess) return JS_ERR_NOMEM;
    JS_CUDA(cudaMemsetAsync(*b.p, 0, b.planes * pl, c->stream));  // ordered with the caller's work
  }
  const size_t spl = sizeof(double) * (size_t)saved_plane(c);
  if (cudaMalloc(&c->wsave, 2 * 4 * 7 * spl) != cudaSuccess || cudaMalloc(&c->fadj, 16 * spl) != cudaSuccess)
    return JS_ERR_NOMEM;
  JS_CUDA(cudaMemsetAsync(c->wsave, 0, 2 * 4 * 7 * spl, c->stream));
  JS_CUDA(cudaMemsetAsync(c->fadj, 0, 16 * spl, c->stream));
  // internals stored by the forward stages 1, 2 of js_step_vjp (2D)
  if (c->g.ny > 1) {
    if (cudaMalloc(&c->wsave_fwd, 2 * 56 * spl) != cudaSuccess) {
      c->wsave_fwd = nullptr;
      return JS_ERR_NOMEM;
    }
    JS_CUDA(cudaMemsetAsync(c->wsave_fwd, 0, 2 * 56 * spl, c->stream));
  }
  const size_t tmax = (size_t)std::max(c->g.nx + 6, c->g.ny);
  const size_t npp = (size_t)js::adj_ppart_doubles(c->lay, c->n_ghost, c->n_src, js::nn_image_vjp_blocks(c->lay));
  if (cudaMalloc(&c->fcell, 24 * spl) != cudaSuccess ||
      cudaMalloc(&c->wrev, sizeof(double) * (size_t)js::adj_wrev_doubles(c->lay)) != cudaSuccess ||
      cudaMalloc(&c->ppart, sizeof(double) * npp) != cudaSuccess)
    return JS_ERR_NOMEM;
  if (cudaMalloc(&c->inflow_part, sizeof(double) * 16 * tmax) != cudaSuccess ||
      cudaMalloc(&c->inflow_prim, 16 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->qIb, sizeof(double) * 4 * (size_t)(c->n_ghost > 0 ? c->n_ghost : 1)) != cudaSuccess)
    return JS_ERR_NOMEM;
  c->adj_ready = true;
  return JS_OK;
}

js::AdjArgs adj_args(js_ctx* c, const double* X, double* Ub, double* p_bar) {
  js::AdjArgs a;
  std::memset(&a, 0, sizeof(a));
  a.lay = c->lay;
  a.X = X;
  a.Q = c->Q;
  a.lam = c->lam;
  a.fcell = c->fcell;
  a.wrev = c->wrev;
  a.pp = c->ppart;
  a.Ub = Ub;
  a.wsave = c->wsave;
  a.fadj = c->fadj;
  a.splane = saved_plane(c);
  a.tpitch = transposed_pitch(c);
  a.pbar = p_bar;
  a.tag = c->tag;
  const double g = c->p.gamma;
  a.gas = js::Gas{g, g - 1.0, 1.0 / (g - 1.0)};
  a.inv_dx = 1.0 / c->g.dx;
  a.inv_dy = 1.0 / c->g.dy;
  a.nu_x1 = 1.0 / (c->g.dx * c->g.dx);
  a.nu_y1 = 1.0 / (c->g.dy * c->g.dy);
  a.nu_x = c->p.nu * a.nu_x1;
  a.nu_y = c->p.nu * a.nu_y1;
  const StageArgs s = base_args(c);
  a.vx = s.vx;
  a.vy = s.vy;
  a.visc = c->p.mu > 0.0 ? 1 : 0;
  a.inv_mu = a.visc ? 1.0 / c->p.mu : 0.0;
  a.kg = -1.0 / (g * (g - 1.0));
  a.kp = a.visc ? -1.0 / c->p.Pr : 0.0;
  a.has_av = c->p.nu > 0.0 ? 1 : 0;
  a.two_d = c->g.ny > 1 ? 1 : 0;
  return a;
}

js::IbTArgs ibt_args(const js_ctx* c) {
  js::IbTArgs t;
  t.nsrc = c->n_src;
  t.cell = c->ibt_cell;
  t.ptr = c->ibt_ptr;
  t.ghost = c->ibt_ghost;
  t.w = c->ibt_w;
  return t;
}

// one stage VJP; `saved` = WENO internals of this stage stored by its forward (or nullptr:
// pass 1 recomputes them into the context's own buffer)
int adj_stage(js_ctx* c, const double* X, const double* Unext, double* Ub, double ra, double rb, double dt,
              bool rhs_mode, double* p_bar, double* saved = nullptr) {
  js::AdjArgs a = adj_args(c, X, Ub, p_bar);
  if (saved) {
    a.wsave = saved;
    a.weno_saved = 1;
  }
  c->nn.g1 = 1.0 / (c->p.gamma - 1.0);
  JS_CUDA(js::launch_adj_stage(a, c->bc, ib_args(c), ibt_args(c), c->p.wall, Unext, c->Uacc, ra, rb, dt, rhs_mode,
                               c->inflow_part, c->inflow_prim, c->qIb, c->stream, &c->launches,
                               c->nn_on ? &c->nn : nullptr));
  return JS_OK;
}

// the inflow states on the device for the reverse pass: uploaded from a pinned buffer when
// they changed (js_create / js_set_params), so that reverse calls do not block the host
int upload_inflow(js_ctx* c) {
  if (!c->inflow_dirty) return JS_OK;
  if (!c->inflow_host && cudaMallocHost(&c->inflow_host, 16 * sizeof(double)) != cudaSuccess) {
    c->inflow_host = nullptr;
    return JS_ERR_NOMEM;
  }
  // the previous upload from this buffer must have completed before it is rewritten
  JS_CUDA(cudaStreamSynchronize(c->stream));
  for (int s = 0; s < 4; ++s)
    for (int k = 0; k < 4; ++k) c->inflow_host[4 * s + k] = c->b.inflow[s][k];
  JS_CUDA(cudaMemcpyAsync(c->inflow_prim, c->inflow_host, 16 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  c->inflow_dirty = false;
  return JS_OK;
}

}  // namespace

int js_rhs_vjp(js_ctx* c, const double* U, const double* lam, double* U_bar, double* p_bar) {
  if (!c || !U || !lam || !U_bar) return JS_ERR_ARG;
  c->svjp_next = 2;  // the stage-wise reverse sequence (js_step_stage_vjp) restarts
  int rc = adj_reserve(c);
  if (rc) return rc;
  if ((rc = upload_inflow(c))) return rc;
  JS_CUDA(js::launch_pack(U, c->N, c->lay, c->stream));
  JS_CUDA(js::launch_pack(lam, c->P0, c->lay, c->stream));
  c->launches += 2;
  if ((rc = fill_halos(c, c->N))) return rc;
  if ((rc = adj_stage(c, c->N, c->P0, c->P1, 0.0, 1.0, 1.0, true, p_bar))) return rc;
  JS_CUDA(js::launch_adj_unpack(c->P1, nullptr, U_bar, c->lay, c->stream));
  ++c->launches;
  return JS_OK;
}

namespace {

// the network's kept forward of stage s (0, 1) of js_step_vjp: c->nn points at set s while the
// forward stage runs (keep = 1) and while its reverse runs (fwd_ready = 1); false when the sets
// are unavailable (the reverse then recomputes the forward)
bool nn_keep_ready(js_ctx* c) {
  if (!c->nn_on || c->nn_keep_failed) return false;
  if (c->nn_keep[0] && c->nn_keep[1]) return true;
  const size_t pix = (size_t)(c->nn.pix0 + (long long)c->nn.H[1] * c->nn.W[1]);
  for (int k = 0; k < 2; ++k)
    if (!c->nn_keep[k] && cudaMalloc(&c->nn_keep[k], sizeof(double) * 56 * pix) != cudaSuccess) {
      c->nn_keep[k] = nullptr;
      cudaGetLastError();  // clear the allocation error
      c->nn_keep_failed = true;
      return false;
    }
  return true;
}
js::NnArgs nn_use_kept(js_ctx* c, int s, bool reverse) {
  const js::NnArgs prev = c->nn;
  const size_t pix = (size_t)(c->nn.pix0 + (long long)c->nn.H[1] * c->nn.W[1]);
  const size_t el = c->nn.fp32 ? sizeof(float) : sizeof(double);
  char* b = static_cast<char*>(c->nn_keep[s]);
  c->nn.X = b;
  c->nn.A1 = b + el * 4 * pix;
  c->nn.A2 = b + el * 20 * pix;
  c->nn.T3 = b + el * 52 * pix;
  c->nn.keep = 1;
  c->nn.fwd_ready = reverse ? 1 : 0;
  return prev;
}

}  // namespace

int js_step_vjp(js_ctx* c, const double* U_n, double dt, const double* lam_np1, double* lam_n, double* p_bar) {
  if (!c || !U_n || !lam_np1 || !lam_n || !(dt > 0.0)) return JS_ERR_ARG;
  c->svjp_next = 2;  // the stage-wise reverse sequence (js_step_stage_vjp) restarts
  c->stage_kept[0] = c->stage_kept[1] = false;  // wsave_fwd is reused here
  int rc = adj_reserve(c);
  if (rc) return rc;
  if ((rc = upload_inflow(c))) return rc;
  // recompute and keep the three filled stage states X0 = N, X1 = A, X2 = B
  JS_CUDA(js::launch_pack(U_n, c->N, c->lay, c->stream));
  JS_CUDA(js::launch_pack(lam_np1, c->P0, c->lay, c->stream));
  c->launches += 2;
  StageArgs a = base_args(c);
  a.cx = dt / c->g.dx;
  a.cy = dt / c->g.dy;
  a.avx = dt * c->p.nu / (c->g.dx * c->g.dx);
  a.avy = dt * c->p.nu / (c->g.dy * c->g.dy);
  const bool visc = c->p.mu > 0.0;
  // 2D: the forward stages 1 and 2 also store their WENO internals, so that their reverse
  // skips the WENO recompute (stage 3 is not run forward; its pass 1 recomputes them)
  const bool keep = c->g.ny > 1 && c->wsave_fwd != nullptr;
  double* saved[3] = {keep ? c->wsave_fwd : nullptr,
                      keep ? c->wsave_fwd + 56 * (size_t)saved_plane(c) : nullptr, nullptr};
  double* in[2] = {c->N, c->A};
  double* outp[2] = {c->A, c->B};
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  // with the neural flux, the network's forward of stages 0 and 1 is kept for their reverse
  const bool nnk = nn_keep_ready(c);
  for (int s = 0; s < 2; ++s) {
    if ((rc = fill_halos(c, in[s]))) return rc;
    a.Uin = in[s];
    a.Un = c->N;
    a.Uout = outp[s];
    a.rk_a = ra[s];
    a.rk_b = rb[s];
    a.use_un = (s > 0) ? 1 : 0;
    const js::NnArgs prev = nnk ? nn_use_kept(c, s, false) : c->nn;
    rc = keep ? stage_save(c, a, visc, saved[s]) : stage(c, a, visc, false);
    c->nn = prev;
    if (rc) return rc;
  }
  if ((rc = fill_halos(c, c->B))) return rc;
  // reverse through the stages: P0 -> P1 -> P0 -> P1
  JS_CUDA(cudaMemsetAsync(c->Uacc, 0, sizeof(double) * 4 * (size_t)c->lay.plane, c->stream));
  double* X[3] = {c->N, c->A, c->B};
  double* src = c->P0;
  double* dst = c->P1;
  for (int s = 2; s >= 0; --s) {
    const js::NnArgs prev = (nnk && s < 2) ? nn_use_kept(c, s, true) : c->nn;
    rc = adj_stage(c, X[s], src, dst, ra[s], rb[s], dt, false, p_bar, saved[s]);
    c->nn = prev;
    if (rc) return rc;
    double* t = src;
    src = dst;
    dst = t;
  }
  JS_CUDA(js::launch_adj_unpack(src, c->Uacc, lam_n, c->lay, c->stream));
  ++c->launches;
  return JS_OK;
}

int js_step_stage_vjp(js_ctx* c, const double* U_in, double dt, int stage_flags, const double* lam_out,
                      double* lam_in, double* p_bar) {
  const int stage_k = stage_flags & ~JS_STAGE_INTERNALS;
  if (!c || !U_in || !lam_out || !lam_in || stage_k < 0 || stage_k > 2 || !(dt > 0.0)) return JS_ERR_ARG;
  if (stage_k != 2 && stage_k != c->svjp_next) return JS_ERR_ARG;
  const bool kept = (stage_flags & JS_STAGE_INTERNALS) && stage_k < 2 && c->g.ny > 1;
  if (kept && !c->stage_kept[stage_k]) return JS_ERR_ARG;
  int rc = adj_reserve(c);
  if (rc) return rc;
  if ((rc = upload_inflow(c))) return rc;
  JS_CUDA(js::launch_pack(U_in, c->N, c->lay, c->stream));
  JS_CUDA(js::launch_pack(lam_out, c->P0, c->lay, c->stream));
  c->launches += 2;
  if ((rc = fill_halos(c, c->N))) return rc;
  // the U^n adjoint of stages 2 and 1 collects in Uacc and is added to stage 0's result
  if (stage_k == 2) JS_CUDA(cudaMemsetAsync(c->Uacc, 0, sizeof(double) * 4 * (size_t)c->lay.plane, c->stream));
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  double* saved = kept ? c->wsave_fwd + 56 * (size_t)saved_plane(c) * stage_k : nullptr;
  if ((rc = adj_stage(c, c->N, c->P0, c->P1, ra[stage_k], rb[stage_k], dt, false, p_bar, saved))) return rc;
  JS_CUDA(js::launch_adj_unpack(c->P1, stage_k == 0 ? c->Uacc : nullptr, lam_in, c->lay, c->stream));
  ++c->launches;
  c->svjp_next = (stage_k == 0) ? 2 : stage_k - 1;
  return JS_OK;
}

namespace {
size_t state_bytes(const js_ctx* c) { return sizeof(double) * 4 * (size_t)c->lay.plane; }
double* tape_state(js_ctx* c, int slot, int s) { return c->tape[(size_t)slot * 3 + s]; }

// one SSP-RK3 step whose three stage inputs live in X[0..2] (X[0] already holds U^n);
// the step result goes to `out` (padded); W[s] (if non-null) receives stage s's internals
int step_through(js_ctx* c, double* const X[3], double* out, double dt, double* const W[3]) {
  StageArgs a = base_args(c);
  a.cx = dt / c->g.dx;
  a.cy = dt / c->g.dy;
  a.avx = dt * c->p.nu / (c->g.dx * c->g.dx);
  a.avy = dt * c->p.nu / (c->g.dy * c->g.dy);
  const bool visc = c->p.mu > 0.0;
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int s = 0; s < 3; ++s) {
    int rc = fill_halos(c, X[s]);
    if (rc) return rc;
    a.Uin = X[s];
    a.Un = X[0];
    a.Uout = (s < 2) ? X[s + 1] : out;
    a.rk_a = ra[s];
    a.rk_b = rb[s];
    a.use_un = (s > 0) ? 1 : 0;
    rc = W[s] ? stage_save(c, a, visc, W[s]) : stage(c, a, visc, false);
    if (rc) return rc;
  }
  return JS_OK;
}
}  // namespace

int js_tape_reserve_ex(js_ctx* c, int n_slots, int flags) {
  if (!c || n_slots < 0 || (flags & ~JS_TAPE_WENO) != 0) return JS_ERR_ARG;
  int rc = adj_reserve(c);
  if (rc) return rc;
  const size_t need = (size_t)n_slots * 3;
  while (c->tape.size() < need) {
    double* p = nullptr;
    if (cudaMalloc(&p, state_bytes(c)) != cudaSuccess) return JS_ERR_NOMEM;
    if (cudaMemsetAsync(p, 0, state_bytes(c), c->stream) != cudaSuccess) { cudaFree(p); return JS_ERR_CUDA; }
    c->tape.push_back(p);
  }
  c->tape_weno = (flags & JS_TAPE_WENO) != 0 && c->g.ny > 1;
  c->tape_w.resize(c->tape.size(), nullptr);
  c->tape_w_ok.resize(c->tape.size() / 3, 0);
  if (c->tape_weno) {
    for (size_t k = 0; k < need; ++k) {
      if (c->tape_w[k]) continue;
      if (cudaMalloc(&c->tape_w[k], internals_bytes(c)) != cudaSuccess) {
        c->tape_w[k] = nullptr;
        c->tape_weno = false;
        return JS_ERR_NOMEM;
      }
    }
  }
  JS_CUDA(cudaStreamSynchronize(c->stream));
  return JS_OK;
}

int js_tape_reserve(js_ctx* c, int n_slots) { return js_tape_reserve_ex(c, n_slots, 0); }

int js_step_taped(js_ctx* c, double* U, double dt, int slot) {
  if (!c || !U || !(dt > 0.0) || slot < 0 || (size_t)(slot + 1) * 3 > c->tape.size()) return JS_ERR_ARG;
  double* X[3] = {tape_state(c, slot, 0), tape_state(c, slot, 1), tape_state(c, slot, 2)};
  const size_t b = (size_t)slot * 3;
  const bool keep = c->tape_weno && c->tape_w[b] && c->tape_w[b + 1] && c->tape_w[b + 2];
  double* W[3] = {keep ? c->tape_w[b] : nullptr, keep ? c->tape_w[b + 1] : nullptr,
                  keep ? c->tape_w[b + 2] : nullptr};
  c->tape_w_ok[slot] = 0;
  JS_CUDA(js::launch_pack(U, X[0], c->lay, c->stream));
  int rc = step_through(c, X, c->N, dt, W);
  if (rc) return rc;
  c->tape_w_ok[slot] = keep ? 1 : 0;
  JS_CUDA(js::launch_unpack(c->N, U, c->lay, c->stream));
  c->launches += 2;
  return JS_OK;
}

int js_step_vjp_taped(js_ctx* c, int slot, double dt, const double* lam_np1, double* lam_n, double* p_bar) {
  if (!c || !lam_np1 || !lam_n || !(dt > 0.0) || slot < 0 || (size_t)(slot + 1) * 3 > c->tape.size())
    return JS_ERR_ARG;
  c->svjp_next = 2;
  int rc = adj_reserve(c);
  if (rc) return rc;
  if ((rc = upload_inflow(c))) return rc;
  JS_CUDA(js::launch_pack(lam_np1, c->P0, c->lay, c->stream));
  ++c->launches;
  JS_CUDA(cudaMemsetAsync(c->Uacc, 0, state_bytes(c), c->stream));
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  double* src = c->P0;
  double* dst = c->P1;
  const bool saved = c->tape_w_ok[slot] != 0;
  for (int s = 2; s >= 0; --s) {
    double* w = saved ? c->tape_w[(size_t)slot * 3 + s] : nullptr;
    if ((rc = adj_stage(c, tape_state(c, slot, s), src, dst, ra[s], rb[s], dt, false, p_bar, w))) return rc;
    double* t = src;
    src = dst;
    dst = t;
  }
  JS_CUDA(js::launch_adj_unpack(src, c->Uacc, lam_n, c->lay, c->stream));
  ++c->launches;
  return JS_OK;
}

int js_sync_status(js_ctx* c) {
  if (!c) return JS_ERR_ARG;
  int h = 0;
  JS_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  JS_CUDA(cudaStreamSynchronize(c->stream));
  JS_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
  JS_CUDA(cudaStreamSynchronize(c->stream));
  if (h & js::ERR_TIMEOUT_BIT) return JS_ERR_TIMEOUT;
  if (h & js::ERR_NONPHYSICAL_BIT) return JS_ERR_NONPHYSICAL;
  return JS_OK;
}

int js_set_arith(js_ctx* c, int mode) {
  if (!c || (mode != JS_ARITH_FAST && mode != JS_ARITH_IEEE)) return JS_ERR_ARG;
  if (mode == JS_ARITH_IEEE && !c->ieee.Q) {
    const size_t nx = (size_t)c->g.nx, ny = (size_t)c->g.ny;
    if (cudaMalloc(&c->ieee.Q, sizeof(double) * 4 * (size_t)c->lay.plane) != cudaSuccess ||
        cudaMalloc(&c->ieee.F, sizeof(double) * 4 * (nx + 1) * ny) != cudaSuccess ||
        (ny > 1 && cudaMalloc(&c->ieee.G, sizeof(double) * 4 * nx * (ny + 1)) != cudaSuccess)) {
      cudaFree(c->ieee.Q);
      cudaFree(c->ieee.F);
      c->ieee = {nullptr, nullptr, nullptr};
      return JS_ERR_NOMEM;
    }
  }
  c->arith = mode;
  return JS_OK;
}

int js_get_arith(js_ctx* c, int* mode) {
  if (!c || !mode) return JS_ERR_ARG;
  *mode = c->arith;
  return JS_OK;
}

int js_set_tuning(js_ctx* c, int variant) {
  if (!c || variant < 0 || variant >= js::STAGE_VARIANTS) return JS_ERR_ARG;
  c->variant = variant;
  return JS_OK;
}

int js_get_tuning(js_ctx* c, int* variant, int* n_variants) {
  if (!c) return JS_ERR_ARG;
  if (variant) *variant = c->variant;
  if (n_variants) *n_variants = js::STAGE_VARIANTS;
  return JS_OK;
}

int js_profile_begin(js_ctx* c, int capacity) {
  if (!c || capacity < 0) return JS_ERR_ARG;
  while ((int)c->ev.size() < 2 * capacity) {
    cudaEvent_t e;
    JS_CUDA(cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  c->ev_used = 0;
  c->launches = 0;
  c->profiling = true;
  return JS_OK;
}

int js_profile_end(js_ctx* c, double* stage_ms, int* stage_launches, long long* kernel_launches) {
  if (!c) return JS_ERR_ARG;
  JS_CUDA(cudaStreamSynchronize(c->stream));
  double total = 0.0;
  for (int k = 0; k + 1 < c->ev_used; k += 2) {
    float ms = 0.0f;
    JS_CUDA(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
    total += ms;
  }
  if (stage_ms) *stage_ms = total;
  if (stage_launches) *stage_launches = c->ev_used / 2;
  if (kernel_launches) *kernel_launches = c->launches;
  c->profiling = false;
  c->ev_used = 0;
  return JS_OK;
}

int js_ib_info(js_ctx* c, int* n_ghost, unsigned char* tag_host) {
  if (!c || !n_ghost) return JS_ERR_ARG;
  *n_ghost = c->n_ghost;
  if (tag_host) {
    const size_t n = (size_t)c->g.nx * c->g.ny;
    if (c->tag_host.empty()) std::memset(tag_host, 0, n);
    else std::memcpy(tag_host, c->tag_host.data(), n);
  }
  return JS_OK;
}

}  // extern "C"

int js_set_neural(js_ctx* c, const double* w, double* w_bar, const double* norm, int precision) {
  if (!c || (w && c->slab && c->slab_nown < c->g.ny)) return JS_ERR_ARG;
  if (!w) {
    c->nn_on = false;
    return JS_OK;
  }
  const bool layerwise = (precision & JS_NN_LAYERWISE) != 0;
  precision &= ~JS_NN_LAYERWISE;
  if (!norm || (precision != JS_NN_F64 && precision != JS_NN_F32 && precision != JS_NN_BF16)) return JS_ERR_ARG;
  for (int k = 0; k < 4; ++k)
    if (!(norm[4 + k] > 0.0) || !std::isfinite(norm[k]) || !std::isfinite(norm[8 + k])) return JS_ERR_ARG;
  js::NnArgs& n = c->nn;
  const bool two_d = c->g.ny > 1;
  n.lay = c->lay;
  n.nimg = two_d ? 2 : 1;
  n.H[0] = c->g.ny;
  n.W[0] = c->g.nx + 1;
  n.H[1] = two_d ? c->g.nx : 0;
  n.W[1] = two_d ? c->g.ny + 1 : 0;
  n.pix0 = (long long)n.H[0] * n.W[0];
  const long long pix = n.pix0 + (long long)n.H[1] * n.W[1];
  if (!c->nnQ) {
    // buffers sized for FP64 (either precision fits): channels 4, 16, 32, 4, 4, 16, 32
    const int ch[7] = {4, 16, 32, 4, 4, 16, 32};
    for (int k = 0; k < 7; ++k)
      if (cudaMalloc(&c->nn_buf[k], sizeof(double) * ch[k] * (size_t)pix) != cudaSuccess) return JS_ERR_NOMEM;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    n.nwblk = 2 * (sms > 0 ? sms : 1);  // weight-gradient blocks (each keeps a partial sum)
    if (cudaMalloc(&c->nn_partial, sizeof(double) * js::NN_NPARAM * (size_t)n.nwblk) != cudaSuccess ||
        cudaMalloc(&c->nnQ, sizeof(double) * 4 * (size_t)c->lay.plane) != cudaSuccess)
      return JS_ERR_NOMEM;
    JS_CUDA(cudaMemsetAsync(c->nnQ, 0, sizeof(double) * 4 * (size_t)c->lay.plane, c->stream));
  }
  n.X = c->nn_buf[0];
  n.A1 = c->nn_buf[1];
  n.A2 = c->nn_buf[2];
  n.T3 = c->nn_buf[3];
  n.G4 = c->nn_buf[4];
  n.G16 = c->nn_buf[5];
  n.G32 = c->nn_buf[6];
  n.partial = c->nn_partial;
  if (precision == JS_NN_BF16 && !c->nn_bf16[0]) {
    if (cudaMalloc(&c->nn_bf16[0], 2 * 16 * (size_t)pix) != cudaSuccess ||
        cudaMalloc(&c->nn_bf16[1], 2 * 32 * (size_t)pix) != cudaSuccess)
      return JS_ERR_NOMEM;
  }
  n.A1h = c->nn_bf16[0];
  n.A2h = c->nn_bf16[1];
  n.fp32 = (precision != JS_NN_F64) ? 1 : 0;
  n.bf16 = (precision == JS_NN_BF16) ? 1 : 0;
  n.fused = layerwise ? 0 : 1;
  n.keep = 0;
  n.fwd_ready = 0;
  n.err = c->err;
  n.w = w;
  n.w_bar = w_bar;
  for (int k = 0; k < 4; ++k) {
    n.mean[k] = norm[k];
    n.inv_sd[k] = 1.0 / norm[4 + k];
    n.scale[k] = norm[8 + k];
  }
  n.g1 = 1.0 / (c->p.gamma - 1.0);
  // 2D: the stage kernel stores the WENO5 internals the face images are formed from
  if (two_d && !c->nn_wsave) {
    if (cudaMalloc(&c->nn_wsave, internals_bytes(c)) != cudaSuccess) {
      c->nn_wsave = nullptr;
      return JS_ERR_NOMEM;
    }
    JS_CUDA(cudaMemsetAsync(c->nn_wsave, 0, internals_bytes(c), c->stream));
  }
  JS_CUDA(cudaStreamSynchronize(c->stream));
  c->nn_on = true;
  return JS_OK;
}

int js_nn_eval(js_ctx* c, const double* X, int H, int W, double* Y) {
  if (!c || !c->nn_on || !X || !Y || H < 1 || W < 1) return JS_ERR_ARG;
  const long long cap = c->nn.pix0 + (long long)c->nn.H[1] * c->nn.W[1];
  if ((long long)H * W > cap) return JS_ERR_ARG;
  JS_CUDA(js::nn_eval(c->nn, X, H, W, Y, c->stream));
  return JS_OK;
}

int js_nn_eval_vjp(js_ctx* c, const double* X, int H, int W, const double* GY, double* GX) {
  if (!c || !c->nn_on || !X || !GY || !GX || H < 1 || W < 1) return JS_ERR_ARG;
  const long long cap = c->nn.pix0 + (long long)c->nn.H[1] * c->nn.W[1];
  if ((long long)H * W > cap) return JS_ERR_ARG;
  JS_CUDA(js::nn_eval_vjp(c->nn, X, H, W, GY, GX, c->stream));
  return JS_OK;
}

// reverse-pass description of a context for the batched reverse kernel (js_batch.cu): reserves
// the reverse workspace and uploads the inflow states (synchronises when they changed)
int js_internal_rev_desc(js_ctx* c, js::InstRev* d) {
  std::memset(d, 0, sizeof(*d));
  int rc = adj_reserve(c);
  if (rc) return rc;
  if (!c->wsave_fwd) return JS_ERR_NOMEM;
  if ((rc = upload_inflow(c))) return rc;
  d->a = adj_args(c, nullptr, nullptr, nullptr);
  d->ibt = ibt_args(c);
  d->P0 = c->P0;
  d->P1 = c->P1;
  d->Uacc = c->Uacc;
  d->wsave_own = c->wsave;
  d->wfwd = c->wsave_fwd;
  d->inflow_part = c->inflow_part;
  d->inflow_prim = c->inflow_prim;
  d->qIb = c->qIb;
  d->ppart = c->ppart;
  d->tmax = std::max(c->g.nx + 6, c->g.ny);
  return JS_OK;
}
