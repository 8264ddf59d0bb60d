/*
 * jaxshock.h -- C ABI of libjaxshock.so, a GB300 (sm_103a) FP64 implementation of the
 * explicit finite-volume right-hand side of the 2D compressible Euler / Navier-Stokes
 * equations of JAX-Shock (arXiv 2601.04400, Sec. 2) and its SSP-RK3 time step.
 *
 * Conventions (all entry points):
 *   - State arrays are FP64, conserved variables stacked as [4][ny][nx], x fastest:
 *     rho, rho*u, rho*v, E (Sec. 2, Eq. 1).  Device pointers unless a name says "host".
 *     The caller owns every array it passes; the library owns its own workspace.
 *   - ny == 1 is a one-dimensional problem: no y fluxes are evaluated.
 *   - Work is enqueued on the context's CUDA stream and is asynchronous, except where an
 *     entry point says it synchronises.  Nothing in js_step/js_rhs/js_*_vjp allocates or
 *     synchronises, so a sequence of these calls can be captured into a CUDA graph.
 *   - Return value: JS_OK (0) or a negative JS_ERR_* code.  Device-side failures (a
 *     non-physical state, a barrier that timed out) are recorded in a device flag and
 *     reported by js_sync_status, which synchronises the stream.
 *   - A context is not thread-safe; use one context per host thread / stream.
 */
#ifndef JAXSHOCK_H
#define JAXSHOCK_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  JS_OK = 0,
  JS_ERR_ARG = -1,          /* invalid argument (sizes, null pointers, kinds)            */
  JS_ERR_CUDA = -2,         /* a CUDA runtime call failed                                 */
  JS_ERR_NONPHYSICAL = -3,  /* a fluid cell had rho <= 0, p <= 0 or a NaN                 */
  JS_ERR_TIMEOUT = -4,      /* a bounded device-side wait gave up                         */
  JS_ERR_IB = -5,           /* immersed boundary: an image point has no fluid neighbour   */
  JS_ERR_NOMEM = -6         /* device allocation failed                                   */
};

/* Domain boundary kinds (Sec. 3: inflow, outflow, reflective walls; periodic for tests). */
enum { JS_BC_TRANSMISSIVE = 0, JS_BC_REFLECTIVE = 1, JS_BC_PERIODIC = 2, JS_BC_INFLOW = 3 };

/* Uniform Cartesian grid of nx*ny cells, lower-left corner (x0, y0), spacing (dx, dy). */
typedef struct { int nx, ny; double x0, y0, dx, dy; } js_grid;

/* Boundary kinds of the x-low, x-high, y-low and y-high sides, and for JS_BC_INFLOW the
 * primitive state (rho, u, v, p) held in the three ghost layers of that side. */
typedef struct { int kind[4]; double inflow[4][4]; } js_boundary;

/* gamma: ratio of specific heats (Sec. 2, EOS).  mu, Pr: constant dynamic viscosity and
 * Prandtl number of the Navier-Stokes terms (mu = 0: Euler).  nu: coefficient of the
 * Laplacian artificial viscosity nu*lap(U) of the update equation in Sec. 2.  wall: the
 * immersed wall condition, 0 = slip (the paper), 1 = no-slip. */
typedef struct { double gamma, mu, Pr, nu; int wall; } js_params;

/* Parameter-gradient layout used by the vjp entry points (20 doubles):
 * [0] gamma, [1] mu, [2] Pr, [3] nu, [4 + 4*side + k] inflow state k (rho,u,v,p) of side. */
#define JS_NPARAM 20

typedef struct js_ctx js_ctx;

/* Create a solver context (Sec. 2 problem statement).
 *   grid, params, bc : problem description (copied).
 *   sdf_host         : optional host array [ny][nx] of signed distances to the immersed
 *                      solid (< 0 inside; Sec. 2, Fig. 1(c)); NULL = no immersed body.
 *                      Ghost cells, image points and interpolation weights are
 *                      precomputed here.
 *   stream           : cudaStream_t to enqueue on (NULL = legacy default stream).
 * Allocates the padded state buffers and IB tables on the current device.
 * Errors: JS_ERR_ARG, JS_ERR_IB (image point outside the domain or without fluid
 * neighbour), JS_ERR_NOMEM, JS_ERR_CUDA. */
int js_create(const js_grid* grid, const js_params* params, const js_boundary* bc,
              const double* sdf_host, void* stream, js_ctx** out);

/* Release a context and its device memory (synchronises its stream). NULL is a no-op. */
void js_destroy(js_ctx* ctx);

/* Replace the physical parameters and boundary states (geometry stays). */
int js_set_params(js_ctx* ctx, const js_params* params, const js_boundary* bc);

/* Change the stream later work is enqueued on. */
int js_set_stream(js_ctx* ctx, void* stream);

/* Primitive (rho, u, v, p) -> conserved state with the context's gamma (Sec. 2, EOS).
 * W, U: device [4][ny][nx]; may alias. */
int js_prim_to_cons(js_ctx* ctx, const double* W, double* U);

/* dUdt = L(U): boundary halos and immersed-boundary ghost states are filled from U, then
 * WENO5 face states of the primitive variables (Sec. 2), HLLC fluxes, viscous fluxes,
 * flux divergence and nu*lap(U).  Solid and ghost cells get dUdt = 0.
 * U, dUdt: device [4][ny][nx], must not alias.  Asynchronous. */
int js_rhs(js_ctx* ctx, const double* U, double* dUdt);

/* Largest stable time step of U: dt = cfl / max over fluid cells of
 * (|u| + a)/dx + (|v| + a)/dy, capped by the explicit viscous limit
 * cfl h^2 rho_min / (2 mu max(4/3, gamma/Pr)), h = min(dx, dy), when mu > 0 (the paper gives
 * no CFL rule; this is the reading both implementations take).  The rates are IEEE-rounded in
 * a fixed operation order, so the result does not depend on the reduction order.
 * U: device [4][ny][nx].  dt_out: host.  Synchronises the stream.
 * JS_ERR_NONPHYSICAL when a fluid cell has rho <= 0, p <= 0 or a value that is not finite
 * (*dt_out is then 0 or not a usable step size). */
int js_max_dt(js_ctx* ctx, const double* U, double cfl, double* dt_out);

/* Advance U in place by n_steps three-stage SSP-RK3 steps of size dt (the solver step
 * S(U, theta) of Sec. 2 applied n_steps times).  U: device [4][ny][nx].  Asynchronous. */
int js_step(js_ctx* ctx, double* U, double dt, int n_steps);

/* Advance U in place by n_steps SSP-RK3 steps, each of the CFL step size of the current state
 * (js_max_dt's rule, computed on the device with the same IEEE operations in the same order, so
 * the steps equal js_max_dt + js_step ones bit for bit).  No host synchronisation: a loop of
 * these calls can be captured into a CUDA graph.
 *   t_dev  : optional device double, the running time; each step adds its dt (t = t + dt)
 *   t_end  : with t_dev and t_end > 0, the end time: a step with t + dt > t_end takes
 *            dt = t_end - t, and steps once t >= t_end leave U unchanged
 *   dt_log : optional device double[n_steps] receiving the step sizes (0 for a step that did
 *            nothing)
 * A non-physical state (rho <= 0, p <= 0 or not finite in a fluid cell) makes its step size 0:
 * the steps leave U unchanged and the device error flag is set (js_sync_status).  Not with
 * the neural flux (JS_ERR_ARG).  U: device [4][ny][nx].  Asynchronous. */
int js_step_cfl(js_ctx* ctx, double* U, double cfl, int n_steps, double* t_dev, double t_end, double* dt_log);

/* Vector-Jacobian product of the RHS (reverse mode of js_rhs, Sec. 2 gradient chain rule):
 *   U_bar  = (dL/dU)^T lam          (overwritten), device [4][ny][nx]
 *   p_bar += (dL/dtheta)^T lam      (accumulated), device double[JS_NPARAM] or NULL
 * lam: device [4][ny][nx].  Asynchronous. */
int js_rhs_vjp(js_ctx* ctx, const double* U, const double* lam, double* U_bar, double* p_bar);

/* Vector-Jacobian product of ONE SSP-RK3 step of size dt taken from U_n:
 *   lam_n  = (dU_{n+1}/dU_n)^T lam_np1     (overwritten), device [4][ny][nx]
 *   p_bar += (dU_{n+1}/dtheta)^T lam_np1   (accumulated), device double[JS_NPARAM] or NULL
 * The three stage states are recomputed from U_n inside the call (on 2D grids the first
 * two forward stages also store their WENO5 internals for the reverse pass, which needs
 * 2 x 56 extra padded planes of workspace; with the neural flux on, their network input and
 * activations are kept too, 2 x 56 face-image channels allocated by the first such call, and
 * recomputed instead when that allocation fails).  lam_n may alias lam_np1.  Asynchronous. */
int js_step_vjp(js_ctx* ctx, const double* U_n, double dt, const double* lam_np1, double* lam_n,
                double* p_bar);

/* Tape for reverse passes over recorded steps (the backward pass of a checkpointed rollout
 * re-runs a segment forward and then reverses it; recording the stage states saves
 * js_step_vjp from recomputing them).
 *   js_tape_reserve(ctx, n)  allocates n slots of three padded stage states (and the adjoint
 *                            workspace); call it before any stream capture.
 *   js_step_taped(ctx, U, dt, slot)  = js_step(ctx, U, dt, 1), keeping the three filled
 *                            stage states of this step in `slot`.
 *   js_step_vjp_taped(ctx, slot, dt, lam_np1, lam_n, p_bar)  = js_step_vjp for the step
 *                            recorded in `slot` (same dt), without recomputing its stages. */
int js_tape_reserve(js_ctx* ctx, int n_slots);

/* js_tape_reserve with options.  JS_TAPE_WENO (2D grids; ignored for ny == 1): every slot
 * also holds the WENO5 internals of its three stages (56 padded planes per stage, about
 * 1.3 KB per cell and slot), written by js_step_taped; js_step_vjp_taped then skips the
 * WENO forward recompute of its reverse pass.  Results are identical with and without.
 * flags = 0 is js_tape_reserve; the choice applies to the js_step_taped calls that follow.
 * Returns JS_ERR_NOMEM (nothing freed) when the device memory does not suffice. */
#define JS_TAPE_WENO 1
int js_tape_reserve_ex(js_ctx* ctx, int n_slots, int flags);
int js_step_taped(js_ctx* ctx, double* U, double dt, int slot);
int js_step_vjp_taped(js_ctx* ctx, int slot, double dt, const double* lam_np1, double* lam_n, double* p_bar);

/* ---- Stage-wise stepping ----------------------------------------------------------------
 * One stage of the SSP-RK3 step (Shu-Osher form; the paper prints forward Euler, Sec. 2):
 *   U_out = a_k U_n + b_k (X + dt L(X)),  (a_k, b_k) = (0, 1), (3/4, 1/4), (1/3, 2/3),
 * X = U_in with its boundary ghost layers and immersed-boundary ghost cells filled.  js_step
 * is stage 0 from U_n, stage 1 from its result, stage 2 from that.  U_n is read only for
 * stage > 0 (may be NULL for stage 0).  All arrays device [4][ny][nx]; any may alias.
 * Asynchronous.  This is the entry for callers that act between stages (the halo exchange of
 * a y-decomposed grid, below).  stage | JS_STAGE_INTERNALS (stages 0 and 1 of a 2D grid; the
 * flag is ignored otherwise) also stores the stage's WENO5 internals in the context (the
 * workspace of js_step_vjp, allocated by the first such call), for a js_step_stage_vjp of the
 * same stage and U_in that passes the flag too. */
#define JS_STAGE_INTERNALS 16
int js_step_stage(js_ctx* ctx, const double* U_n, const double* U_in, double* U_out, double dt, int stage);

/* Reverse of js_step_stage, called for the stages of one step in the order 2, 1, 0 (any other
 * order returns JS_ERR_ARG; js_rhs_vjp / js_step_vjp / js_step_vjp_taped restart the order):
 *   lam_in  = (dU_out/dX)^T lam_out through the ghost fills to U_in   (overwritten)
 *   p_bar  += (dU_out/dtheta)^T lam_out                                (accumulated, or NULL)
 * The U_n part a_k lam_out of stages 2 and 1 is kept in the context and added to the lam_in
 * of stage 0 (whose U_in is U_n): with lam_out of stage k-1 = lam_in of stage k, the stage-0
 * lam_in equals js_step_vjp's lam_n.  lam_in may alias lam_out.  stage | JS_STAGE_INTERNALS
 * uses the internals js_step_stage stored for that stage (stages 0, 1 of a 2D grid; JS_ERR_ARG
 * when it stored none since the last js_step_vjp) instead of recomputing WENO5: same results.
 * Asynchronous. */
int js_step_stage_vjp(js_ctx* ctx, const double* U_in, double dt, int stage, const double* lam_out,
                      double* lam_in, double* p_bar);

/* ---- Single-grid domain decomposition in y slabs -----------------------------------------
 * A grid is split into slabs of whole rows, one context (one rank, one GPU) per slab.  A slab
 * context holds a window of the grid: its own rows [row0, row0 + nrows) and `overlap` rows of
 * each neighbouring slab (clipped at non-periodic y sides; wrapping around when both y sides
 * are periodic).  A stage output reads cells within 3 rows, so when, after every stage, the
 * overlap rows are overwritten with their owners' new values (the halo exchange), the owned
 * rows evolve exactly as in the undecomposed grid and the overlap rows' own stage outputs are
 * never used.  Reverse mode transposes the exchange: after every reversed stage the adjoint
 * of the overlap rows is added to the owner's rows and cleared locally; p_bar is then the sum
 * over the slabs.  The CFL step of the grid is the minimum of the slabs' js_max_dt. */

/* Create the context of one slab.
 *   grid, params, bc, sdf_host : the WHOLE grid, as for js_create (sdf_host [grid->ny][nx]).
 *   row0, nrows                : owned rows; nrows == grid->ny gives a plain context.
 *   overlap                    : rows of each neighbour held (>= 3; with an immersed body,
 *                                also enough that every ghost cell within 3 rows of the owned
 *                                rows has its image-point cells inside the window).
 * The context's arrays are [4][rows][nx] over the window (js_slab_info); y sides that border
 * another slab get transmissive ghost layers.  Immersed-boundary tables are those of the
 * whole grid restricted to the window; a ghost cell whose image-point cells leave the window
 * is frozen (it reaches no owned output), or JS_ERR_IB when it lies within 3 rows of the
 * owned rows.  The neural flux (js_set_neural) is not available on a slab of a decomposed grid.
 * Errors: JS_ERR_ARG (ny == 1, rows out of range, overlap < 3, a window that would wrap onto
 * itself or fewer than 6 rows, only one y side periodic), JS_ERR_IB, JS_ERR_NOMEM, JS_ERR_CUDA. */
int js_create_slab(const js_grid* grid, const js_params* params, const js_boundary* bc, const double* sdf_host,
                   int row0, int nrows, int overlap, void* stream, js_ctx** out);

/* Window of a context: its first row in the whole grid (row_lo; local row k is grid row
 * (row_lo + k) mod grid ny), its number of rows, the local index of its first owned row and
 * the number of owned rows.  A plain context reports 0, ny, 0, ny.  Any output may be NULL. */
int js_slab_info(js_ctx* ctx, int* row_lo, int* rows, int* own_lo, int* own_rows);

/* Row blocks for the halo exchange: rows [row0, row0 + nrows) of the four planes of a
 * context-shaped array U ([4][rows][nx]) to / from a contiguous device buffer [4][nrows][nx].
 *   js_rows_pack   : buf = those rows; zero != 0 also sets them to 0 in U (reverse exchange).
 *   js_rows_unpack : those rows = buf, or += buf when add != 0.
 * JS_ERR_ARG when the rows leave the context's window.  Asynchronous. */
int js_rows_pack(js_ctx* ctx, double* U, int row0, int nrows, double* buf, int zero);
int js_rows_unpack(js_ctx* ctx, double* U, int row0, int nrows, const double* buf, int add);

/* Neural flux (Sec. 2.3).  A fully convolutional network of three 3x3 layers with zero
 * ("SAME") padding, 4 -> 16 -> 32 -> 4 channels, ReLU, ReLU, tanh (JS_NN_NPARAM = 6388
 * parameters, the paper's count), evaluated on one image per direction and added to the HLLC
 * flux of every face; the update then takes the divergence of F_HLLC + F_neural.
 *   image: x faces [4][ny][nx+1], y faces transposed [4][nx][ny+1] (1D: x faces only);
 *   pixel (line, face f) = (m - mean) / sd per frame channel, m = the mean of the two WENO5
 *   face states of face f in conserved variables of the face frame (rho, normal momentum,
 *   tangential momentum, E); both directions share the network;
 *   neural flux of frame component k through the face = scale[k] * output channel k.
 * Parameter layout (doubles): w1[16][4][3][3], b1[16], w2[32][16][3][3], b2[32],
 * w3[4][32][3][3], b3[4].
 *   w      device pointer to the parameters, read at every later stage (so they may be
 *          updated in place between calls); NULL switches the neural flux off
 *   w_bar  device pointer, JS_NN_NPARAM doubles, or NULL: every later js_rhs_vjp /
 *          js_step_vjp / js_step_vjp_taped ADDS the parameter gradient (summed in a fixed
 *          order: reproducible)
 *   norm   host array mean[4], sd[4] (> 0), scale[4] (copied)
 *   precision  JS_NN_F64 (FP64 network arithmetic), JS_NN_F32 (FP32 on the CUDA cores) or
 *          JS_NN_BF16 (the three layers of the forward pass on the tensor cores with BF16
 *          operands and FP32 accumulation; in the reverse the data and weight gradients of
 *          layers 3 and 2 likewise, the first layer's FP32); the solver
 *          stays FP64 (with FP32 and BF16 networks the face images and the network's flux
 *          divergence are formed in FP32 and added to the FP64 state).
 *          In BF16 precision the stages that no reverse pass reads evaluate the whole network
 *          in one launch (activations kept on chip); JS_NN_BF16 | JS_NN_LAYERWISE runs its
 *          three layers as separate launches instead, with bit-identical results
 * Applies to js_rhs, js_step, the taped steps and the reverse calls of this context (not to
 * js_batch_*).  The first call allocates the network workspace (before any stream capture).
 * Returns JS_ERR_ARG for a bad norm or precision, JS_ERR_NOMEM. */
#define JS_NN_NPARAM 6388
#define JS_NN_F64 0
#define JS_NN_F32 1
#define JS_NN_BF16 2
#define JS_NN_LAYERWISE 0x100
int js_set_neural(js_ctx* ctx, const double* w, double* w_bar, const double* norm, int precision);

/* The network of js_set_neural alone (its parameters, normalisation scale and precision) on one
 * normalised image: X [4][H][W] (device, FP64) -> Y [4][H][W] = scale[k] * output channel k
 * (device, FP64).  H * W may not exceed the context's face-image capacity (2 nx ny + nx + ny on 2D
 * grids) or JS_ERR_ARG; JS_ERR_ARG also without the neural flux on.  Asynchronous. */
int js_nn_eval(js_ctx* ctx, const double* X, int H, int W, double* Y);

/* Reverse of js_nn_eval on the same image (the network's forward is recomputed):
 *   GX     = (dY/dX)^T GY          (overwritten), device [4][H][W] FP64
 *   w_bar += (dY/dw)^T GY          (the w_bar of js_set_neural, when one was given)
 * In BF16 precision the data and weight gradients of layers 3 and 2 run on the tensor cores
 * (BF16 operands, FP32 accumulation); the first layer's are FP32.  GX may alias X or GY.
 * Errors as js_nn_eval.  Asynchronous. */
int js_nn_eval_vjp(js_ctx* ctx, const double* X, int H, int W, const double* GY, double* GX);

/* Block average (the downsampling that turns high-resolution states into the coarse
 * training targets of Sec. 2.4): out[4][ny/fy][nx/fx] (device) = the means of the fx x fy
 * cell blocks of U[4][ny][nx] (device).  nx % fx == 0 and ny % fy == 0 or JS_ERR_ARG.
 * Asynchronous on `stream` (a cudaStream_t, NULL = default stream); no context needed. */
int js_block_average(const double* U, int nx, int ny, int fx, int fy, double* out, void* stream);

/* Read and clear the device error flag; synchronises the stream.  Returns JS_OK,
 * JS_ERR_NONPHYSICAL or JS_ERR_TIMEOUT (or JS_ERR_CUDA if the stream itself failed). */
int js_sync_status(js_ctx* ctx);

/* Number of immersed-boundary ghost cells and, if tag_host != NULL, the cell tags
 * (0 fluid, 1 solid, 2 ghost) as host uint8 [ny][nx]. */
int js_ib_info(js_ctx* ctx, int* n_ghost, unsigned char* tag_host);

/* ---- batched path ---------------------------------------------------------------------
 * Many independent 2D problems (uneven grids, parameters, boundaries, immersed bodies)
 * advanced together by ONE persistent cooperative kernel launch per js_batch_step call (the
 * solver step mapped over a batch of problems; the paper's vmap, Sec. 1).  Each instance's
 * dt is recomputed on the device before every step from its own state (CFL rule of
 * js_max_dt, same arithmetic, so a batched run equals per-instance js_max_dt + js_step runs
 * bit for bit).  Grid barriers inside the launch wait at most 2 s each; a wait that runs out
 * sets JS_ERR_TIMEOUT (read by js_batch_sync_status) and the launch returns. */
typedef struct js_batch js_batch;

/* Create a batch of `count` problems: arrays grids[count], params[count], bcs[count];
 * sdf_host: NULL or an array of `count` host pointers (entries may be NULL).  All grids must
 * be 2D.  Allocates per-instance buffers.  Errors as js_create. */
int js_batch_create(int count, const js_grid* grids, const js_params* params, const js_boundary* bcs,
                    const double* const* sdf_host, void* stream, js_batch** out);

/* Register the instances' states: U is a host array of `count` device pointers, each
 * [4][ny_k][nx_k], advanced in place by js_batch_step.  Copies the pointer table to the
 * device and synchronises; call again when the pointers change (not inside a capture). */
int js_batch_set_states(js_batch* b, double* const* U);

/* Advance every instance by n_steps SSP-RK3 steps with its own CFL time step (cfl > 0) in
 * one launch.  t_dev: optional device double[count] to which each instance's elapsed time
 * is added.  dt_log: optional device double[n_steps][count] receiving the step sizes used
 * (the reverse pass needs them).  Asynchronous; allocates nothing, so it can be captured
 * into a CUDA graph. */
int js_batch_step(js_batch* b, double cfl, int n_steps, double* t_dev, double* dt_log);

/* Reverse of one batched step (the gradient chain rule of Sec. 2 per instance) in ONE
 * persistent cooperative launch over all instances: for every instance k,
 * lam_n[k] = (dU_{n+1}/dU_n)^T lam_np1[k] for the step of size dt[k] taken from U_n[k]
 * (the same values as js_step_vjp, bit for bit), and p_bar[k] += (dU_{n+1}/dtheta_k)^T
 * lam_np1[k] (JS_NPARAM doubles each, summed in a fixed order; p_bar or an entry may be NULL).
 * dt: host array of `count` step sizes (e.g. a row of the dt log, which treats each CFL step
 * size as fixed).  U_n, lam_np1, lam_n, p_bar: host arrays of device pointers; lam_n[k] may
 * alias lam_np1[k].  The first call allocates each instance's reverse workspace; every call
 * copies its pointer table to the device and synchronises the stream before returning (use
 * js_batch_rollout_vjp inside a stream capture). */
int js_batch_step_vjp(js_batch* b, double* const* U_n, const double* dt, double* const* lam_np1,
                      double* const* lam_n, double* const* p_bar);

/* Advance every registered state n_steps SSP-RK3 steps of the given sizes dt[step][count]
 * (device) instead of CFL step sizes, e.g. to replay a run logged by js_batch_step.  One launch;
 * asynchronous; allocates nothing. */
int js_batch_step_fixed(js_batch* b, int n_steps, const double* dt);

/* Reverse of a batched rollout of n_steps steps (the chain rule of Sec. 2 through the whole
 * run): the instances start from the registered states (js_batch_set_states; left unchanged)
 * and take the step sizes dt_log[step][count] (device; e.g. logged by js_batch_step, each CFL
 * step size treated as fixed).
 *   lam   : host array of `count` device pointers; in: dL/dU_{n_steps}, out: dL/dU_0
 *   p_bar : host array of device pointers (JS_NPARAM doubles each, accumulated) or NULL
 *   ckpt  : checkpoint spacing (<= 0: js_batch_rollout_spacing's choice): the forward keeps the
 *           state after every ckpt-th step (or those of js_batch_rollout_forward are used, see
 *           there); then, from the last segment back, each segment is re-run keeping its
 *           states and its steps' stage states U1, U2, and reversed step by step by the
 *           persistent reverse launch of js_batch_step_vjp, which takes the stage states as
 *           given instead of recomputing them.  Spacing 1: the forward keeps every state and
 *           stage state, nothing is re-run.
 * Workspace: ceil(n_steps/ckpt) + 3 ckpt + 2 states per instance (3 n_steps + 3 with spacing
 * 1) and the reverse workspace,
 * allocated by the first call for these n_steps and ckpt (synchronises; make it before any
 * stream capture).  Later calls with the same n_steps, ckpt, lam and p_bar pointers enqueue
 * only kernels (one launch per copy, segment re-run and reverse step) and can be captured into
 * a CUDA graph.  Asynchronous otherwise. */
int js_batch_rollout_vjp(js_batch* b, int n_steps, const double* dt_log, int ckpt, double* const* lam,
                         double* const* p_bar);

/* The forward of a checkpointed rollout: advance the registered states n_steps CFL steps
 * (cfl > 0; each instance's step sizes written to dt_log[step][count], device), keeping the
 * state after every ckpt-th step (ckpt <= 0: js_batch_rollout_spacing's choice).  A js_batch_rollout_vjp
 * that follows with the same n_steps, ckpt and dt_log, with no batched step or
 * js_batch_set_states in between, reverses from these checkpoints and skips its own forward
 * pass.  Workspace as js_batch_rollout_vjp's. */
int js_batch_rollout_forward(js_batch* b, double cfl, int n_steps, int ckpt, double* dt_log);

/* The checkpoint spacing the rollout calls use for n_steps when given ckpt <= 0 (*ckpt, host):
 * the spacing of the rollout workspace already prepared for n_steps; otherwise 1 (every state
 * and stage state kept: the reverse re-runs nothing) when that workspace (3 n_steps + 3 states of
 * all instances) fits in half of the device memory free now, else the integer nearest
 * sqrt(n_steps).  Synchronous (queries
 * the free memory); allocates nothing. */
int js_batch_rollout_spacing(js_batch* b, int n_steps, int* ckpt);

/* Read and clear the batch's device error flag (synchronises): JS_OK, JS_ERR_NONPHYSICAL,
 * JS_ERR_TIMEOUT. */
int js_batch_sync_status(js_batch* b);

/* Launch shape and size: resident blocks of the persistent kernel, 32x16 tiles, cells. */
int js_batch_info(js_batch* b, int* blocks, int* tiles, long long* cells);

/* Launch shape and schedule of the forward launch (js_batch_step, js_batch_step_fixed and the
 * rollout's forward runs): blocks_per_sm resident blocks on every SM (0 = the most that fit),
 * and the order in which the blocks take the tiles of all instances: 0 instance by instance,
 * 1 interleaved (tile j of every instance, then tile j + 1), 2 the largest instances first.
 * Results are identical for every choice; only speed differs (the Python autotuner times them
 * and caches the choice per mix of instances).  Schedules 1 and 2 upload a tile table
 * (synchronises: before any stream capture).  js_batch_get_tuning reports the current choice,
 * the most blocks per SM and the number of schedules. */
int js_batch_set_tuning(js_batch* b, int blocks_per_sm, int schedule);
int js_batch_get_tuning(js_batch* b, int* blocks_per_sm, int* max_blocks_per_sm, int* schedule, int* n_schedules);

/* Launch form of the batched reverse step (js_batch_step_vjp and every reverse step of
 * js_batch_rollout_vjp; the gradient chain rule of Sec. 2 applied to each instance):
 *   split = 0 (default): ONE persistent cooperative launch per reverse step, its phases (pack,
 *     forward recompute, then per stage: seed + primitives, pass 1, pass 2, primitive reverse,
 *     transposed halos, inflow gradient and IB ghosts, IB sources; unpack) separated by
 *     bounded grid barriers, every phase at the register allocation of the heaviest one;
 *   split = 1: one ordinary launch per phase (34 per reverse step; 37 when the batch mixes
 *     viscous and inviscid instances), in the same order on the batch's stream, each phase
 *     kernel at its own occupancy.
 * Both run the same device code on the same work items in the same order: lambda and the
 * parameter gradient agree to rounding (separately compiled kernels may contract different
 * products into fused multiply-adds), and each form repeats its own results bit for bit.
 * Both can be captured in a CUDA graph.
 * Synchronises the batch's stream (call before any stream capture).  Errors: JS_ERR_ARG for a
 * split value other than 0 or 1. */
int js_batch_set_reverse_launch(js_batch* b, int split);
int js_batch_get_reverse_launch(js_batch* b, int* split);

/* The context of instance k (owned by the batch; do not destroy it), e.g. for js_step_vjp. */
js_ctx* js_batch_instance(js_batch* b, int k);

/* Failure-detection check of the bounded barrier: launches the persistent kernel with a
 * barrier that can never complete (one arrival short) and a wait budget of budget_s
 * (0 < budget_s <= 2) seconds; the launch must end by itself with JS_ERR_TIMEOUT in the
 * batch's error flag.  Requires js_batch_set_states. */
int js_batch_test_timeout(js_batch* b, double budget_s);

void js_batch_destroy(js_batch* b);

/* Arithmetic mode of the forward path (js_rhs, js_step, and js_step_stage without
 * JS_STAGE_INTERNALS) of this context:
 *   JS_ARITH_FAST (default): the fused stage kernel, which contracts products into fused
 *     multiply-adds and replaces division and square root by a refined reciprocal (within
 *     about 2 ulp) -- each stage agrees with the IEEE-order result to about 1e-15 relative;
 *   JS_ARITH_IEEE: every operation of the right-hand side (Sec. 2: WENO5 of the primitive
 *     variables, HLLC with the positivity fallback, viscous fluxes, divergence, artificial
 *     viscosity), the immersed-boundary ghost fill and the Runge-Kutta stage is one
 *     IEEE-rounded double operation in a fixed canonical expression order (written out in
 *     js_ieee.cu), each face and cell computed on its own: the results are reproducible bit for
 *     bit by any implementation that follows that order, independent of launch shape or
 *     device.  About 3x slower; extra workspace of 4 padded planes plus the face fluxes
 *     (allocated by the first switch to it: call before any stream capture).
 * The reverse-mode entry points, the taped steps and the batched path keep the fast
 * arithmetic.  JS_ARITH_IEEE does not combine with the neural flux (js_rhs / js_step then
 * return JS_ERR_ARG).  Errors: JS_ERR_ARG, JS_ERR_NOMEM. */
#define JS_ARITH_FAST 0
#define JS_ARITH_IEEE 1
int js_set_arith(js_ctx* ctx, int mode);
int js_get_arith(js_ctx* ctx, int* mode);

/* Stage-kernel tuning: tile shape variant (0 .. n_variants-1) used by this context's
 * js_rhs / js_step / js_step_vjp; 0 = 32x32-cell tiles staged by TMA with concurrent x/y sweeps.  Results are identical for every
 * variant; only speed differs (the Python autotuner times them and caches the choice). */
int js_set_tuning(js_ctx* ctx, int variant);
int js_get_tuning(js_ctx* ctx, int* variant, int* n_variants);

/* Instrumentation.  js_profile_begin(ctx, capacity) starts timing every launch of the fused
 * stage kernel (up to `capacity` launches) with CUDA events recorded on the context's stream,
 * and counting every kernel the context launches.  js_profile_end synchronises the stream,
 * stops recording and returns the summed stage-kernel time in ms, the number of stage
 * launches timed and the number of kernels launched in between (any pointer may be NULL). */
int js_profile_begin(js_ctx* ctx, int capacity);
int js_profile_end(js_ctx* ctx, double* stage_ms, int* stage_launches, long long* kernel_launches);

/* Allocation-free CFL time step -- the paper has no counterpart.  It serves callers that
 * cannot allocate device memory, such as a host application or plugin that owns every
 * device allocation through its own pool and forbids libraries to call cudaMalloc.  Same
 * result as js_max_dt, bit for bit (the same IEEE operation order; JS_ERR_NONPHYSICAL for the
 * same states), without a context:
 *   grid, params : the problem (only nx, ny, dx, dy, gamma, mu, Pr are used)
 *   U            : device [4][ny][nx];  tag: optional device uint8 [ny][nx], 0 = fluid
 *                  cell (only fluid cells count), or NULL for all cells
 *   dt_out       : host; the stream is synchronised before returning.
 * The reduction's scratch is one 64 KiB file-scope device array per GPU, kept until the
 * process exits: grids above JS_NOALLOC_MAX_CELLS cells return JS_ERR_ARG.  All calls on a
 * device share the array and it keeps the last call's partial results, so calls whose
 * kernels overlap on the GPU race -- serialise them.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it for the process; make that
 * first call before any stream capture, and do not call it after a cudaDeviceReset of that
 * device (the kept address belongs to the destroyed context).  Calls no allocating routine. */
#define JS_NOALLOC_MAX_CELLS 8388608
int js_max_dt_noalloc(const js_grid* grid, const js_params* params, const double* U,
                      const unsigned char* tag, double cfl, void* stream, double* dt_out);

/* Human-readable text of a JS_* code (static storage). */
const char* js_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* JAXSHOCK_H */
