/*
 * hevi.h -- C ABI of the GB300 (sm_103a) HEVI vertical column solver.
 *
 * The library solves, independently in every vertical atmospheric column,
 * the vertically implicit stage problem of a horizontally explicit,
 * vertically implicit (HEVI) IMEX Runge-Kutta integrator (Giraldo, Alves,
 * Kelly, Kang & Reinecke, arXiv:2311.11425):
 *
 *   linear form (LHEVI, Sec. 4.3, Eq. lhevi-ark-final-2):
 *       (I - Lambda L(q0)) x = b,   Lambda = gamma * dt,
 *   Newton form (NHEVI-LU, Sec. 4.2.3, Eqs. nl_function, Newton-system):
 *       F(q) = q - Lambda V(q) - R = 0,   J(q_m) dq = -F(q_m),
 *
 * where V is the vertical operator of set 2C (App. A.1-A.2) restricted to a
 * flat column and discretised with continuous-Galerkin spectral elements on
 * Legendre-Gauss-Lobatto points (Sec. 3), and L = dV/dq (Sec. 4.3.1, App.
 * A.3).  Band half-widths are k_l = k_u = 3 (N + 1) - 1 (Sec. 4.2.3).
 *
 * State layout (caller-owned device buffers, FP64): columns are packed one
 * after another (column c starts at offset hevi_column_offset(c)); within a
 * column the unknowns are point-major and variable-fastest,
 *   [point I = 0 .. n_z-1][v = rho, m = rho*w, Theta = rho*theta],
 * n_z = Nez * N + 1.  Heights are measured from z = 0 to the column's top.
 * w = 0 is imposed at the bottom and top point (the m-rows there are
 * identity rows; V_m and (L x)_m are reported as 0 there).
 *
 * Every call is asynchronous on the context's CUDA stream unless stated
 * otherwise.  Pointers marked (dev) are device pointers; (host) are host
 * pointers.  No call allocates or frees caller memory.  Errors are returned
 * as hevi_status values; nothing aborts or traps on the device.  Per-column
 * failures (singular pivot, no convergence) are recorded in the context and
 * read back with hevi_column_status.
 */
#ifndef HEVI_H
#define HEVI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HEVI_OK = 0,
  HEVI_ERR_INVALID_ARG = 1,  /* bad argument (null pointer, size, order) */
  HEVI_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  HEVI_ERR_OOM = 3,          /* device allocation failed in setup */
  HEVI_ERR_SINGULAR = 4,     /* some column met an exactly zero pivot */
  HEVI_ERR_NOT_CONVERGED = 5, /* some column's refinement or Newton hit its limit */
  HEVI_ERR_BAD_INPUT = 6,     /* some column's state is non-physical (rho or Theta <= 0, NaN) */
  HEVI_ERR_WAIT_TIMEOUT = 7   /* a device-side wait for an asynchronous copy exceeded its limit */
} hevi_status;

/* One column size class: Nez elements of LGL order N (1 <= N <= 5). */
typedef struct {
  int32_t nez;
  int32_t order;
} hevi_size_class;

/* The set of columns.  class_of_col (host, ncols entries, values in
 * [0, nclasses)) may be NULL when nclasses == 1.  z_top (host, ncols
 * entries, metres) gives each column's model top. */
typedef struct {
  int64_t ncols;
  const hevi_size_class* classes;
  int32_t nclasses;
  const int32_t* class_of_col;
  const double* z_top;
} hevi_column_grid;

/* Isothermal hydrostatic reference state and constants: T0 (K), p0 (Pa),
 * R and cp (J kg^-1 K^-1), g (m s^-2).  NULL in hevi_setup selects
 * 300, 1e5, 287.17, 1004.67, 9.80616. */
typedef struct {
  double T0, p0, R, cp, g;
} hevi_ref_params;

/* Precision of the band factorisation:
 *   HEVI_FP64     plain FP64 band LU with partial pivoting (LAPACK dgbtrf
 *                 semantics, Sec. 4.2.3), one column per thread;
 *   HEVI_FP32_IR  the band is equilibrated with the reference-state scales
 *                 (rho_bar, rho_bar c_s, Theta_bar), rounded to FP32 and
 *                 LU-factored WITHOUT interchanges (L and U each keep the K
 *                 band diagonals; an exactly zero pivot marks the column
 *                 SINGULAR); solves are refined with residuals carried to
 *                 about 48 significant bits (double-float arithmetic), so the
 *                 result is the solution of the FP64 system to the
 *                 refinement tolerance. */
typedef enum { HEVI_FP64 = 0, HEVI_FP32_IR = 1 } hevi_precision;

typedef struct hevi_ctx hevi_ctx;

/* Per-column status codes written by hevi_column_status. */
#define HEVI_COL_OK 0
#define HEVI_COL_SINGULAR 4
#define HEVI_COL_NOT_CONVERGED 5
#define HEVI_COL_BAD_INPUT 6
/* A device-side wait for an asynchronous copy of the column's factor records
 * exceeded its limit (about a second); the column's output is NaN. */
#define HEVI_COL_WAIT_TIMEOUT 7

/* Create a context: builds the LGL tables of each size class (Sec. 3) and
 * the reference state of every column on the device, and allocates the
 * factor, pivot, status and workspace buffers.  stream is a cudaStream_t
 * (NULL = legacy default stream).  Synchronous.  Returns OOM if the device
 * buffers do not fit. */
hevi_status hevi_setup(hevi_ctx** out, const hevi_column_grid* grid,
                       const hevi_ref_params* ref, hevi_precision precision,
                       void* stream);

/* Release every device buffer of the context.  Synchronous. */
void hevi_destroy(hevi_ctx* ctx);

/* Change the stream later calls launch on (cudaStream_t). */
hevi_status hevi_set_stream(hevi_ctx* ctx, void* stream);

/* Total number of FP64 entries of one state vector (sum of 3 n_z). */
int64_t hevi_state_size(const hevi_ctx* ctx);
/* Offset (in doubles) of column c within a state vector; -1 if out of range. */
int64_t hevi_column_offset(const hevi_ctx* ctx, int64_t c);
/* Device bytes held by the context. */
int64_t hevi_device_bytes(const hevi_ctx* ctx);

/* Write the rest state q_bar = (rho_bar, 0, Theta_bar) of every column
 * (dev, state layout).  Reference state: isothermal, hydrostatic. */
hevi_status hevi_reference_state(hevi_ctx* ctx, double* q_bar);

/* As hevi_reference_state for the columns [first, first + count) only; the
 * rest of q_bar is not touched.  INVALID_ARG if the range leaves the
 * context. */
hevi_status hevi_reference_columns(hevi_ctx* ctx, int64_t first, int64_t count, double* q_bar);

/* New model tops for the columns [first, first + count): z_top (host, count
 * values, each > 0 and finite; it may be released when the call returns).
 * Recomputes those columns' element height and reference state on the
 * context's stream, in order with the calls around it; other columns and the
 * size classes are unchanged.  The factors of the last hevi_factor become
 * stale (the next stage solve needs a new hevi_factor; the step calls factor
 * anyway).  With it a long-lived context serves as a pool of column slots
 * that are reused for new columns of the same size class, with no device
 * allocation.  INVALID_ARG on a bad range or top. */
hevi_status hevi_set_column_tops(hevi_ctx* ctx, int64_t first, int64_t count,
                                 const double* z_top);

/* Assemble A = I - Lambda L(q0) = I + Lambda Dcal K(q0) + Lambda G in band
 * form (Sec. 4.2.3; App. A.3 with the gravity entry coupling the m-row to
 * the rho-column) and LU-factor it with partial pivoting, for every column.
 * lin_state (dev, state layout) is q0; NULL linearises about the rest state
 * (LHEVI-RS, Sec. 4.3.1).  Lambda = gamma_dt.  The factors, pivots and the
 * point coefficients of L(q0) stay in the context for later solves.  A column
 * with an exactly zero pivot is marked SINGULAR. */
hevi_status hevi_factor(hevi_ctx* ctx, double gamma_dt, const double* lin_state);

/* Solve (I - Lambda L(q0)) x = rhs for every column with the factors of the
 * last hevi_factor (Sec. 4.3, Eq. lhevi-ark-final-2).  rhs, x (dev, state
 * layout, may not alias).  In HEVI_FP32_IR mode the FP32 solution is refined
 * with residuals b - A x carried to about 48 significant bits (double-float
 * arithmetic) until the predicted relative error (2-norm,
 * |d_k|^2 / |d_(k-1)| / |x|) is below 1e-11, at most 10 sweeps
 * (hevi_set_refinement).  A device-side wait that exceeds its limit marks
 * the column WAIT_TIMEOUT (its x is NaN) and returns HEVI_ERR_WAIT_TIMEOUT.
 * Blocking: returns SINGULAR / NOT_CONVERGED if any column failed. */
hevi_status hevi_stage_solve(hevi_ctx* ctx, const double* rhs, double* x);
/* As hevi_stage_solve but does not wait: failures are only recorded for
 * hevi_column_status. */
hevi_status hevi_stage_solve_async(hevi_ctx* ctx, const double* rhs, double* x);

/* Refinement controls for HEVI_FP32_IR solves: tolerance on the predicted
 * relative error and the sweep limit (defaults 1e-11 and 10). */
hevi_status hevi_set_refinement(hevi_ctx* ctx, double tol, int32_t max_sweeps);

/* Equation set of the context's unknowns (App. A.1):
 *   HEVI_SET_2C (default): (rho, m = rho w, Theta = rho theta), pressure from
 *     the equation of state of set 2C;
 *   HEVI_SET_3C: (rho, m, E) with E the total energy (internal, kinetic,
 *     potential: E = rho (c_v T + w^2/2 + g z)), P = (gamma - 1)(E - m^2/(2 rho)
 *     - rho g z) (Eq. set3c), in a column without horizontal momentum (an
 *     invariant subspace of the vertical operator); the flux Jacobian is that
 *     of Eq. set3c_jacobian restricted to it.  Both precisions; the FP64 band
 *     of set 3C is factored equilibrated with (rho_bar, rho_bar c_s, E_bar),
 *     as the FP32 band always is.  The NHEVI-GMRES solve refuses a set-3C
 *     context.
 *   HEVI_SET_2NC: (rho, w, theta), the advective set of Sec. 2.1 (Eq. set2nc)
 *     in the same column: V_rho = -Dcal[rho w], V_w = -(w Dcal w + (Dcal[P -
 *     P_bar] + g (rho - rho_bar)) / rho), V_theta = -w Dcal theta; its Jacobian
 *     is the Frechet derivative of that V, with terms local to each point
 *     (w' Dcal w0, w' Dcal theta0, the 1/rho0 factor), factored equilibrated
 *     with (rho_bar, c_s, theta_bar).  HEVI_FP64 contexts only (an
 *     HEVI_FP32_IR context returns HEVI_ERR_INVALID_ARG); the first selection
 *     allocates 6 doubles per point of coefficient scratch
 *     (HEVI_ERR_OOM if that fails).  The NHEVI-GMRES solve refuses a
 *     set-2NC context too.
 * Recomputes the reference table (E_bar = P_bar / (gamma - 1) + rho_bar g z for
 * set 3C, theta_bar for set 2NC; hevi_reference_state then writes (rho_bar, 0,
 * E_bar) or (rho_bar, 0, theta_bar)) on the context's stream; the factors of
 * the last hevi_factor become stale.  Call it before the states of the new set
 * are used. */
#define HEVI_SET_2C 0
#define HEVI_SET_3C 1
#define HEVI_SET_2NC 2
hevi_status hevi_set_equation_set(hevi_ctx* ctx, int32_t set);

/* How hevi_nhevi_step ends its Newton sequences.  on = 1 (default): after
 * each iteration the host reads the device's count of still-iterating
 * columns (a stream synchronisation) and enqueues no more iterations once it
 * is zero.  on = 0: every sequence enqueues max_iter iterations without
 * waiting, each gated on the device by that count (the kernels of an
 * iteration after convergence return at once), so that a step call never
 * blocks the calling thread.  Results are the same either way. */
hevi_status hevi_set_newton_host_check(hevi_ctx* ctx, int32_t on);

/* How hevi_lhevi_step sequences an HEVI_FP32_IR step (Sec. 4.3, Eq.
 * lhevi-ark-final-3).  on = 1 (default): each stage's combinations (the stage
 * value Q_i from the solve's result, the next stage's right-hand side, and
 * q^{n+1} after the last stage) are formed inside the tendency pass of that
 * stage, so a step launches no combination kernel (equation set 2C; a
 * set-3C context and an HEVI_FP64 context always use separate combination
 * launches).  on = 0: separate combination launches.  Both evaluate the same
 * FMA chains in the same order and give the same bits.  HEVI_ERR_INVALID_ARG
 * for on outside {0, 1}. */
hevi_status hevi_set_fused_stages(hevi_ctx* ctx, int32_t on);

/* Resident warps per SM of the HEVI_FP32_IR stage solve (1 .. 32; 0 restores
 * the default).  The solve is ONE persistent launch over the tiles of every
 * polynomial order of the context: each warp takes the next tile of 32
 * columns from a device counter, the costliest tiles (longest records) first,
 * so that short tiles fill the end of the launch.  A launch takes about
 * ceil(tiles / warps) rounds; by default the library takes the fewest rounds
 * its occupancy (18 warps per SM) allows and then the fewest warps per SM
 * that keep that many.  The setting changes the speed, not the result.  Not a
 * paper quantity: a launch-shape control of this implementation. */
hevi_status hevi_set_solve_warps(hevi_ctx* ctx, int32_t warps_per_sm);

/* Launch-shape autotuner of the HEVI_FP32_IR stage solve (not a paper
 * quantity).  After hevi_factor, solves A x = rhs (rhs, x: device, state
 * layout, distinct) `reps` times (1 .. 1000) at the default launch shape and at
 * every count of resident warps per SM from 1 to the kernel's occupancy
 * limit, each after one untimed solve, timed with CUDA events on the
 * context's stream; keeps the fastest count (a larger count must win by more
 * than 1%) as if set by hevi_set_solve_warps.  Writes the choice to
 * *warps_per_sm, the mean time of one solve at it to *ms and at the default
 * shape to *ms_default (ms; any of the three may be null).  x holds the
 * solution afterwards.  HEVI_ERR_INVALID_ARG for an FP64 context (its launch
 * shape is fixed), without factors, with bad arguments or while the stream is
 * being captured; HEVI_ERR_CUDA on a CUDA error.  Synchronises the stream. */
hevi_status hevi_autotune_solve(hevi_ctx* ctx, const double* rhs, double* x, int32_t reps,
                                int32_t* warps_per_sm, double* ms, double* ms_default);

/* Test hook for the bounded device waits: with step >= 0 every later
 * HEVI_FP32_IR stage solve announces, but does not issue, the asynchronous
 * copy of the chunk of factor records that holds forward pivot step `step`
 * in each tile's first sweep, so that the wait for it runs out (about a
 * second) and the tile's columns end HEVI_COL_WAIT_TIMEOUT; step < 0 turns it
 * off.  No copy is left in flight and the context stays usable. */
hevi_status hevi_test_drop_record_copy(hevi_ctx* ctx, int32_t step);

/* NHEVI-LU (Sec. 4.2.3): for every column, Newton-Raphson on
 * F(q) = q - gamma_dt V(q) - R, rebuilding and LU-factoring the Jacobian at
 * every iteration; state (dev) holds the initial guess on entry and the
 * root on exit; R (dev).  Stops when ||S^-1 F(q_m)||_2 <= rtol ||S^-1 F(q_0)||_2
 * (S = reference scales rho_bar, rho_bar c_s, Theta_bar) or after max_iter
 * updates.  Blocking. */
hevi_status hevi_newton_solve(hevi_ctx* ctx, double gamma_dt, double* state, const double* R,
                              double rtol, int32_t max_iter);
hevi_status hevi_newton_solve_async(hevi_ctx* ctx, double gamma_dt, double* state,
                                    const double* R, double rtol, int32_t max_iter);

/* Newton solve for callers that cannot allocate device memory.
 *
 * Code that runs inside another framework's memory pool, holds an allocator
 * lock, or lives in a plugin that must not touch the device heap cannot call
 * cudaMalloc, and hevi_setup allocates.  This entry point needs no context
 * and allocates nothing: it runs a fused NHEVI-LU Newton kernel (one column
 * per thread; the Jacobian assembled from FP64 point coefficients, factored
 * in FP32 with partial pivoting, stop test |S^-1 F(q_m)| <= rtol
 * |S^-1 F(q_0)| or the FP64 rounding floor) on ncols uniform columns (nez
 * elements of order `order`, model top z_top in metres, default reference
 * constants) with every piece of scratch -- column table, reference state,
 * linearisation coefficients and factor rows -- in one file-scope device
 * array of 64 MiB that every GPU which loads this library holds until the
 * process exits.  Its result agrees with hevi_newton_solve's to the Newton
 * tolerance.  The paper has no counterpart; it is a deployment variant of
 * NHEVI-LU.
 *
 * state (dev, in/out) and R (dev) use the state layout with columns packed
 * back to back (column c at offset 3 (nez order + 1) c); status and iters
 * (dev, ncols int32 each) receive the per-column status (HEVI_COL_*) and the
 * number of Newton updates.  stream is a cudaStream_t (NULL = legacy default
 * stream).  The call is blocking and returns the aggregated status.
 *
 * Limit: the scratch per column is about 3 n doubles plus n (2K+1) floats
 * (n = 3 (nez order + 1), K = 3 (order + 1) - 1), e.g. about 4,000 columns
 * of (16, 3) or (10, 4); larger ncols returns HEVI_ERR_INVALID_ARG before
 * any device work, and so does a column so long that the kernel's shared
 * memory (per one-warp block) exceeds the device's per-block limit.
 *
 * The first call on a device looks up the array's device address and copies
 * the LGL tables to the device (under a process-wide lock); make that first
 * call before any stream capture.  All calls share the array and it keeps
 * the last call's contents: calls that overlap on the GPU (other streams,
 * other threads) race.  The failure counters in it are cleared by every
 * call. */
hevi_status hevi_newton_solve_noalloc(int32_t nez, int32_t order, double z_top, int64_t ncols,
                                      double gamma_dt, double* state, const double* R,
                                      double rtol, int32_t max_iter, int32_t* status,
                                      int32_t* iters, void* stream);

/* NHEVI-GMRES (Sec. 4.2.1): the stage problem F(q) = q - gamma_dt V(q) - R = 0
 * per column by Jacobian-free Newton-Krylov: Newton updates, each solving
 * J dq = -F by unpreconditioned GMRES (started at zero, not restarted) on the
 * equilibrated system S^-1 J S y = -S^-1 F, dq = S y, with the Frechet
 * difference (Eq. Frechet-derivative) J^ v ~ S^-1 [F(q + eps S v) - F(q)] /
 * eps, i.e. the diagonal perturbation eps S of the reference scales S =
 * (rho_bar, rho_bar c_s, Theta_bar) (the paper's configuration: eps = 0.05,
 * Newton tolerance rtol = 1e-5, GMRES tolerance gtol = 1e-9).  GMRES stops
 * when its residual estimate is <= gtol |S^-1 F| or after kmax iterations
 * (kmax = 0: the context's longest column length n, after which GMRES is
 * exact).  Newton stops as hevi_newton_solve.  state (dev, in/out) holds the
 * initial guess; R (dev) as hevi_newton_solve; krylov (dev, ncols int32, may
 * be NULL) receives the Krylov iterations per column, hevi_column_status the
 * Newton updates.  FP64 throughout; scratch of about 8 (kmax + 1) (n + kmax /
 * 2) bytes per column is allocated on first use.  Status as
 * hevi_newton_solve; the _async form only records per-column status. */
hevi_status hevi_newton_gmres_solve(hevi_ctx* ctx, double gamma_dt, double* state, const double* R,
                                    double eps, double rtol, double gtol, int32_t max_newton,
                                    int32_t kmax, int32_t* krylov);
hevi_status hevi_newton_gmres_solve_async(hevi_ctx* ctx, double gamma_dt, double* state,
                                          const double* R, double eps, double rtol, double gtol,
                                          int32_t max_newton, int32_t kmax, int32_t* krylov);

/* Vertical operator apply (App. A.2 / Sec. 4.3.1), x, y (dev, state layout):
 *   nonlinear != 0:  y = V(x);
 *   nonlinear == 0:  y = L(q0) x with q0 of the last hevi_factor. */
hevi_status hevi_apply_Lv(hevi_ctx* ctx, const double* x, double* y, int nonlinear);

/* Copy the per-column status (HEVI_COL_*) and iteration count (refinement
 * sweeps of the last solve, or Newton updates of the last Newton solve) of
 * the last call into status and iters (dev, ncols int32 each; either may be
 * NULL). */
hevi_status hevi_column_status(hevi_ctx* ctx, int32_t* status, int32_t* iters);

/* One IMEX ARK time step with the HEVI split (Sec. 4.1), ESDIRK tableau of
 * s stages given row-major on the host: A (explicit, s x s), At (implicit,
 * s x s, At[0][0] = 0, constant diagonal gamma), b (weights, shared).
 * q_in, H, q_out (dev, state layout); H is the explicit (horizontal) tendency,
 * held constant over the step; q_out may not alias q_in.
 *   hevi_lhevi_step: LHEVI (Sec. 4.3), one stage solve per implicit stage;
 *     lin_about_rest selects the Jacobian: 0 = refactor with L linearised
 *     about q_in (LHEVI-PS), 1 = refactor about the rest state (LHEVI-RS),
 *     2 = keep the current factorisation and its L (a Jacobian update interval
 *     of more than one step, Sec. 4.3 and the update time-step of Sec. 7.1;
 *     INVALID_ARG unless the context holds factors of the same gamma * dt).
 *   hevi_nhevi_step: NHEVI-LU (Sec. 4.2): one Newton solve per implicit stage
 *     from the previous stage value.
 * Asynchronous; per-column failures are recorded for hevi_column_status. */
hevi_status hevi_lhevi_step(hevi_ctx* ctx, int32_t s, const double* A, const double* At,
                            const double* b, double dt, const double* q_in, const double* H,
                            double* q_out, int32_t lin_about_rest);
hevi_status hevi_nhevi_step(hevi_ctx* ctx, int32_t s, const double* A, const double* At,
                            const double* b, double dt, const double* q_in, const double* H,
                            double* q_out, double rtol, int32_t max_iter);

/* A time loop of nsteps LHEVI or NHEVI-LU steps captured once into a CUDA
 * graph and replayed with one launch (the stage loop of Sec. 4.2/4.3 with the
 * same kernels and arithmetic as hevi_lhevi_step / hevi_nhevi_step, so a
 * replay gives bit-identical results to the same steps called one by one).
 * The steps ping-pong between two caller buffers: step k reads q_a and writes
 * q_b for even k, the reverse for odd k, so after a replay the state is in
 * q_b when nsteps is odd and in q_a when it is even.  H is read at every
 * replay (its contents may change between replays, its address may not);
 * the tableau arrays are copied at creation.  Capture runs on a private
 * stream, so ctx's stream may be any stream including the legacy default;
 * the workspace the steps need is allocated before capture.  Replays run on
 * ctx's stream at the time of hevi_graph_launch.  The context must outlive
 * the graph; hevi_graph_destroy frees it (NULL is a no-op).
 * INVALID_ARG for bad arguments (as the step calls, nsteps < 1, q_a == q_b);
 * CUDA if capture or instantiation fails. */
typedef struct hevi_graph hevi_graph;
hevi_status hevi_lhevi_graph_create(hevi_ctx* ctx, int32_t s, const double* A, const double* At,
                                    const double* b, double dt, double* q_a, double* q_b,
                                    const double* H, int32_t nsteps, int32_t lin_about_rest,
                                    hevi_graph** out);
hevi_status hevi_nhevi_graph_create(hevi_ctx* ctx, int32_t s, const double* A, const double* At,
                                    const double* b, double dt, double* q_a, double* q_b,
                                    const double* H, int32_t nsteps, double rtol,
                                    int32_t max_iter, hevi_graph** out);
hevi_status hevi_graph_launch(hevi_graph* g);
void hevi_graph_destroy(hevi_graph* g);

/* Device bytes that hevi_setup(grid, precision) allocates, plus the
 * workspace of the first step call of one kind: kind 0 = setup only, 1 = an
 * LHEVI step (hevi_lhevi_step / hevi_lhevi_graph_create) with `stages`
 * stages, 2 = an NHEVI-LU step (hevi_nhevi_step / hevi_nhevi_graph_create,
 * Newton scratch included).  Equal to hevi_device_bytes() after those calls.
 * Host arithmetic only (no device call, z_top not read); -1 for invalid
 * arguments (as hevi_setup, or kind outside 0..2, stages outside 2..8). */
int64_t hevi_estimate_bytes(const hevi_column_grid* grid, hevi_precision precision, int32_t kind,
                            int32_t stages);

/* Named ESDIRK tableaux of Sec. 6 (the paper names them; the coefficients
 * come from the cited constructions): "ARK2" = ARK(2,3,2)b with a32 = 1/2,
 * "ARK3" = ARK3(2)4L[2]SA and "ARK4" = ARK4(3)6L[2]SA of Kennedy & Carpenter,
 * "ARS3" = ARK(3,4,3) of Ascher, Ruuth & Spiteri.
 * Writes the stage count to *s and the row-major A, At (s x s) and b (s) to
 * host arrays of at least 64, 64 and 8 doubles.  INVALID_ARG for an unknown
 * name. */
hevi_status hevi_tableau(const char* name, int32_t* s, double* A, double* At, double* b);

/* Wait for the context's stream and return the aggregated status of the
 * calls since the last wait (SINGULAR / NOT_CONVERGED if any column failed). */
hevi_status hevi_sync(hevi_ctx* ctx);

/* Per-kernel timing with CUDA events recorded around each launch on the
 * context's stream (not while the stream is being captured into a graph).
 * hevi_profile(ctx, 1) clears the totals and starts timing, 0 stops it.
 * hevi_profile_read waits for the stream and returns the total milliseconds
 * and launch count of one kernel kind; kinds are 0 .. hevi_profile_kinds()-1
 * with names from hevi_profile_kind_name ("setup", "factor", "stage_solve",
 * "apply", "apply_stage", "newton", "combine"). */
hevi_status hevi_profile(hevi_ctx* ctx, int32_t enable);
int32_t hevi_profile_kinds(void);
const char* hevi_profile_kind_name(int32_t kind);
hevi_status hevi_profile_read(hevi_ctx* ctx, int32_t kind, double* total_ms, int64_t* launches);

/* Number of kernel launches issued by the context so far. */
int64_t hevi_launch_count(const hevi_ctx* ctx);

/* Human-readable name of a status code. */
const char* hevi_status_string(hevi_status s);

#ifdef __cplusplus
}
#endif
#endif /* HEVI_H */
