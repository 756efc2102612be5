/*
 * pdhg.h -- C ABI of the GB300 space-time PDHG solver for implicit schemes of
 * scalar conservation laws (Liu, Osher, Li, Shu, arXiv 2207.07234).
 *
 * The solver finds the saddle point of the discrete Lagrangian of Sec. 3.3
 * (Eq. 3.10) with the preconditioned primal-dual iteration of Algorithm 1:
 * every time slice of the implicit scheme (backward Euler or BDF2 in t,
 * Sec. 3.1; upwind / Lax-Friedrichs finite differences or DG P2 in x,
 * Sec. 3.2) is updated at once on the GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: PDHG_OK (0) or a negative pdhg_status.  Nothing aborts and
 *   no kernel traps; pdhg_last_error() gives a message for the calling thread.
 * - Memory: the library allocates NO device memory.  The caller owns one
 *   device workspace of pdhg_workspace_size() bytes (256-byte aligned) and
 *   passes it to pdhg_create(); the handle (host memory, owned by the
 *   library) only points into it.  The workspace must stay alive and untouched
 *   until pdhg_destroy().
 * - Streams: every device operation is enqueued on the handle's stream (a
 *   cudaStream_t passed as void*; NULL is the legacy default stream).
 * - Layouts (one time slice, "dofs"): 1D finite differences: u[j], j = 0..nx-1,
 *   x_j = j*lx/nx.  2D: u[y][x], x fastest.  DG P2: U[m][j], m = 0..2 Legendre
 *   mode, j = cell, cell fastest.  DG P1 (the nodal basis of Sec. 3.2.2): U[m][j],
 *   m = 0, 1 the values at x_{j-1/4}, x_{j+1/4} of cell j = [j h, (j+1) h].  Space-time fields are slice-major: u has
 *   nt+1 slices (l = 0..nt), phi and phit have nt slices (one per equation).
 * - Precision: fields are stored as double (PDHG_FP64) or float (PDHG_FP32);
 *   buffers passed to pdhg_get_field/pdhg_set_field use that element type.
 *   Residual norms are always accumulated in double.
 * - Determinism: the same inputs on the same GPU give bitwise-identical results.
 */
#ifndef PDHG_H
#define PDHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PDHG_OK = 0,
    PDHG_ERR_INVALID_ARG = -1,          /* a size, step, pointer or enum is invalid */
    PDHG_ERR_WORKSPACE_TOO_SMALL = -2,  /* workspace smaller than pdhg_workspace_size() */
    PDHG_ERR_CUDA = -3,                 /* a CUDA runtime call failed (message has the cudaError) */
    PDHG_ERR_NONFINITE = -4,            /* a residual norm became NaN or Inf */
    PDHG_ERR_DIVERGED = -5,             /* the primal residual grew by more than 1e10 */
    PDHG_ERR_TIMEOUT = -6,              /* a bounded device wait gave up */
    PDHG_ERR_UNSUPPORTED = -7,          /* valid but not implemented (e.g. a 2D nx not a power of two) */
    PDHG_ERR_BOUNDS = -8                /* a debug build (-DPDHG_DEBUG) caught an out-of-range index */
} pdhg_status;

enum { PDHG_TIME_BE = 0, PDHG_TIME_BDF2 = 1 };
enum { PDHG_SPACE_FD_UPWIND = 0, PDHG_SPACE_FD_LF = 1, PDHG_SPACE_DG_P2_LF = 2,
       PDHG_SPACE_DG_P1_UPWIND = 3, PDHG_SPACE_DG_P1_LF = 4 };
enum { PDHG_FP64 = 0, PDHG_FP32 = 1 };
enum { PDHG_INIT_LAMBDA = 0, PDHG_INIT_PINNED = 1 };
enum { PDHG_PATH_AUTO = 0, PDHG_PATH_PLAIN = 1, PDHG_PATH_FUSED = 2 };
enum { PDHG_FIELD_U = 0, PDHG_FIELD_PHI = 1, PDHG_FIELD_PHIT = 2,
       PDHG_FIELD_LAMBDA = 3, PDHG_FIELD_LAMBDAT = 4, PDHG_FIELD_U_TERMINAL = 5 };

/* Stages of one iteration, for pdhg_stage_times(). */
enum { PDHG_STAGE_PRIMAL = 0,      /* primal step + lambda update (Algorithm 1 steps 1, 2b) */
       PDHG_STAGE_RESIDUAL_FFT = 1,/* R(u^n) and its forward x-transform */
       PDHG_STAGE_FFT_Y = 2,       /* 2D: forward and inverse y-transforms */
       PDHG_STAGE_TSOLVE = 3,      /* tridiagonal solve in t per Fourier mode */
       PDHG_STAGE_DUAL = 4,        /* inverse x-transform, dual step and extrapolation */
       PDHG_STAGE_CHECK = 5,       /* residual norms (every check_every iterations) */
       PDHG_STAGE_FUSED_ROWS = 6,  /* fused 2D path: residual + x-FFT, spectrum stored transposed
                                      (its primal step is STAGE_PRIMAL, its dual step STAGE_DUAL) */
       PDHG_STAGE_FUSED_COLS = 7,  /* fused 2D path: y-FFT + t-solve + inverse y-FFT */
       PDHG_NUM_STAGES = 8 };

/*
 * The conservation law u_t + f(u)_x - (gamma u_x)_x = 0 on a periodic domain
 * (Eq. 2.1; 2D: f(u)_x + f(u)_y), the preconditioner and the step sizes.
 *   f(u) = alpha*u^2 + beta*u                   (Sec. 3.2.3; linear: alpha = 0)
 *   nu          constant viscosity: adds -nu * central second difference
 *   gamma_half  host pointer to gamma_{j+1/2}, j = 0..nx-1 (1D FD only) or NULL;
 *               adds -Lap(u) of Sec. 3.2.1.  Copied at create.
 *   u0          host pointer to the initial slice (dof layout above), or a device pointer
 *               with PDHG_FLAG_U0_ON_DEVICE.  Copied at create.
 *   lf_a        global Lax-Friedrichs constant for the LF schemes (0: max |f'(u0)|);
 *               the upwind schemes use f(u-) and are monotone where f' >= 0
 *   c, gamma_hat  K = -d_tt - c^2 d_xx + gamma_hat^2 d_xxxx (Eq. 2.8, 2.10);
 *                 DG uses c only.  c shapes the iteration, never its fixed point; for
 *                 finite differences max |f'(u0)| serves well, while DG P2 Burgers past
 *                 a shock converges far faster with c well below it (0.25 against 1.5).
 *   tau_u, tau_u0, tau_phi, tau_lambda   step sizes of Algorithm 1 (> 0).
 */
typedef struct {
    double alpha, beta;
    double nu;
    const double *gamma_half;
    const double *u0;
    double lf_a;
    double c, gamma_hat;
    double tau_u, tau_u0, tau_phi, tau_lambda;
} pdhg_problem;

/* Uniform space-time grid (Sec. 3.1, 3.2): h_x = lx/nx, h_y = ly/ny, h_t = T/nt.
 * dims = 1 or 2; ny = 1 in 1D; for DG, nx is the number of cells.  nx and ny are
 * powers of two in [4, 8192] (ny <= 2048), 1 <= nt <= 65534; 1D finite differences
 * also take any nx in [4, 4096] (the preconditioner's x-DFT then runs as a
 * Bluestein chirp convolution through power-of-two FFTs).  Others:
 * PDHG_ERR_UNSUPPORTED. */
typedef struct {
    int32_t dims;
    int64_t nx, ny;
    double lx, ly;
    double T;
    int64_t nt;
} pdhg_grid;

/* time: PDHG_TIME_*; space: PDHG_SPACE_*; precision: PDHG_FP64 / PDHG_FP32;
 * init: PDHG_INIT_LAMBDA (Algorithm 1's multiplier on u^0 = u0) or
 * PDHG_INIT_PINNED (u^0 held at u0); path: PDHG_PATH_*; flags: 0 or a combination
 * of PDHG_FLAG_EXACT_TIME_PRECOND, PDHG_FLAG_U0_ON_DEVICE, PDHG_FLAG_T_SOLVE_FP64 and
 * PDHG_FLAG_MIXED_STEPS.
 *
 * PDHG_FLAG_EXACT_TIME_PRECOND (an ablation of the preconditioner of Sec. 3.3): the
 * time part of K_d is the scheme's own h_t^2 D_t D_t^T (D_t the BE or BDF2 time
 * difference with u^0 held fixed) instead of T_t = tridiag(-1; 1, 2, ..., 2; -1).  For
 * BE the two are the same matrix; for BDF2 D_t D_t^T is pentadiagonal, applied per
 * Fourier mode by LDL^T factors computed at create.  Plain path only (PDHG_PATH_AUTO
 * then chooses it; PDHG_PATH_FUSED gives PDHG_ERR_UNSUPPORTED), at most 2^24
 * (mode, slice) pairs.  The fixed point does not depend on it. */
enum { PDHG_FLAG_EXACT_TIME_PRECOND = 1,
/* PDHG_FLAG_U0_ON_DEVICE: pdhg_problem.u0 is a device pointer (float64, ndof values, kept
 * by the caller).  The library converts it on the device and takes the finite check and
 * the Lax-Friedrichs constant (lf_a = 0) from a device scan: u0 is not copied to the
 * host.  Accepted by pdhg_create and every entry point built on it (mixed, refine,
 * gradient, batch); PDHG_ERR_UNSUPPORTED for pdhg_solve_one_step. */
       PDHG_FLAG_U0_ON_DEVICE = 2,
/* PDHG_FLAG_T_SOLVE_FP64 (float32 handles; an ablation of the precision of the t-solve):
 * the recurrences of the tridiagonal t-solve (the closed-form pivots and the running
 * forward and backward values) in float64, each stored value rounded to float32 once.
 * Finite differences with T_t only (PDHG_ERR_UNSUPPORTED with DG or the exact time
 * operator); on the fused path only for ny = 1024 (PDHG_PATH_AUTO then takes the plain
 * path for other ny).  No effect on float64 handles. */
       PDHG_FLAG_T_SOLVE_FP64 = 4,
/* PDHG_FLAG_MIXED_STEPS (pdhg_one_step_workspace_size / pdhg_solve_one_step only;
 * scheme->precision is then ignored): each step of Algorithm 3 runs in float32 until its
 * Res reaches tol or stops falling (the worse entry not 5% lower than three checks
 * before: float32's rounding floor), then goes on in float64 from the widened state
 * (K_d^{-1} applied in float32, as the float64 phase of pdhg_solve_mixed) to tol; u_out
 * holds float64 values and iters_per_step counts both phases.  Other entry points:
 * PDHG_ERR_INVALID_ARG. */
       PDHG_FLAG_MIXED_STEPS = 8 };
typedef struct {
    int32_t time, space, precision, init, path, flags;
} pdhg_scheme;

typedef struct pdhg_handle pdhg_handle;

/* Bytes of device workspace that pdhg_create() needs for this problem. */
pdhg_status pdhg_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                const pdhg_scheme *scheme, size_t *bytes);

/* Validate, lay out the workspace, upload u0 and the preconditioner tables,
 * and set the initial guess [u0 extended in t, 0, 0] (Sec. 3.3).  The
 * workspace (device pointer, >= pdhg_workspace_size bytes, 256-byte aligned)
 * stays owned by the caller.  Synchronises the stream before returning. */
pdhg_status pdhg_create(const pdhg_problem *prob, const pdhg_grid *grid,
                        const pdhg_scheme *scheme, void *workspace, size_t bytes,
                        void *stream, pdhg_handle **out);

/* Free the host handle (the workspace is the caller's to free). NULL is a no-op. */
pdhg_status pdhg_destroy(pdhg_handle *h);

/* Change the stream used by later calls.  Waits for the work already queued on the old
 * stream first, so later calls on the new stream see a finished state.  Errors:
 * INVALID_ARG, CUDA. */
pdhg_status pdhg_set_stream(pdhg_handle *h, void *stream);

/* Run iterations of Algorithm 1.
 * check_every > 0: every check_every iterations compute Res (Eq. 2.12) and stop
 *   once both entries are <= tol (absolute; relative to ||A(u_init)|| when
 *   relative != 0); synchronises at each check.  Returns NONFINITE/DIVERGED on
 *   a bad residual, TIMEOUT when a bounded device wait of the fused path gave
 *   up since the last check (the state is then invalid).
 * check_every <= 0: enqueue max_iters iterations asynchronously (no host sync).
 * *iters_done (may be NULL) receives the iterations performed by this call. */
pdhg_status pdhg_iterate(pdhg_handle *h, int64_t max_iters, double tol, int32_t check_every,
                         int32_t relative, int64_t *iters_done);

/* Res of Eq. 2.12 at the current state, absolute, synchronously:
 * out[0] = ||A(u)|| (equations and initial row), out[1] = ||grad_u L|| =
 * ||J(u)^T phi|| (rows l >= 1, plus the u^0 row h_t (J^T phi)^0 + lambda with
 * init LAMBDA), out[2] = ||u^0 - u0||, out[3] = the Lagrangian <phi, R(u)> +
 * <lambda, u^0 - u0> (the duality-gap diagnostic; the objective is 0).
 * Norms are discrete L2 with weights h_t*w_x per equation dof, w_x per
 * initial-row dof (w_x = h_x, or h_x*h_y in 2D).  TIMEOUT as pdhg_iterate. */
pdhg_status pdhg_residual(pdhg_handle *h, double out[4]);

/* Residual history (a diagnostic of this library; the paper plots Res against the
 * iteration count, Sec. 4): every check of pdhg_iterate (every check_every iterations,
 * and the last iteration of a call) -- and every check of pdhg_batch_iterate for the
 * instance's handle -- records one row of 5 doubles: the handle's iterations so far,
 * then the four entries of pdhg_residual at that point (absolute values).  The newest
 * 65536 rows are kept (host memory of the handle; nothing on the device).
 * max_rows = 0: *rows = the number of rows held (out may be NULL).  max_rows > 0: the
 * oldest min(max_rows, held) rows are copied to out (host, row-major, 5 doubles per
 * row) and *rows is that number.  clear != 0 empties the history after the copy (rows
 * not copied are dropped).  Errors: INVALID_ARG (null handle or rows, max_rows < 0, out
 * NULL with max_rows > 0). */
pdhg_status pdhg_residual_history(pdhg_handle *h, double *out, int64_t max_rows, int64_t *rows, int32_t clear);

/* Copy a field (PDHG_FIELD_*) out of / into the state.  dst/src has the
 * handle's element type; on_device != 0 means a device pointer.  Sizes in
 * elements: U (nt+1)*ndof, U_TERMINAL ndof (get only), PHI/PHIT nt*ndof,
 * LAMBDA/LAMBDAT ndof.  Synchronous. */
pdhg_status pdhg_get_field(pdhg_handle *h, int32_t field, void *dst, int32_t on_device);
pdhg_status pdhg_set_field(pdhg_handle *h, int32_t field, const void *src, int32_t on_device);

/* The solution read of Algorithm 1's state: which = PDHG_FIELD_U (all slices u^0..u^nt),
 * PDHG_FIELD_U_TERMINAL (u^nt), PDHG_FIELD_PHI or PDHG_FIELD_LAMBDA (the multipliers);
 * the same copy as pdhg_get_field.  Other values: INVALID_ARG. */
pdhg_status pdhg_solution(pdhg_handle *h, void *dst, int32_t dst_on_device, int32_t which);

/* Element counts and iteration counter of the handle. */
pdhg_status pdhg_info(pdhg_handle *h, int64_t *ndof, int64_t *nt, int64_t *iterations,
                      int32_t *precision, int32_t *path);

/* Kernel launches issued by this handle since create (or the last reset). */
pdhg_status pdhg_launch_count(pdhg_handle *h, int64_t *launches, int32_t reset);

/* Per-stage timing with CUDA events on the handle's stream.  While enabled,
 * pdhg_iterate records an event pair around every stage launch (and marks each
 * stage's launches with an NVTX range named "pdhg <stage>", for ncu --nvtx);
 * stage_times returns accumulated milliseconds and launch counts per
 * PDHG_STAGE_* and resets them.  Synchronises the stream. */
pdhg_status pdhg_set_profiling(pdhg_handle *h, int32_t enable);
pdhg_status pdhg_stage_times(pdhg_handle *h, double ms[PDHG_NUM_STAGES],
                             int64_t launches[PDHG_NUM_STAGES]);

/* CUDA graphs (not used while profiling): with check_every = m > 0, pdhg_iterate
 * captures m iterations plus the residual check as one graph on first use and
 * replays it on the handle's stream for every full chunk of m iterations (fewer
 * launches for small, launch-bound problems; the kernels and their order are
 * unchanged, so results are identical).  A capture the driver refuses falls back
 * to kernel-by-kernel launches.  Default: on for the plain path and for fused
 * problems of at most 2^23 cell-iterations (nt x ndof), off for larger fused ones;
 * enable = 0 turns graphs off, enable = 1 on.  pdhg_set_wait_budget drops a
 * captured graph (the budget is a launch argument of the fused rows-C kernel). */
pdhg_status pdhg_set_graphs(pdhg_handle *h, int32_t enable);

/* Budget, in nanoseconds, of each bounded device wait (the TMA stage waits of the
 * fused path's nx = 1024 rows-C kernel; default 1e9).  A wait that runs out sets a
 * device flag, its block drains its copies in flight and returns, and the next
 * residual evaluation returns PDHG_ERR_TIMEOUT (the state is then invalid; the
 * CUDA context stays usable).  ns = 0 gives up at once: the host-side way to
 * exercise that path.  No effect on handles without bounded waits. */
pdhg_status pdhg_set_wait_budget(pdhg_handle *h, uint64_t ns);

/* Message of the last error on the calling thread ("" if none). */
const char *pdhg_last_error(void);

/*
 * Algorithm 2 (Sec. 3.4): refinement of the time mesh.  Solves the problem on
 * nt/2^(levels-1), nt/2^(levels-2), ..., nt slices of the same horizon T, each
 * level started from the previous level's (u, phi, lambda) carried to the finer
 * mesh: u and phi linearly in t (u^l sits at time l h_t, phi^l -- the multiplier
 * of R^l -- at (l+1) h_t, constant below the first coarse time), lambda copied,
 * and phit = phi, lamt = lambda.  The first level starts from [u0, 0, 0].
 *
 * levels in [1, 16]; grid->nt divisible by 2^(levels-1).  iters[k] (host,
 * `levels` entries, coarsest first) bounds level k's iterations; a level stops
 * early once Res <= tol when check_every > 0 (same rules as pdhg_iterate, with
 * `relative` relative to that level's cold-start residual).  iters_done (host,
 * `levels` entries, may be NULL) receives the counts.
 *
 * The workspace (device, caller-owned, 256-byte aligned, size from
 * pdhg_refine_workspace_size) holds two alternating regions; the returned
 * handle is the finest level, lives in the workspace, and is used and
 * destroyed like one from pdhg_create.  Errors as pdhg_create/pdhg_iterate;
 * on an error no handle is returned.
 */
pdhg_status pdhg_refine_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                       const pdhg_scheme *scheme, int32_t levels, size_t *bytes);
pdhg_status pdhg_solve_refine(const pdhg_problem *prob, const pdhg_grid *grid,
                              const pdhg_scheme *scheme, int32_t levels, const int64_t *iters,
                              double tol, int32_t check_every, int32_t relative, void *workspace,
                              size_t bytes, void *stream, pdhg_handle **out, int64_t *iters_done);

/*
 * Algorithm 3 (Sec. 3.5): one time step at a time.  For l = 0..nt-1, runs
 * Algorithm 1 on the two-slice problem over [l h_t, (l+1) h_t] whose initial
 * data is u*^l (u*^0 = u0), started from [u*^l, u*^l], 0, 0, until both
 * entries of its Res are <= tol, checked every check_every iterations, or
 * max_iters_per_step.  Res here is the L2 norm over the domain at one time
 * (weight w_x, no h_t), as Sec. 3.5 defines it.  Every input of the full
 * problem is kept (flux, c, step sizes, h_t, and the Lax-Friedrichs constant
 * computed from the full problem's u0 when prob->lf_a is 0), so with tol -> 0
 * the result is the full scheme's solution.  BDF2: the equation of step l >= 1,
 * (3 v - 4 u^l + u^{l-1}) / (2 h_t) + D(v) = 0, is the backward-Euler equation of a
 * step of length 2 h_t / 3 from w = (4 u*^l - u*^{l-1}) / 3, so that step runs as the
 * two-slice BE problem started from w (step 0 is the scheme's BE start).
 * The step handles take scheme->path: float32 2D finite-difference steps (and the
 * float32 phase of PDHG_FLAG_MIXED_STEPS) run on the fused path with PDHG_PATH_AUTO or
 * PDHG_PATH_FUSED where it applies (nx in [256, 2048], ny in [256, 1024]); float64
 * steps run on the plain path.
 *
 * u_out: device, (nt+1)*ndof values of the scheme's precision (float64 with
 * PDHG_FLAG_MIXED_STEPS), written with u*^0..u*^nt.  iters_per_step (host, nt entries)
 * and iters_total may be NULL.  workspace: device, caller-owned, 256-byte aligned, size
 * from pdhg_one_step_workspace_size (one handle with nt = 1, or a float32 and a float64
 * one with PDHG_FLAG_MIXED_STEPS; twice that for BDF2, the second for the step length
 * 2 h_t / 3).  Synchronises the stream before returning.  A step that fails (NONFINITE, DIVERGED, CUDA)
 * returns its status; u_out then holds the steps completed so far.
 */
pdhg_status pdhg_one_step_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                         const pdhg_scheme *scheme, size_t *bytes);
pdhg_status pdhg_solve_one_step(const pdhg_problem *prob, const pdhg_grid *grid,
                                const pdhg_scheme *scheme, double tol, int64_t max_iters_per_step,
                                int32_t check_every, void *workspace, size_t bytes, void *stream,
                                void *u_out, int64_t *iters_per_step, int64_t *iters_total);

/*
 * Gradient of a terminal objective through the solve.  (An addition of this
 * library: the paper solves forward problems only.)  With u the scheme's
 * solution for the problem's u0 and nu,
 *     Loss = w_x sum_j (u_j^nt - target_j)^2      (w_x = h_x, or h_x h_y in 2D),
 * returns Loss, dLoss/du0_j (for every dof j) and dLoss/dnu.  Both come from the
 * saddle form of Eq. 2.7 / 3.10 with Loss added as the primal objective: at its
 * stationary point phi and lambda are the discrete adjoint, dLoss/du0 = -w_x lambda
 * and dLoss/dnu = h_t w_x sum_l <phi^l, dR^l/dnu> = -h_t w_x sum_l <phi^l, Lap_h u^{l+1}>.
 *
 * Two runs of Algorithm 1 on one handle (plain path): the forward problem to
 * Res <= tol (absolute, checked every check_every iterations, at most max_iters),
 * then the same problem linearised at the forward solution u* (residual
 * J(u*) v, transposes at u*) with the objective |u*^nt + v^nt - target|^2,
 * whose last-slice update is the objective's proximal step; this linearised
 * saddle problem is convex, so Algorithm 1 converges on it like on a linear
 * problem.  Stops at Res <= adj_tol or adj_max_iters.
 *
 * Finite-difference schemes (1D or 2D, BE or BDF2, constant or zero nu, with or
 * without gamma_half), PDHG_INIT_LAMBDA; PDHG_ERR_UNSUPPORTED otherwise (DG,
 * PDHG_INIT_PINNED, PDHG_PATH_FUSED).  target: host, ndof float64 values.
 * workspace: device, caller-owned, 256-byte aligned, size from
 * pdhg_gradient_workspace_size.  loss, du0 (host, ndof), dnu, iters (host, 2:
 * forward and adjoint iterations) may be NULL.  Synchronises the stream.
 * Errors as pdhg_iterate (NONFINITE, DIVERGED, CUDA), for either solve.
 */
pdhg_status pdhg_gradient_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                         const pdhg_scheme *scheme, size_t *bytes);
pdhg_status pdhg_solve_gradient(const pdhg_problem *prob, const pdhg_grid *grid,
                                const pdhg_scheme *scheme, const double *target, double tol,
                                int64_t max_iters, double adj_tol, int64_t adj_max_iters,
                                int32_t check_every, void *workspace, size_t bytes, void *stream,
                                double *loss, double *du0, double *dnu, int64_t *iters);

/*
 * Mixed-precision solve (an addition of this library: the paper states no
 * precision).  Algorithm 1 runs in float32 -- on the fused path where
 * pdhg_create would choose it, scheme->path as given -- until both entries of
 * Res are <= tol (absolute, or relative to ||A(u_init)||), checked every
 * check_every iterations, or until the larger entry has not fallen by 5% over
 * the last three checks (float32's rounding floor); then the state (u, phi,
 * phit, lambda, lamt) is widened to float64 on the device and Algorithm 1 goes
 * on in float64 on the plain path to tol (from the float32 state this phase is
 * short: checked after 1, 2, 3, 4, 6, 9, 13, ... of its iterations, the gaps
 * growing to at most max(1, check_every/5)), within max_iters iterations in all.
 * For finite differences with nx a power of two that phase applies K_d^{-1} in
 * float32 (residual, u, phi, lambda and Res stay float64): the preconditioner
 * shapes the iteration, not its fixed point, so the result is the float64 one.
 * scheme->precision is ignored.
 *
 * workspace: device, caller-owned, 256-byte aligned, size from
 * pdhg_mixed_workspace_size (a float32 and a float64 handle's regions).  The
 * returned handle is the float64 one, in the workspace; use and destroy it like
 * one from pdhg_create.  iters (host, 2 entries, may be NULL): float32 and
 * float64 iterations.  Errors as pdhg_create / pdhg_iterate; on an error no
 * handle is returned.
 */
pdhg_status pdhg_mixed_workspace_size(const pdhg_problem *prob, const pdhg_grid *grid,
                                      const pdhg_scheme *scheme, size_t *bytes);
pdhg_status pdhg_solve_mixed(const pdhg_problem *prob, const pdhg_grid *grid,
                             const pdhg_scheme *scheme, double tol, int32_t relative,
                             int32_t check_every, int64_t max_iters, void *workspace, size_t bytes,
                             void *stream, pdhg_handle **out, int64_t iters[2]);

/*
 * Batches of independent 1D instances (an addition of this library: the paper
 * solves one problem at a time).  Each instance is an ordinary problem (any 1D
 * scheme of this library, its own nx, nt, flux, time scheme and step sizes;
 * one precision for all) held as a handle on the plain path; every stage of
 * Algorithm 1 is one launch over all active instances, whose blocks run the
 * same per-block code as the single-instance launches, so a batched instance
 * follows exactly the iterates it would follow alone.  Instances that reach
 * the tolerance, or whose residual stops being finite or grows by 1e10, leave
 * the launches at the next check.
 *
 * pdhg_batch_workspace_size / pdhg_batch_create: `count` structs each (host
 * arrays); workspace device, caller-owned, 256-byte aligned.  Errors as
 * pdhg_create, naming the failing instance; PDHG_ERR_UNSUPPORTED for 2D or
 * PDHG_PATH_FUSED.
 * pdhg_batch_iterate: up to max_iters iterations of every active instance,
 * Res checked every check_every iterations (0: never) against tol (absolute,
 * or relative to each instance's cold-start residual).  iters (host, count
 * entries, may be NULL): iterations each instance ran in this call; state
 * (host, count, may be NULL): 1 converged, 0 still active, -1 non-finite or
 * diverged.  Returns PDHG_OK unless a launch fails.
 * pdhg_batch_reset: makes every instance active again (their states are kept).
 * pdhg_batch_instance: borrowed handle of instance i (fields, residual, info;
 * owned and destroyed by the batch).
 */
typedef struct pdhg_batch pdhg_batch;
pdhg_status pdhg_batch_workspace_size(int32_t count, const pdhg_problem *probs,
                                      const pdhg_grid *grids, const pdhg_scheme *schemes,
                                      size_t *bytes);
pdhg_status pdhg_batch_create(int32_t count, const pdhg_problem *probs, const pdhg_grid *grids,
                              const pdhg_scheme *schemes, void *workspace, size_t bytes,
                              void *stream, pdhg_batch **out);
pdhg_status pdhg_batch_destroy(pdhg_batch *b);
pdhg_status pdhg_batch_iterate(pdhg_batch *b, int64_t max_iters, double tol, int32_t check_every,
                               int32_t relative, int64_t *iters, int32_t *state);
pdhg_status pdhg_batch_reset(pdhg_batch *b);
pdhg_status pdhg_batch_instance(pdhg_batch *b, int32_t i, pdhg_handle **h);
pdhg_status pdhg_batch_launch_count(pdhg_batch *b, int64_t *launches, int32_t reset);

/*
 * How a batch iteration is launched (an addition of this library).  persistent != 0:
 * ONE cooperative launch per iteration whose resident blocks take work items from a
 * queue -- every active instance's primal items, its residual + x-FFT rows, its t-solve
 * columns, its inverse x-FFT + dual rows; order 0: stage after stage, instances with
 * most cells first within a stage; order 1: instance after instance (most cells first),
 * each with its four stages in turn.  An item of a later stage of an
 * instance starts once that instance's items of the stage before are finished (a wait
 * bounded by the budget of pdhg_batch_set_wait_budget; one that gives up makes the next
 * residual check of pdhg_batch_iterate return PDHG_ERR_TIMEOUT and leaves the state
 * invalid; the context stays usable).  persistent == 0 (the default): one launch per
 * stage (four per iteration).  Both run the same per-block code, so results are
 * identical.
 * blocks_per_sm: resident blocks per multiprocessor of the persistent launch (0: as
 * many as fit).  tiles (host, 8 entries, may be NULL to keep): row items per queue entry
 * for each size class c = clamp(log2(row transform length) - 8, 0, 7) (the Bluestein
 * length L, or nx/2 for the packed real FFT), each in [1, 64]; chosen per class by the
 * library's autotuner (paper_2207_07234_gb300/autotune.py).  Errors: INVALID_ARG.
 */
pdhg_status pdhg_batch_set_launch(pdhg_batch *b, int32_t persistent, int32_t blocks_per_sm, int32_t order,
                                  const int32_t *tiles);

/* Budget in nanoseconds of each bounded wait of the persistent batch iteration
 * (default 1e9); 0 gives up at the first wait: the host-side way to exercise the
 * PDHG_ERR_TIMEOUT path. */
pdhg_status pdhg_batch_set_wait_budget(pdhg_batch *b, uint64_t ns);

/* CUDA graphs for the batch (default on): pdhg_batch_iterate captures check_every
 * iterations plus the residual check kernels once and replays the graph for each whole
 * chunk of check_every iterations (a tail shorter than check_every, and runs with
 * check_every == 0, launch kernel by kernel).  The graph is rebuilt when the active set
 * or the launch choice changes.  The replayed launches are those of the kernel-by-kernel
 * run, so results are identical.  enable == 0: no graphs.  Errors: INVALID_ARG. */
pdhg_status pdhg_batch_set_graphs(pdhg_batch *b, int32_t enable);

/*
 * Residual norms of a caller-held state, with no handle, no workspace and no
 * device allocation.  (An addition of this library: the paper has no
 * counterpart.)  For callers that cannot allocate device memory -- e.g. code
 * that may only use buffers it was handed, or that runs where the allocator
 * must not be entered -- and so cannot provide pdhg_create()'s workspace.
 *
 * Computes the same out[0..3] as pdhg_residual() for the state given by device
 * pointers in the scheme's element type: u ((nt+1)*ndof), phi (nt*ndof), lambda
 * (ndof; may be NULL with PDHG_INIT_PINNED), u0 (ndof) and gamma_half (nx, or
 * NULL).  prob->u0 and prob->gamma_half are ignored; prob->lf_a must be > 0
 * for the Lax-Friedrichs schemes.  The grid, scheme and coefficients pass the
 * same checks as in pdhg_create (sizes, powers of two, nu >= 0, finite
 * coefficients; the step sizes and scheme->path are not used):
 * PDHG_ERR_INVALID_ARG / PDHG_ERR_UNSUPPORTED otherwise, before any device work.
 * Enqueued on `stream`, then synchronised.
 *
 * Scratch: a fixed 2 MiB array in device memory, part of the library image
 * (held on every GPU that uses it until the process exits).  Problems with
 * min(ceil(units/4096), max(32, 1216/(nt+1)))*(nt+1) > 43685 partial blocks (units = ndof, or
 * cells for DG; so nt <= 1364 always fits) are rejected with
 * PDHG_ERR_UNSUPPORTED before any device work.  All calls share the array: calls that overlap on
 * the GPU race; calls ordered on one stream are safe.  The first call in each
 * CUDA context (a device's primary context; again after cudaDeviceReset) looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make it before any stream capture.
 */
pdhg_status pdhg_residual_noalloc(const pdhg_problem *prob, const pdhg_grid *grid,
                                  const pdhg_scheme *scheme, const void *u, const void *phi,
                                  const void *lambda, const void *u0, const void *gamma_half,
                                  double out[4], void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PDHG_H */
