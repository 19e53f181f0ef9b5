/*
 * molt.h -- C ABI of libmolt, a GB300 (sm_103a) implementation of the MOL^T
 * recursive-convolution wave solver of Causley & Christlieb,
 * "Higher order A-stable schemes for the wave equation using a recursive
 * convolution approach" (arXiv:1308.3214).
 *
 * What it computes
 *   The wave equation u_tt = c^2 Lap u on a rectangle / box (1D, 2D, 3D) with
 *   homogeneous Dirichlet or periodic boundaries, advanced by the A-stable
 *   scheme of order 2P (Sec. 3 eq. update_P in 1D; Sec. 4 eq. Full_2D with the
 *   ADI operators C and D in 2D/3D):
 *       u^{n+1} = 2 u^n - u^{n-1} + F[u^n],
 *       F = sum_{p=1}^{P} sum_{m=1}^{p} (-1)^m 2 beta^{2m}/(2m)! binom(p-1,m-1) C^m D^{p-m}.
 *   Every operator is built from the per-axis convolution
 *       L_gamma^{-1} = (1 - d^2/dgamma^2 / alpha^2)^{-1},  alpha = beta/(c dt)
 *   (eqs. L_def, L_Inverse), evaluated on each grid line by two exponential
 *   recurrences (Sec. 2) plus the boundary terms A e^{-alpha(x-a)} +
 *   B e^{-alpha(b-x)}, and D_gamma = 1 - L_gamma^{-1} (eq. LD_gam).  The local
 *   increments integrate the quadratic interpolant exactly (the rule that
 *   reproduces Table 2); the linear rule is available as an option.
 *
 * Conventions
 *   - Fields are contiguous, x fastest: index = x + nx*(y + ny*z), with
 *     grid.n[0] = nx, grid.n[1] = ny, grid.n[2] = nz.
 *   - A Dirichlet axis of n points includes both end nodes (spacing
 *     (hi-lo)/(n-1)); a periodic axis holds n distinct points ((hi-lo)/n).
 *     Dirichlet data must vanish on the boundary (homogeneous condition).
 *   - Field pointers are DEVICE pointers to float64 arrays owned by the caller
 *     unless a function says "host".  The library never frees them.
 *   - Every call is asynchronous on the given CUDA stream (a cudaStream_t
 *     passed as void*, NULL = legacy default stream) unless stated otherwise;
 *     errors that the host can see are returned at once, device errors at the
 *     next synchronising call (mol_sync, mol_solve_host).
 *   - Nothing throws across the ABI.  On error a call returns a nonzero
 *     mol_status and mol_last_error(handle) describes it.
 *   - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef MOLT_H
#define MOLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MOL_OK = 0,
    MOL_EINVAL = 1,     /* bad argument (sizes, pointers, P, axis, ...)        */
    MOL_ENOMEM = 2,     /* device or host allocation failed                     */
    MOL_ECUDA = 3,      /* a CUDA runtime call failed                            */
    MOL_EUNSTABLE = 4,  /* beta above beta_max(P): the scheme is not A-stable    */
    MOL_ETIMEOUT = 5    /* a bounded device wait gave up                         */
} mol_status;

typedef enum { MOL_BC_PERIODIC = 0, MOL_BC_DIRICHLET = 1 } mol_bc;

/* Arithmetic of the line sweeps.
 *   MOL_FP64:  everything in float64.
 *   MOL_MIXED: sweeps and intermediate fields in float32; the time levels are
 *              kept as float32 pairs (hi + lo, about 48 significant bits) and
 *              the level update and the first second difference of u^n are
 *              formed in that pair arithmetic. */
typedef enum { MOL_FP64 = 0, MOL_MIXED = 1 } mol_prec;

typedef struct {
    int ndim;           /* 1, 2 or 3                                   */
    int64_t n[3];       /* points per axis, x first                    */
    double lo[3];       /* domain lower corner                         */
    double hi[3];       /* domain upper corner                         */
} mol_grid;

typedef struct {
    int quad_order;     /* 2 (default): quadratic local interpolant; 1: linear */
    int lines_per_block;/* 0 = automatic; else 1, 2, 4, 8 or 16 lines per CTA    */
    int use_graphs;     /* 1 (default): replay the time loop as a CUDA graph;
                         * 0: direct launches; 2 (batches): graphs with the
                         * passes of all problems joined at every step (1 runs
                         * the launches of a batch's size classes as
                         * independent chains where each class's y and x
                         * launches cover the same problems)                 */
} mol_options;

typedef struct mol_ctx *mol_handle;

/* Defaults for mol_options (quad_order 2, automatic tiling, graphs on). */
void mol_default_options(mol_options *opt);

/*
 * Create a solver.  Host-only work (constants, coefficient expansion) plus the
 * device workspace allocation; no kernel runs.
 *   grid  : domain and points; every axis needs n >= 3 and n <= mol_max_line().
 *   c, dt : wave speed and time step (> 0); alpha = beta/(c dt) (eq. L_def).
 *   beta  : 0 < beta <= beta_max(P) (Theorem of Sec. 3.1, Table 1); beta <= 0
 *           selects beta_max(P).  beta > beta_max(P) -> MOL_EUNSTABLE.
 *   P     : 1..5, the scheme has order 2P.
 *   bc    : boundary condition of every axis.
 *   prec  : sweep arithmetic (see mol_prec).
 *   opt   : NULL for defaults.
 *   out   : receives the handle (NULL on failure).
 * The handle owns its device workspace until mol_destroy.
 */
mol_status mol_create(const mol_grid *grid, double c, double dt, double beta, int P,
                      mol_bc bc, mol_prec prec, const mol_options *opt, mol_handle *out);

/* (2D Dirichlet grids with at most 1024 points per axis whose lines do not
 * split into whole register segments run mol_apply_F, mol_start, mol_step
 * and mol_solve_host on the batched kernels, as a batch of one problem.) */

/* Free the workspace and the handle (waits for the handle's work). */
mol_status mol_destroy(mol_handle h);

/* Message of the last failed call on h (static text if h is NULL). */
const char *mol_last_error(mol_handle h);

/* beta_max(P): the first positive root of -sum_{p<=P} A_p(beta) = 4
 * (eq. Stab_cond; Table 1).  Returns -1 for P outside 1..5. */
double mol_beta_max(int P);

/* Longest line (points per axis) the on-chip sweep supports for prec. */
int64_t mol_max_line(mol_prec prec);

/* Scalars of the solver: out[0] = alpha, out[1] = beta, out[2..4] = nu per
 * axis (alpha * h_gamma), out[5..7] = d = e^{-nu} per axis. */
mol_status mol_get_params(mol_handle h, double out[8]);

/*
 * out = D_axis^power v  (eq. LD_gam: D_gamma = 1 - L_gamma^{-1}, Sec. 3:
 * powers by repeated application).  v, out: device float64 fields of the
 * grid's size; they may not overlap.  axis in [0, ndim), 1 <= power <= 8.
 */
mol_status mol_apply_D(mol_handle h, const double *v, double *out, int axis, int power,
                       void *stream);

/* F = F[u], the spatial operator of the update (eq. update_P / Full_2D). */
mol_status mol_apply_F(mol_handle h, const double *u, double *F, void *stream);

/* Start value for zero initial velocity: u1 = u0 + F[u0]/2 (Sec. 3.2). */
mol_status mol_start(mol_handle h, const double *u0, double *u1, void *stream);

/*
 * Advance (u_prev, u_cur) = (u^{n-1}, u^n) by nsteps >= 0 steps in place:
 * on return u_prev = u^{n+nsteps-1}, u_cur = u^{n+nsteps}.  The two buffers
 * are device float64 fields and may not overlap.  The library keeps the
 * levels in its own workspace during the call.
 */
mol_status mol_step(mol_handle h, double *u_prev, double *u_cur, int64_t nsteps, void *stream);

/*
 * End-to-end solve from HOST memory: copies u0 (host float64, grid size) to
 * the device, forms u1 = mol_start(u0), advances to u^{nsteps} and copies it
 * back into u_out (host float64).  Synchronous.  nsteps >= 1.
 */
mol_status mol_solve_host(mol_handle h, const double *u0, double *u_out, int64_t nsteps,
                          void *stream);

/*
 * Autotuner: times the launch variants that change something for this grid
 * -- the float32 x pass with one warp per row (1, 2 or 4 warps per CTA) or
 * each row split over 2, 4 or 8 warps (rows of 32 W RPT points), one CTA per
 * row or persistent CTAs that prefetch their next row (MOL_TUNE_ROWS_PERSIST),
 * the strided segment length (64 or 32 points per thread for float32 sweeps)
 * and the segments per CTA at most (8 or 4, hence the cluster size) -- on the
 * handle's own workspace (a few steps each, CUDA events, minimum of 3
 * timings) and keeps the fastest for every later call.  Synchronous on the
 * stream; the caller's fields are not touched.  The paper has no counterpart.
 */
mol_status mol_autotune(mol_handle h, void *stream);

/* Force launch choices (e.g. a tuning result kept from an earlier run):
 * res_warps 1, 2 or 4; strided_rpt 0 (default) or 32; strided_warps 1..8;
 * rows_warps 0 (one warp per row) or 2, 4, 8 (each row split over that many
 * warps, where the row length allows it).  MOL_EINVAL if a choice is out of
 * range or does not fit an axis. */
mol_status mol_set_tuning(mol_handle h, int res_warps, int strided_rpt, int strided_warps, int rows_warps);

/* The launch choices in use: out[0] = warps per CTA of the resident x pass,
 * out[1] = strided segment length (0 = default), out[2] = segments per CTA at
 * most, out[3] = warps per row (0 = one); *ms_per_step (may be NULL) = the
 * tuned step time (0 before tuning). */
mol_status mol_get_tuning(mol_handle h, int out[4], double *ms_per_step);

/* The full set of launch choices, by index (later indices may be added; a
 * caller passes how many it knows):
 *   MOL_TUNE_RES_WARPS .. MOL_TUNE_ROWS_WARPS: as mol_set_tuning;
 *   MOL_TUNE_ROWS_PERSIST: 1 = the row-split x pass runs persistent CTAs
 *     (as many as fit on the device) that walk the rows and prefetch the
 *     next row's fields into L2 while they work on the current one; 0 = one
 *     CTA per row;
 *   MOL_TUNE_STRIDED_NB: 1 (default) = the float32 strided passes (powers,
 *     and the Horner pass of 3D grids) exchange once per sweep between
 *     neighbouring segments wherever the decay over one segment makes that
 *     exact to below 2^-30 (d^(RPT-1) <= 2^-30); 2 = the same, and the
 *     Horner pass stages the CTA's rows of its input fields in shared memory
 *     once instead of reading them from global memory for every output and
 *     power (where two CTAs per SM still fit; else as 1); 0 = the full-carry
 *     passes (three exchanges per sweep) always;
 *   MOL_TUNE_STRIDED_STAGE: how that pass moves its tiles: 0 direct
 *     coalesced loads and stores from registers; 1 the pair level's tile (the
 *     CTA's rows plus halos, 32 lines) copied into shared memory by TMA tensor
 *     loads on an mbarrier; 2 (default) each output power staged in shared
 *     memory and written by TMA tensor stores; 3 both.  Grids whose 32-line
 *     groups would straddle an outer slice (inner extent not a multiple of 32)
 *     take 0;
 *   MOL_TUNE_ROWS_NB: 1 (default) = the row-split x pass exchanges once per
 *     sweep between neighbouring segments where the dropped inflows are below
 *     1/8 of a float32 unit in the last place: two warps per row with the two
 *     neighbours (d^(RPT-1) <= 2^-27) or four warps per row with two on each
 *     side (d^(2 RPT - 1) <= 2^-27); 0 = the full carries (scans over the
 *     warp and a combine over the warps, three barriers per sweep);
 *   MOL_TUNE_PDL: 1 = the register-resident pass kernels are launched as
 *     programmatic dependents of the kernel before them in the stream (their
 *     CTAs are scheduled while it finishes and wait for its completion before
 *     touching memory); 0 (default) = ordinary stream order.  Bitwise the
 *     same results; measured 2 % (2D) to 4 % (3D) slower per step, the
 *     waiting CTAs holding SM slots through the previous pass's last wave.
 * mol_set_tuning_ex takes count >= 4 values (indices past count keep their
 * setting); mol_get_tuning_ex fills count values.  MOL_EINVAL on a value out
 * of range, a count out of range or a choice that does not fit the grid. */
enum {
    MOL_TUNE_RES_WARPS = 0,
    MOL_TUNE_STRIDED_RPT = 1,
    MOL_TUNE_STRIDED_WARPS = 2,
    MOL_TUNE_ROWS_WARPS = 3,
    MOL_TUNE_ROWS_PERSIST = 4,
    MOL_TUNE_STRIDED_NB = 5,
    MOL_TUNE_STRIDED_STAGE = 6,
    MOL_TUNE_ROWS_NB = 7,
    MOL_TUNE_PDL = 8,
    MOL_TUNE_COUNT = 9
};
mol_status mol_set_tuning_ex(mol_handle h, const int *vals, int count);
mol_status mol_get_tuning_ex(mol_handle h, int *vals, int count, double *ms_per_step);

/*
 * Adjoint on a single-problem handle (2D Dirichlet, at most 1024 points per
 * axis; MOL_EINVAL otherwise): F^T, receiver traces and the gradient of a
 * trace loss with respect to the initial field, as mol_batch_apply_FT /
 * mol_batch_traces / mol_batch_adjoint for a batch of this one problem
 * (receivers: flat indices y nx + x; host arrays).  The paper has no adjoint.
 */
mol_status mol_apply_FT(mol_handle h, const double *w, double *out, void *stream);
mol_status mol_traces(mol_handle h, const double *u0, int nrec, const int64_t *rec, int64_t nsteps, double *traces,
                      void *stream);
mol_status mol_adjoint(mol_handle h, int nrec, const int64_t *rec, int64_t nsteps, const double *tgrad, double *grad,
                       void *stream);

/* Wait for the handle's work on the stream; reports device-side errors. */
/* Time-dependent Dirichlet data on a 1D Dirichlet handle (Sec. 3.2):
 * u(a, t) = u_L(t), u(b, t) = u_R(t), zero initial velocity.  u0: device,
 * float64, the n points of u^0 (its end values the data at t_0); u_out:
 * device, float64, receives u^nsteps.  data: HOST, float64,
 * [nsteps + 1][2][P + 1]: data[k][side][m] = (d^2/dt^2 / c^2)^m u_side(t_k),
 * t_k = k dt, side 0 = a, 1 = b (m = 0: the value itself).  The boundary
 * values of D^p u come from the operator identity D = -(d_xx/alpha^2)
 * (1 - d_xx/alpha^2)^{-1} with d_xx -> d_tt/c^2 at the ends (the inverse
 * Lax-Wendroff limit of Sec. 3.2), expanded to the scheme's order:
 * (-1)^p sum_{j=p..P} C(j-1, p-1) alpha^{-2j} data[k][side][j].  The end
 * nodes of every new level take the data.  Runs on the shared-memory line
 * kernels, one launch per step (no graph).  Errors: MOL_EINVAL for another
 * grid or NULL pointers. */
mol_status mol_solve_dirichlet(mol_handle h, const double *u0, int64_t nsteps, const double *data, double *u_out,
                               void *stream);

/* Source terms (Sec. 4.1): (1/c^2) u_tt = lap u + S with a separable source
 * S(x, t) = g(x) f(t), zero initial velocity, P = 1 or 2.  P = 1 adds
 * (c dt)^2 S^n to each step; P = 2 is the fourth-order scheme,
 * + (c dt)^2 (S^{n+1} + 10 S^n + S^{n-1}) / 12 - beta^2 (c dt)^2 C[S^n] / 12,
 * C the ADI operator of eq. C_def_ADI (the printed scale of the C[S] term is
 * dimensionally inconsistent; this is the one the Taylor expansion gives).
 * The start takes f(t_{-1}) = f(t_1).  u0, g: device float64 fields of the
 * grid; u_out: device float64, receives u^nsteps; f: HOST float64,
 * nsteps + 1 values f(t_k) = f(k dt).  Direct launches (no graph); C[g] is
 * formed once per call with mol_apply_D (it uses the handle's levels).
 * MOL_EINVAL for P > 2 or NULL pointers. */
mol_status mol_solve_source(mol_handle h, const double *u0, int64_t nsteps, const double *g, const double *f,
                            double *u_out, void *stream);

/*
 * Gradient of a loss of the whole field history by checkpoint-and-recompute
 * (the paper has no adjoint; the discrete adjoint of the implemented forward
 * map, as mol_adjoint).
 *
 * J = sum_{n=0}^{nsteps} phi_n(u^n) over the forward run from u0 with zero
 * initial velocity (u^1 = u^0 + F u^0 / 2).  grad_fn(n, u_n, g_n, stream,
 * user) is called on the host for n = nsteps .. 0 (each n once, in that
 * order); u_n (device, float64, the grid's layout; packed for a batch) holds
 * u^n and must not be written; the function writes dphi_n/du^n into g_n
 * (device, float64, same layout) with work ordered on `stream` and returns 0,
 * or returns 1 when phi_n is absent (g_n is then not read); any other return
 * value aborts the call with MOL_EINVAL.
 *
 * The adjoint states obey mu^n = 2 mu^{n+1} - mu^{n+2} + F^T mu^{n+1} + g^n
 * (n = N .. 1, mu^{N+1} = mu^{N+2} = 0) and grad = mu^1 + F^T mu^1 / 2 -
 * mu^2 + g^0.  g^n needs u^n in reverse order: the forward pass keeps
 * (u^{c-1}, u^c) at c = 1, 1 + K, 1 + 2K, ... (K = checkpoint_every >= 1) and
 * the backward pass recomputes one segment of at most K states at a time
 * from its checkpoint on the device, holding 2 ceil(N/K) + K + 4 fields
 * (allocated for the call and freed before it returns).  grad: device,
 * float64.  Synchronous.  Errors: MOL_EINVAL (arguments, callback failure),
 * MOL_ENOMEM, MOL_ECUDA.
 */
typedef int (*mol_grad_fn)(int64_t n, const double *u_n, double *g_n, void *stream, void *user);
mol_status mol_adjoint_history(mol_handle h, const double *u0, int64_t nsteps, int64_t checkpoint_every,
                               mol_grad_fn grad_fn, void *user, double *grad, void *stream);

/*
 * Robustness (no counterpart in the paper).
 *
 * mol_field_norm: *norm = the discrete L2 norm (prod_a h_a * sum u^2)^(1/2) of
 * a device float64 field of the handle's grid (NaN or Inf propagate).
 * Synchronous on the stream.
 *
 * mol_step_checked: mol_step plus an instability check: the norm of u_cur is
 * taken before and after; MOL_EUNSTABLE if the field is no longer finite or
 * its norm grew by more than growth_limit (> 0) times (an A-stable run at
 * beta <= beta_max stays bounded, Sec. 3.1).  The fields hold the advanced
 * levels either way.  Synchronous.
 *
 * mol_checkpoint_write / mol_checkpoint_read: save and restore a run's state
 * -- the two levels u^{n-1}, u^n (device float64, caller-owned) and the step
 * index -- in a file with a header naming the problem (grid, c, dt, beta, P,
 * boundary condition, precision, quadrature) and a hash of the data.  Reading
 * refuses (MOL_EINVAL, with the reason) a file written for another problem, a
 * truncated file or data that do not match their hash.  Synchronous; the
 * stream orders the copies.
 */
mol_status mol_field_norm(mol_handle h, const double *u, double *norm, void *stream);

/* The level conversions of the mixed path (MOL_MIXED keeps each time level
 * as a pair of float32 planes, hi + lo): mol_pair_split sets hi[i] = x[i]
 * rounded to float32 (to nearest, ties to even) and lo[i] = (x[i] - hi[i])
 * rounded to float32; mol_pair_join sets x[i] = hi[i] + lo[i] evaluated in
 * float64.  n elements of caller-owned device memory (x float64, hi and lo
 * float32; 16-byte aligned buffers take the vectorised kernels); asynchronous
 * on the stream.  MOL_EINVAL for a NULL pointer or n < 0. */
mol_status mol_pair_split(const double *x, float *hi, float *lo, int64_t n, void *stream);
mol_status mol_pair_join(const float *hi, const float *lo, double *x, int64_t n, void *stream);
mol_status mol_step_checked(mol_handle h, double *u_prev, double *u_cur, int64_t nsteps, double growth_limit,
                            void *stream);
mol_status mol_checkpoint_write(mol_handle h, const char *path, const double *u_prev, const double *u_cur,
                                int64_t step, void *stream);
mol_status mol_checkpoint_read(mol_handle h, const char *path, double *u_prev, double *u_cur, int64_t *step,
                               void *stream);

/*
 * Test hooks (no counterpart in the paper).
 *
 * mol_wait_selftest: launches one CTA whose bounded wait (the same code as the
 * tile-copy barriers) cannot succeed, with a limit of limit_cycles SM cycles
 * (1 .. 2^40), and synchronizes.  Returns MOL_ETIMEOUT when the wait gave up
 * and raised the device flag, as it must; the GPU context stays usable.
 *
 * mol_debug_fail_alloc(after): the next `after` device allocations of the
 * library succeed and every one after them fails as if the device were full
 * (MOL_ENOMEM from the creating call, with everything it had allocated freed);
 * after < 0 switches the injection off.  Process-wide.
 *
 * mol_debug_allow_unstable(on): with on != 0, mol_create accepts beta above
 * beta_max(P) (to exercise the instability check); 0 restores the refusal.
 * Process-wide.
 */
mol_status mol_wait_selftest(int64_t limit_cycles, void *stream);
void mol_debug_fail_alloc(int64_t after);
void mol_debug_allow_unstable(int on);

/*
 * Measurement of a design alternative (the paper has no counterpart): the
 * chunk-local causal recurrence of a strided sweep, y_i = d y_{i-1} + q_i on
 * 32-point chunks with zero inflow (Sec. 2), over an nrows x ncols float32
 * field (multiples of 32; chunks along the rows, seeded uniform q), computed
 * [0] by the in-register scan of the pass kernels and [1] as the product with
 * the 32 x 32 lower-triangular Toeplitz matrix d^(i-j) on the tensor cores
 * (mma.sync m16n8k8 TF32, operands split into head and tail: three products).
 * ms_per_launch[v] = mean CUDA-event time of `reps` launches of variant v
 * after three warm-ups; *max_rel_diff = max |y_1 - y_0| / max |y_1|.
 * Allocates and frees its own buffers; synchronous.  MOL_EINVAL for sizes
 * that are not multiples of 32, d outside (0, 1) or reps < 1.
 */
mol_status mol_toeplitz_experiment(int nrows, int ncols, double d, int reps, double ms_per_launch[2],
                                   double *max_rel_diff, void *stream);

/* Synchronize the stream and report device-side failures: MOL_ECUDA for a
 * CUDA error, MOL_ETIMEOUT when a bounded wait inside a kernel (the strided
 * pass's tile-copy barrier, MOL_TUNE_STRIDED_STAGE 1 or 3) gave up since the
 * last mol_sync -- the results computed since then are not valid.  The wait
 * limit is about two seconds, far beyond any healthy copy. */
mol_status mol_sync(mol_handle h, void *stream);

/* Number of kernel launches this handle issued so far (all entry points). */
int64_t mol_launch_count(mol_handle h);

/*
 * Per-pass timing, for benchmarks.  While enabled, mol_step launches every
 * pass directly (no graph) between two CUDA events on the caller's stream
 * and accumulates the device time of each pass.  Enabling (or re-enabling)
 * clears the totals.
 */
mol_status mol_set_pass_timing(mol_handle h, int enable);

/*
 * Device time of the passes timed since timing was enabled (synchronises
 * the streams used).  Index = axis of the pass (0 = x, the last pass of a
 * step; 1 = y; 2 = z): total_ms[a] = summed duration, launches[a] = count.
 * Arrays of length 3.
 */
mol_status mol_pass_times(mol_handle h, double total_ms[3], int64_t launches[3]);

/* ------------------------------------------------------------------------
 * Batches of independent 2D problems
 *
 * Many Dirichlet problems of uneven size stepped together: every pass runs
 * all problems in a few launches over flat work lists (the x pass one per
 * row-length class, over the rows; the y pass one per cluster size, a
 * cluster of CTAs per group of 32 columns), the launches of a pass running
 * concurrently on streams forked from the caller's and joined back into it;
 * mol_batch_step captures its time loop in a CUDA graph.  Problem i has its own grid
 * (ndim = 2, 3 <= n <= 1024 per axis), c, dt, beta and P; all share the
 * boundary condition (homogeneous Dirichlet only) and the precision.  Each
 * problem follows the same scheme as a single mol_create handle (eq.
 * update_P; Sec. 4, eq. Full_2D).
 *
 * Fields are PACKED float64 device arrays: problem after problem, each
 * C-contiguous (ny, nx) with x fastest; mol_batch_offsets gives where each
 * starts.  The library keeps the levels in its own padded layout.
 * ------------------------------------------------------------------------ */
typedef struct mol_batch_ctx *mol_batch;

/* grids, c, dt, P: arrays of nprob entries; beta may be NULL (beta_max(P_i)
 * for every problem) or hold entries <= 0 with the same meaning.  bc must
 * be MOL_BC_DIRICHLET.  opt as for mol_create (lines_per_block ignored). */
mol_status mol_batch_create(int nprob, const mol_grid *grids, const double *c, const double *dt,
                            const double *beta, const int *P, mol_bc bc, mol_prec prec,
                            const mol_options *opt, mol_batch *out);
mol_status mol_batch_destroy(mol_batch b);

/* Message of the last failed call on b (that of mol_last_error(NULL) if b is NULL). */
const char *mol_batch_last_error(mol_batch b);

/* offsets[0..nprob]: element offset of every problem in a packed field;
 * offsets[nprob] = the packed field's length. */
mol_status mol_batch_offsets(mol_batch b, int64_t *offsets);

/* F = F[u] for every problem (packed fields, may not overlap). */
mol_status mol_batch_apply_F(mol_batch b, const double *u, double *F, void *stream);

/* u1 = u0 + F[u0]/2 for every problem (zero initial velocity, Sec. 3.2). */
mol_status mol_batch_start(mol_batch b, const double *u0, double *u1, void *stream);

/* Advance every problem by nsteps in place; as mol_step. */
mol_status mol_batch_step(mol_batch b, double *u_prev, double *u_cur, int64_t nsteps, void *stream);

/* ---- adjoint (the paper has none): receivers and the gradient of a loss
 * of the receiver traces with respect to the initial field.
 *
 * Receivers are HOST arrays of packed-field indices (problem offset + y nx
 * + x).  The forward map is u^1 = u^0 + F u^0 / 2, u^{n+1} = 2 u^n - u^{n-1}
 * + F u^n; the traces are t[(n-1) nrec + r] = u^n[rec_r], n = 1..nsteps.
 * For a loss J(t) with tgrad[(n-1) nrec + r] = dJ/dt^n_r, the adjoint states
 * mu^n = dJ/du^n satisfy mu^N = g^N, mu^n = 2 mu^{n+1} - mu^{n+2} + F^T
 * mu^{n+1} + g^n (g^n = the trace gradients of step n added at the
 * receivers), and dJ/du^0 = mu^1 + F^T mu^1 / 2 - mu^2.  The scheme is
 * linear with fixed coefficients, so the adjoint needs no stored forward
 * level: only tgrad.  F^T = sum f_ij (D_x^T)^i (D_y^T)^j with the transposed
 * per-axis operators. */

/* out = F^T w for every problem (packed fields, may not overlap). */
mol_status mol_batch_apply_FT(mol_batch b, const double *w, double *out, void *stream);

/* One update on packed fields: un = ea u + eb up + ec Op(u) + add, Op = F
 * (transpose = 0) or F^T (transpose = 1); up is read only when eb != 0, add
 * may be NULL.  The building block of adjoints of general history losses
 * (one adjoint step: u = mu^{n+1}, up = mu^{n+2}, ea = 2, eb = -1, ec = 1,
 * F^T, add = dJ/du^n). */
mol_status mol_batch_update(mol_batch b, const double *u, const double *up, double *un, double ea, double eb,
                            double ec, int transpose, const double *add, void *stream);

/* traces (device, nsteps * nrec float64) of the forward run from u0 (packed,
 * device) with zero initial velocity. */
mol_status mol_batch_traces(mol_batch b, const double *u0, int nrec, const int64_t *rec, int64_t nsteps,
                            double *traces, void *stream);

/* grad (device, packed) = dJ/du^0 given tgrad (device, nsteps * nrec). */
mol_status mol_batch_adjoint(mol_batch b, int nrec, const int64_t *rec, int64_t nsteps, const double *tgrad,
                             double *grad, void *stream);

/* mol_adjoint_history for a batch (fields packed; grad_fn sees packed u_n
 * and writes packed g_n). */
mol_status mol_batch_adjoint_history(mol_batch b, const double *u0, int64_t nsteps, int64_t checkpoint_every,
                                     mol_grad_fn grad_fn, void *user, double *grad, void *stream);

/* End-to-end from HOST memory, as mol_solve_host: packed u0 (host float64)
 * in, u^{nsteps} of every problem out (host float64, packed).  Synchronous. */
mol_status mol_batch_solve_host(mol_batch b, const double *u0, double *u_out, int64_t nsteps, void *stream);

mol_status mol_batch_sync(mol_batch b, void *stream);
int64_t mol_batch_launch_count(mol_batch b);

/* Autotuner of a batch: times the x pass with 2, 4 and 8 warps per CTA for
 * each of its one-warp-per-row launches (rows of <= 256 points; rows of more
 * than 512 points, which are also timed split over the two warps of one CTA
 * per row; rows of 257..512 points always run split, 8-point segments, when
 * their buffers fit shared memory, else with the short rows), then the y pass
 * with each problem's columns on the fewest 4-warp CTAs whose segments cover
 * them, on twice as many, and with full carries only, on the batch's own
 * workspace, and keeps the fastest.  Synchronous; the caller's fields are not touched.
 * mol_batch_get_tuning: out[0], out[1] = warps per CTA of the two x launches
 * (out[1] = 0: the long rows run split, one CTA of two warps per row),
 * out[2] = y rule: bit 0 the segment length (0 smallest, 1 doubled), bit 1
 * set = full carries in every column; clear (the default) = the float32 y
 * pass exchanges once per sweep between neighbouring segments in the
 * problems where the decay over a segment is below 2^-30 and a column has
 * more than two segments; ms (may be NULL) = the tuned x and y pass times. */
mol_status mol_batch_autotune(mol_batch b, void *stream);
mol_status mol_batch_get_tuning(mol_batch b, int out[3], double ms[2]);
/* Sets the launch variants by hand, in the encoding of mol_batch_get_tuning:
 * x_warps_short, x_warps_long in {2, 4, 8} (x_warps_long 0: split long
 * rows), y_rule in {0, 1, 2, 3}.  MOL_EINVAL (nothing changed) for a value outside
 * those sets or one whose buffers exceed shared memory.  Synchronous. */
mol_status mol_batch_set_tuning(mol_batch b, int x_warps_short, int x_warps_long, int y_rule);

/* Per-pass CUDA-event timing as mol_set_pass_timing / mol_pass_times
 * (index 0 = x pass, 1 = y pass). */
mol_status mol_batch_set_pass_timing(mol_batch b, int enable);
mol_status mol_batch_pass_times(mol_batch b, double total_ms[3], int64_t launches[3]);

/* ------------------------------------------------------------------------
 * Embedded boundaries (Sec. 4.3: the ADI lines as "line objects")
 *
 * A 2D domain cut out of an nx x ny grid of spacing (hx, hy), x fastest.
 * Each grid line meets the domain in one interval: a line object made of the
 * interior grid nodes of the line (row j: x indices row_lo[j] .. row_hi[j];
 * none when row_lo[j] > row_hi[j]) and two boundary points off the grid, at
 * distance row_gap_lo[j] > 0 before the first interior node and row_gap_hi[j]
 * > 0 after the last; columns likewise (y indices col_lo[i] .. col_hi[i]).
 * The boundary points carry homogeneous Dirichlet data.  Rows and columns
 * must agree on which nodes are interior; a line object holds at most 2046
 * interior nodes.  The geometry arrays are HOST arrays, read at creation.
 *
 * L_gamma^{-1} on a line object (Sec. 2 with the boundary points as the line's
 * ends, Sec. 4.3): the increments integrate the quadratic through a node and
 * its two neighbours (one node inward at the ends; the boundary points are
 * nodes) exactly against the kernel over cells of their true length, the
 * recurrences decay by e^{-alpha dx} per cell, and A, B make the result
 * vanish at both boundary points.  The scheme is eq. (Full_2D) with C and D of
 * eqs. (C_def_ADI), (D_def_ADI) built from these operators, its terms formed
 * in the order of Table 3: on a curved domain the x and y operators do not
 * commute, so the order is part of the scheme.
 *
 * Fields: caller-owned device float64 arrays (ny, nx) that vanish outside the
 * domain (outputs vanish there too).  The library owns its tables and work
 * fields (P + 4 fields of nx ny doubles; mixed: P + 11 of floats) and frees
 * them in mol_embed_destroy.
 * Calls are asynchronous on the given stream; errors are returned statuses
 * (MOL_EINVAL arguments or geometry, MOL_EUNSTABLE beta above beta_max(P),
 * MOL_ENOMEM, MOL_ECUDA), text via mol_embed_last_error.
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t nx, ny;
    double hx, hy;
    const int64_t *row_lo, *row_hi;        /* ny entries */
    const double *row_gap_lo, *row_gap_hi; /* ny entries */
    const int64_t *col_lo, *col_hi;        /* nx entries */
    const double *col_gap_lo, *col_gap_hi; /* nx entries */
} mol_embed_geom;

typedef struct mol_embed_ctx *mol_embed;

/* alpha = beta / (c dt) (eq. L_def); beta <= 0 selects beta_max(P); P in 1..5.
 * prec MOL_FP64: float64 sweeps.  MOL_MIXED: float32 sweeps in the difference
 * form of D (the line object's rows 1 and N-1 with their own weights on the
 * second divided differences of the end triples), the time levels as
 * float32 pairs; the caller's fields stay float64 (converted once per call). */
mol_status mol_embed_create(const mol_embed_geom *g, double c, double dt, double beta, int P, mol_prec prec,
                            mol_embed *out);
mol_status mol_embed_destroy(mol_embed e);
/* Message of the last failed call on e (that of mol_last_error(NULL) if e is NULL). */
const char *mol_embed_last_error(mol_embed e);

/* w = L_gamma^{-1} v on every line object of axis 0 (x) or 1 (y). */
mol_status mol_embed_linv(mol_embed e, const double *v, double *w, int axis, void *stream);
/* F = F[u] (eq. Full_2D on the domain). */
mol_status mol_embed_apply_F(mol_embed e, const double *u, double *F, void *stream);
/* u1 = u0 + F[u0]/2 (zero initial velocity, Sec. 3.2). */
mol_status mol_embed_start(mol_embed e, const double *u0, double *u1, void *stream);
/* nsteps of u^{n+1} = 2 u^n - u^{n-1} + F[u^n]; (u_prev, u_cur) advance in place. */
mol_status mol_embed_step(mol_embed e, double *u_prev, double *u_cur, int64_t nsteps, void *stream);
/* End to end from HOST memory: u0 in, u^{nsteps} out (start, then steps).  Synchronous. */
mol_status mol_embed_solve_host(mol_embed e, const double *u0, double *u_out, int64_t nsteps, void *stream);
mol_status mol_embed_sync(mol_embed e, void *stream);
int64_t mol_embed_launch_count(mol_embed e);
/* Per-kind CUDA-event timing of the launches made while enabled: kind 0 =
 * x line-object sweeps, 1 = y sweeps, 2 = the linear combinations of F and
 * the level update.  mol_embed_pass_times synchronizes, returns the totals
 * since the last call and resets them. */
mol_status mol_embed_set_pass_timing(mol_embed e, int enable);
mol_status mol_embed_pass_times(mol_embed e, double total_ms[3], int64_t launches[3]);

/*
 * F = F[u] in float64 (the operator of eq. update_P / Full_2D, as
 * mol_apply_F on a MOL_FP64 handle) WITHOUT ALLOCATING: no handle, no
 * cudaMalloc / cudaFree or any other allocating routine.  The paper has no
 * counterpart; this serves callers that cannot allocate device memory where
 * they need F -- a process whose caching allocator already holds nearly all
 * of the device, or a loop that cannot afford cudaFree's device-wide
 * synchronisation.
 *
 * Scratch: the intermediate planes, the tables d^j and the Horner
 * coefficients live in one static device array of 32 MiB (32 << 20 bytes)
 * inside libmolt.  A call needs 512 + sum_a roundup32(n_a + 1) +
 * planes * roundup32(N) doubles, planes = 0 (1D), P (2D), 2P + 1 (3D),
 * N = the number of grid points; larger grids are rejected with MOL_EINVAL
 * and a message giving both sizes (2D, P = 3: up to about 1.39 M points).
 * Nothing in the array needs to start at zero: every word a call reads was
 * written earlier in the same call.
 *
 * Set-up: the first call on each device (with that device current) looks
 * up the array's address and sets the kernels' shared-memory limits; make
 * that first call before any stream capture.  First calls from several host
 * threads are serialised by a lock inside the library.
 *
 * Concurrency: the array is shared by all calls on a device.  Calls that
 * overlap in time on one device (different streams, or threads without
 * ordering) race on it and give wrong results; order them on one stream.
 *
 * grid, c, dt, beta (<= 0 selects beta_max(P)), P, bc and quad_order (1 or
 * 2) mean what they mean for mol_create; u, F: device float64 fields of the
 * grid's size, both on the CURRENT device (the kernels run there), whose
 * byte ranges must not intersect; stream: a stream of the current device
 * (NULL = legacy default).  Errors: MOL_EINVAL (arguments, size, a field on
 * another device, overlapping fields), MOL_EUNSTABLE (beta), MOL_ECUDA
 * (launch); text via mol_last_error(NULL).
 */
mol_status mol_apply_F_noalloc(const mol_grid *grid, double c, double dt, double beta, int P, mol_bc bc,
                               int quad_order, const double *u, double *F, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MOLT_H */
