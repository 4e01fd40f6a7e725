/*
 * teuk.h -- C ABI of libteuk, a GB300 (sm_103a) time stepper for the
 * mode-decomposed (2+1)-D Teukolsky equation of Khanna & McKennon,
 * "An exploration of CUDA and CBEA for a gravitational wave
 * source-modelling application" (arXiv:0909.4039), Sec. 2.
 *
 * What one step computes (all in hand-written CUDA kernels):
 *   - the first-order system d_t u + D d_{r*} u = S of Eqs. 9-12 for
 *     u = {Phi_R, Phi_I, Pi_R, Pi_I}, Pi = Phi_t + b Phi_{r*} (Eqs. 5-7),
 *     on a uniform r* grid (nodes, both ends included) times a cell-centred
 *     theta grid theta_j = (j + 1/2) pi / Ntheta;
 *   - TEUK_SCHEME_SPLIT (default): an implicit-explicit Strang splitting.
 *     The algebraic terms -L u - A u of S (angular operator with the pole
 *     potential, c_t, c_0) advance by two half-steps of the L-stable
 *     two-stage SDIRK method of order 2 (one complex tridiagonal solve in
 *     theta per r* row and stage); the two-step Lax-Wendroff update of
 *     Eqs. 13-14 carries the transport D and S = T - (M - D) d_{r*} u.
 *     TEUK_SCHEME_LITERAL evaluates all of S inside the Lax-Wendroff stages,
 *     as Eqs. 12-14 read literally; it is unstable at dt = dr* / 2 and is
 *     refused there unless allow_unstable is set;
 *   - the radial boundary rows Phi = Pi = 0 and the angular parity
 *     conditions of Sec. 2.2 (last paragraph);
 *   - the particle source T of Eq. 1 (which the paper does not print) as a
 *     Gaussian on a circular equatorial orbit, see teuk_set_source;
 *   - FP64 waveform extraction h_n = sum_j w_j Phi_{i_ext, j} every step.
 *
 * Conventions for every function:
 *   - returns TEUK_OK (0) or a positive TEUK_E_* code; no exception crosses
 *     the ABI; teuk_last_error(ctx) gives a message for the last failure;
 *   - device memory is owned by the caller.  The library allocates no
 *     device memory; ctx is a host object that only records pointers;
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy stream);
 *     calls that take a stream are asynchronous unless stated otherwise;
 *   - units G = c = 1; the mass M is set in the descriptor.
 */
#ifndef TEUK_H
#define TEUK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TEUK_OK 0
#define TEUK_E_INVAL 1      /* invalid argument or descriptor */
#define TEUK_E_CUDA 2       /* a CUDA runtime call failed */
#define TEUK_E_NONFINITE 3  /* a non-finite waveform sample was produced */
#define TEUK_E_UNSTABLE 4   /* radial Courant number > 1, or literal scheme past its bound */
#define TEUK_E_TIMEOUT 5    /* a bounded device wait on a tile copy gave up */
#define TEUK_E_STATE 6      /* call out of order (e.g. no context) */
#define TEUK_E_RANGE 7      /* requested waveform steps are not in the ring buffer */

/* precision of the evolved state and stencil arithmetic; coefficients,
 * time, source phase and extraction sums are generated in FP64 always */
#define TEUK_FP64 0
#define TEUK_FP32 1

#define TEUK_SCHEME_SPLIT 0
#define TEUK_SCHEME_LITERAL 1

/* largest number of r* rows the source patch may cover (9 sigma_r each side) */
#define TEUK_MAX_PATCH_ROWS 4096
/* largest Ntheta (one theta row of a tile must fit in shared memory) */
#define TEUK_MAX_NTHETA 1024

typedef struct teuk_grid_desc {
    int32_t s;              /* spin weight of Eq. 1 (|s| <= 2) */
    int32_t m;              /* azimuthal mode of Eq. 4 */
    double M;               /* black-hole mass (> 0) */
    double a;               /* spin parameter, 0 <= |a| < M */
    int64_t Nr;             /* r* nodes, >= 3; node i at rstar_min + i dr* */
    int64_t Ntheta;         /* theta cells, 1 .. TEUK_MAX_NTHETA */
    double rstar_min;       /* r* of node 0 */
    double rstar_max;       /* r* of node Nr-1 (> rstar_min) */
    double dt;              /* time step; <= 0 selects dt = dr* / 2 */
    double rstar_extract;   /* extraction radius; the nearest node is used */
    int32_t precision;      /* TEUK_FP64 or TEUK_FP32 */
    int32_t scheme;         /* TEUK_SCHEME_SPLIT or TEUK_SCHEME_LITERAL */
    int32_t allow_unstable; /* nonzero: accept the literal scheme past its bound */
    int32_t reserved;       /* must be 0 */
} teuk_grid_desc;

typedef struct teuk_ctx teuk_ctx;

/* Sizes of the three caller-owned device buffers for a descriptor.
 *   state_bytes:          two time levels of u, each [2][Nr][Ntheta]
 *                         complex values of the state precision
 *                         (plane 0 = Phi, plane 1 = Pi; theta fastest);
 *   coef_bytes:           FP64-generated coefficient tables, the Thomas
 *                         pivots of the implicit stages, the source patch,
 *                         weights, control words and a staging area;
 *   wave_bytes_per_step:  one ring-buffer slot: h_n (complex double) then
 *                         the extraction row Phi_{i_ext, .} (Ntheta complex
 *                         doubles).
 * Returns TEUK_E_INVAL for an invalid descriptor. */
int teuk_workspace_bytes(const teuk_grid_desc *desc, size_t *state_bytes,
                         size_t *coef_bytes, size_t *wave_bytes_per_step);

/* Validate the descriptor, record the buffers, generate the coefficient
 * tables in FP64 on the device (r(r*) by Newton's method on ln(r - r_+);
 * Eq. 2 integrated with the usual constant), zero the state at step 0, set
 * the default extraction weights and a zero source.  d_state, d_coef and
 * d_wave must be device pointers of at least the sizes given by
 * teuk_workspace_bytes, 256-byte aligned; wave_capacity >= 1 slots.
 * Synchronises the stream before returning.  Errors: TEUK_E_INVAL,
 * TEUK_E_UNSTABLE (radial Courant number max b dt/dr* > 1; literal scheme
 * past its bound without allow_unstable), TEUK_E_CUDA. */
int teuk_init_grid(const teuk_grid_desc *desc, void *d_state, void *d_coef,
                   void *d_wave, int64_t wave_capacity, void *stream,
                   teuk_ctx **out);

/* Source T of Eq. 1 for this mode (the slot the paper fills with the
 * particle source of its ref. [14]):
 *   T_m = A exp(-(r* - r0*)^2/(2 sigma_rstar^2) - (theta - pi/2)^2/(2 sigma_theta^2))
 *         exp(-i m Omega t),   A = amp_re + i amp_im,
 * entering the Pi rows as F = 4 pi (r^2 + a^2 cos^2 theta) Delta/(Sigma^2 r^3) T_m
 * (the right side of Eq. 1 after the division that gives Eq. 9).
 * r0 is the Boyer-Lindquist orbital radius (> r_+); Omega = NaN selects the
 * prograde Kepler frequency M^{1/2}/(r0^{3/2} + a M^{1/2}).  amp = 0
 * disables the source.  The Gaussian is sampled where it exceeds double
 * precision resolution (|r* - r0*| <= 9 sigma_rstar).  Synchronous.
 * Errors: TEUK_E_INVAL (sigma <= 0, r0 <= r_+, patch wider than
 * TEUK_MAX_PATCH_ROWS rows), TEUK_E_CUDA. */
int teuk_set_source(teuk_ctx *ctx, double amp_re, double amp_im, double r0,
                    double sigma_rstar, double sigma_theta, double Omega);

/* Extraction weights w_j (host array of Ntheta doubles).  NULL selects the
 * default: projection on Y = sin(theta/2)^{|m+s|} cos(theta/2)^{|m-s|} in
 * the measure sin theta dtheta, normalised so that sum_j w_j Y_j = 1.
 * Applies to samples taken after the call.  Synchronous: it first waits for
 * all work on the device (steps in flight on any stream read the weights),
 * then writes them. */
int teuk_set_weights(teuk_ctx *ctx, const double *w);

/* Replace the state by src, a [2][Nr][Ntheta] array of complex doubles
 * (re, im interleaved), host or device memory, and set the step counter to
 * `step` (>= 0).  This starts a new run: the error flags that
 * teuk_extract_waveform reports (TEUK_E_NONFINITE, TEUK_E_TIMEOUT) are
 * cleared.  Records the waveform sample of this state.  Asynchronous on
 * `stream` for device src; synchronous for host src. */
int teuk_set_state(teuk_ctx *ctx, const void *src, int64_t step, void *stream);

/* Copy the current state to dst ([2][Nr][Ntheta] complex doubles, host or
 * device memory) and its step number to *step (may be NULL).  Synchronous. */
int teuk_get_state(teuk_ctx *ctx, void *dst, int64_t *step, void *stream);

/* Where the current state lives in the caller's d_state buffer: its byte
 * offset (one of the two time levels), the level's size in bytes
 * ([2][Nr][Ntheta] complex values of the state precision, Phi plane then
 * Pi plane, theta fastest) and whether it holds the shifted split-scheme
 * state s_n = C_{dt/2}^{-1} u_n (1) or the physical u_n (0).  The caller may
 * read or overwrite rows of that level between steps, on the context's
 * stream, e.g. the halo rows of an r* slab of a larger grid (Sec. 4's
 * decomposition of the grid work); the next teuk_step reads them.  Any
 * pointer may be NULL. */
int teuk_state_level(const teuk_ctx *ctx, int64_t *offset_bytes, size_t *level_bytes, int *shifted);

/* Advance nsteps >= 0 time steps on `stream` (asynchronous).  The step
 * counter lives on the device as well, so the launches can be captured in
 * a CUDA graph; long runs replay a cached graph of a fixed chunk of steps.
 * Errors: TEUK_E_INVAL, TEUK_E_CUDA. */
int teuk_step(teuk_ctx *ctx, int64_t nsteps, void *stream);

/* Copy waveform samples of steps [first_step, first_step + count) to host
 * memory: h_out gets 2*count doubles (re, im), row_out (optional, NULL to
 * skip) gets 2*Ntheta*count doubles.  The steps must still be in the ring
 * buffer (the last wave_capacity recorded steps), else TEUK_E_RANGE.
 * Synchronises `stream` first.  Returns TEUK_E_TIMEOUT if a step since the
 * last teuk_init_grid / teuk_set_state gave up waiting for a tile copy (the
 * state is then not valid), else TEUK_E_NONFINITE if a sample taken since
 * then was non-finite. */
int teuk_extract_waveform(teuk_ctx *ctx, int64_t first_step, int64_t count,
                          double *h_out, double *row_out, void *stream);

/* Launch configuration of the split-scheme step kernel: r* rows per CTA
 * tile, threads per CTA, dynamic shared memory per CTA, and G, the threads
 * that share one theta row in the implicit solve.  Any pointer may be NULL. */
int teuk_tiling(const teuk_ctx *ctx, int *tile_rows, int *threads, size_t *smem_bytes, int *group);

/* Which split-scheme kernel steps the grid.  *persistent = 1: the
 * persistent kernel (one CTA per SM walks the tiles; a producer warp moves
 * them by TMA into two shared-memory buffers while *consumer_threads threads
 * compute, so tile loads and stores overlap the arithmetic); 2: the
 * pipelined kernel (two steps per launch; about two CTAs per SM walk the
 * tiles, each double-buffering them, so the copies of a CTA's next tile
 * land while the current one computes); 0: the tiled kernel (one CTA per
 * tile).  *grid is the number of CTAs per launch.
 * *steps_per_launch is 2 or 3 when the tiled kernel advances that many
 * time steps per launch (temporal blocking: as many halo rows on either
 * side, one state read and write per launch), else 1.  Any pointer may be
 * NULL.  For the literal scheme *persistent = 0 and *steps_per_launch = 1. */
int teuk_kernel_config(const teuk_ctx *ctx, int *persistent, int *consumer_threads, int *grid,
                       int *steps_per_launch);

/* Measured tile autotuner.  Ranks the launch configurations that fit on the
 * device (tile heights of the tiled kernel with one or two steps per launch,
 * the pipelined kernel, and tile height x consumer count of the persistent
 * kernel) by a wave-quantisation cost model, times the best four of each
 * kind, and the tiled kernel with three steps per launch at the heights of
 * the four two-step candidates, for
 * trial_steps launches each on this grid (CUDA events on `stream`), in two
 * interleaved rounds, and keeps the fastest per time step (a candidate's
 * better round).  The trials overwrite the
 * state: afterwards the field is zero at step 0 and the waveform ring buffer
 * is empty (the source and weights are kept).  Call it right after
 * teuk_init_grid / teuk_set_source.  Synchronous.  *tile_rows_out (may be
 * NULL) receives the chosen tile height. */
int teuk_autotune(teuk_ctx *ctx, int trial_steps, void *stream, int *tile_rows_out);

/* teuk_autotune for steps that start from a cold L2 (state larger than L2,
 * or a caller that evicts it between steps): before every timed trial step
 * the caller-owned device buffer d_flush (flush_bytes, larger than the L2)
 * is overwritten, outside the timed interval, and a round's score is the
 * median of the single-launch times per step.  Same outcome otherwise. */
int teuk_autotune_cold(teuk_ctx *ctx, int trial_steps, void *d_flush, size_t flush_bytes, void *stream,
                       int *tile_rows_out);

/* Select the tiled split-scheme kernel with the given tile height (r*
 * output rows per CTA) by hand; TEUK_E_INVAL if such a tile does not fit in
 * shared memory.  The result of a step depends on neither the kernel nor
 * the tile height. */
int teuk_set_tiling(teuk_ctx *ctx, int tile_rows);

/* Select the tiled split-scheme kernel with the given tile height and
 * steps_per_launch = 1 (as teuk_set_tiling), 2 or 3 (that many time steps
 * per launch; the first step of a run and the steps left over at the end of
 * a call still take one each).  The result does not depend on the choice.
 * TEUK_E_INVAL if the tile does not fit, tile_rows is above 254 - 2
 * steps_per_launch, or steps_per_launch is not 1, 2 or 3. */
int teuk_set_tiling_steps(teuk_ctx *ctx, int tile_rows, int steps_per_launch);

/* Select the pipelined split-scheme kernel (two time steps per launch,
 * persistent CTAs of `threads` threads, 256 or 512, double-buffered tiles;
 * see teuk_kernel_config) with the given tile height.  The first step of a
 * run and an odd last step take the one-step tiled kernel at the same
 * height.  The result does not depend on the choice.  TEUK_E_INVAL if the
 * rows are not 16-byte multiples (Ntheta odd in FP32), two tile buffers do
 * not fit in shared memory, or the CTA does not fit an SM (512 threads:
 * Ntheta <= 256 and the FP32 state only in practice). */
int teuk_set_pipelined(teuk_ctx *ctx, int tile_rows, int threads);

/* Select the persistent split-scheme kernel with the given tile height and
 * consumer_threads in {384, 480}.  It exists for the FP32 state with
 * Ntheta <= 128 whose theta rows are 16-byte multiples; TEUK_E_INVAL
 * otherwise, or if the two tile buffers do not fit in shared memory. */
int teuk_set_persistent(teuk_ctx *ctx, int tile_rows, int consumer_threads);

/* Bound of the waits of the tiled split-scheme kernels on their state
 * copies, for testing the failure path without a fault: rounds >= 0 limits
 * each tile's waits on its state tile to that many mbarrier try_wait rounds
 * (0: give up at once); rounds < 0 restores the default bound (about four
 * million rounds, far longer than any copy takes).  A tile whose wait gives
 * up records TEUK_E_TIMEOUT in the context's control block, then waits for
 * its own copies with the default bound (so none is in flight when it
 * exits) and returns without writing its output rows.  teuk_extract_waveform
 * then returns TEUK_E_TIMEOUT; teuk_set_state clears it and the context
 * steps normally again.  Drops the context's captured graphs. */
int teuk_set_wait_limit(teuk_ctx *ctx, int rounds);

/* One literal-scheme step (all of S inside the two Lax-Wendroff stages)
 * that allocates nothing and needs no caller-allocated scratch.  The paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate device memory at the point where they step -- for example code
 * running while a framework's caching allocator has claimed the device
 * memory, or a latency-critical loop in which cudaMalloc/cudaFree, which
 * synchronise the device, are not allowed.  It computes what teuk_step
 * computes for a TEUK_SCHEME_LITERAL context, but keeps the midpoint
 * scratch in a fixed array inside the library's device image (8 MiB,
 * resident on every GPU that loads the library until the process exits)
 * instead of the caller's coefficient workspace.
 *   ctx    a context created with TEUK_SCHEME_LITERAL (its tables and source
 *          are read, its state, step counter and waveform are not touched);
 *   d_in   device buffer, [2][Nr][Ntheta] complex values of the context's
 *          state precision (plane 0 Phi, plane 1 Pi); read only;
 *   d_out  device buffer of the same shape; written.  It must not overlap
 *          d_in in any byte (the kernels write d_out while others still
 *          read d_in): overlapping ranges are refused with TEUK_E_INVAL;
 *   n      step index of d_in (the source phase uses t = n dt).
 * Grids whose midpoints need more than 8 MiB (2 (Nr-1) Ntheta complex
 * values) are rejected with TEUK_E_INVAL before anything is launched.  The
 * first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array: calls whose
 * work overlaps on the GPU race on it.  Nothing in it needs to start at
 * zero (every midpoint is written before it is read).  Asynchronous on
 * `stream`. */
int teuk_literal_step_static(const teuk_ctx *ctx, const void *d_in, void *d_out, int64_t n, void *stream);

/* FMA throughput of the current device, the ceiling of an ALU-bound step
 * kernel (the FP64 path is bound by the FP64 pipe: the paper requires double
 * precision for these evolutions, Sec. 4 and Sec. 5.2).  Runs 8 independent
 * FMA chains per thread, 256 threads per CTA, 8 CTAs per SM, `iters` rounds
 * (>= 1), timed with CUDA events on `stream`, and writes the rate in flop/s
 * (two per FMA) to *flops_per_s.  d_sink: caller-owned device memory of
 * 8 bytes (written only in an impossible case; it keeps the loop alive).
 * precision: TEUK_FP64 or TEUK_FP32.  Synchronous.  Errors: TEUK_E_INVAL,
 * TEUK_E_CUDA. */
int teuk_fma_rate(int precision, int iters, void *d_sink, void *stream, double *flops_per_s);

/* Current step number (host mirror of the device counter). */
int64_t teuk_current_step(const teuk_ctx *ctx);

/* Message of the last error on ctx (or of the last failed init if ctx is
 * NULL).  The string is owned by the library. */
const char *teuk_last_error(const teuk_ctx *ctx);

/* Human-readable name of a status code. */
const char *teuk_status_string(int status);

/* Release the host context (the caller frees its device buffers). */
int teuk_destroy(teuk_ctx *ctx);

/* ------------------------------------------------- operator and adjoint
 * The step as an operator on caller buffers, and its Hermitian adjoint (for
 * the inner product <x, y> = Re sum conj(x) y over both planes), for
 * gradients of waveform losses.  Split scheme only.  With s_n the internal
 * state (u_n = C_{dt/2} s_n the physical one, Sec. 2.2 split as described
 * for teuk_step):
 *   s_1 = M_0(u_0) = LW_0 C_{dt/2} u_0,   s_{n+1} = M_n(s_n) = LW_n C_dt s_n,
 *   h_0 = E u_0,  h_n = E C_{dt/2} s_n,   E u = sum_j w_j Phi_{i_ext, j}.
 * LW_n is affine (the source at t_n and t_n + dt/2); C_h is linear.  All
 * buffers are device memory of [2][Nr][Ntheta] complex in the context's
 * state precision, distinct from each other and from the context's own.
 * The context's state, step counter and waveform are not touched.  All
 * calls are asynchronous on `stream`. */

/* d_out = M_n(d_in) (first = 1: the first step from a physical state). */
int teuk_apply_step(teuk_ctx *ctx, const void *d_in, void *d_out, int64_t n, int first, void *stream);

/* teuk_apply_step that also writes the sample E C_{dt/2} d_out of its
 * output state to d_h (one complex double, device), in the same launch;
 * bit for bit what teuk_apply_sample(d_out, physical = 0) writes.  d_h must
 * not overlap d_in or d_out.  NULL d_h: TEUK_E_INVAL. */
int teuk_apply_step_sample(teuk_ctx *ctx, const void *d_in, void *d_out, int64_t n, int first, void *d_h,
                           void *stream);

/* One waveform sample into d_h (one complex double, device): E d_s if
 * physical, else E C_{dt/2} d_s; the same FP64 sum the steps write. */
int teuk_apply_sample(teuk_ctx *ctx, const void *d_s, int physical, void *d_h, void *stream);

/* Device workspace of teuk_adjoint_step, teuk_adjoint_step_spin and
 * teuk_dot, in *bytes (256-byte aligned, caller-owned).  Its first eight
 * doubles accumulate the parameter derivatives (see teuk_adjoint_step and
 * teuk_adjoint_step_spin); zero them before a backward sweep.  In FP64 its
 * tail holds the coefficient planes teuk_adjoint_prepare writes (for an
 * Nr x Ntheta grid 17 Nr Ntheta + 8 (2 Nr - 1) Ntheta doubles). */
int teuk_adjoint_workspace_bytes(const teuk_ctx *ctx, size_t *bytes);

/* Fills the workspace's coefficient planes for teuk_adjoint_step_spin (FP64
 * contexts; FP32 contexts form them in place and only record d_ws): the
 * coefficients of the full step's implicit stage and Lax-Wendroff stages
 * (Eqs. 13-14, the implicit reading of S) at every grid element, and their
 * exact spin derivatives, formed by the same device functions the step
 * uses (so the adjoint reads bit for bit the coefficients the forward step
 * forms).  Asynchronous on `stream`.  The
 * context remembers d_ws; teuk_adjoint_step_spin with another workspace
 * returns TEUK_E_STATE.  Keep the planes unmodified between the calls;
 * after writing over them (or after reusing the memory), call this again.
 * Errors: TEUK_E_INVAL for a NULL or unaligned d_ws. */
int teuk_adjoint_prepare(teuk_ctx *ctx, void *d_ws, void *stream);

/* One step of the backward (adjoint) sweep:
 *   d_lam_out = M_n^H d_lam_in + C_{dt/2}^H E^H g_n   (E^H g_0 if first),
 * where d_lam_in is the adjoint of s_{n+1}, d_lam_out that of s_n (of u_0
 * if first), and d_gseed points to g_n = dL/dRe h_n + i dL/dIm h_n (one
 * complex double on the device; NULL: no sample term).  The step's source
 * derivatives are added to the workspace accumulators acc[0..3]:
 *   dL/dRe A = acc[0],  dL/dIm A = -acc[1],  dL/dr0 = acc[2]
 * (A the source amplitude, r0 the orbit radius through r0* and the Kepler
 * frequency; sum over the backward sweep, in a fixed order).  In FP64, full
 * steps (first = 0) with the workspace last passed to teuk_adjoint_prepare
 * read its coefficient planes (the same results up to rounding; the FP64
 * pipe bounds this step); otherwise the coefficients are formed in place. */
int teuk_adjoint_step(teuk_ctx *ctx, const void *d_lam_in, void *d_lam_out, int64_t n, int first,
                      const void *d_gseed, void *d_ws, void *stream);

/* teuk_adjoint_step together with the step's part of the spin derivative:
 * the same lam_n and source accumulators, plus
 *   acc[4] += Re <lam_{n+1}, dM_n/da s_n> + Re <g_n, d(E C_{dt/2})/da s_n>
 * (the second term for n >= 1 with d_gseed), so that after a backward sweep
 * dL/da = acc[4].  d_s holds s_n, the state the step took (u_0 if first),
 * in the same layout; it is read only.  The spin a enters every coefficient
 * of Eq. 1 after Eqs. 2-4 (through r(r*; a), Delta and Sigma^2 of Eq. 7),
 * the source prefactor, the orbit's r0*(a) and Kepler frequency.  The
 * contraction uses exact derivatives of the FP64 coefficient tables
 * (forward-mode, r(r*; a) by implicit differentiation of Eq. 2) with the
 * forward stage values the kernel recomputes from s_n: no extra step
 * applications.  Zero acc[4] (with acc[0..3]) before a sweep.  Full steps
 * read the coefficient planes: d_ws must be the workspace last passed to
 * teuk_adjoint_prepare (else TEUK_E_STATE). */
int teuk_adjoint_step_spin(teuk_ctx *ctx, const void *d_lam_in, void *d_lam_out, const void *d_s, int64_t n,
                           int first, const void *d_gseed, void *d_ws, void *stream);

/* The forward tape: what teuk_apply_step_tape records of one step so that
 * teuk_adjoint_step_tape need not recompute it.  *bytes = the size of one
 * step's record (a multiple of 256): the first SDIRK2 stage value U1 and
 * the implicit stage's output U2 = C_h s_n of every row, each [2][Nr][Ntheta]
 * complex in the state precision, then the input's extraction row. */
int teuk_tape_bytes(const teuk_ctx *ctx, size_t *bytes);

/* teuk_apply_step_sample that also writes the step's record to d_tape
 * (device, 256-byte aligned, teuk_tape_bytes long, not overlapping the other
 * buffers).  The state and sample are bit for bit those of
 * teuk_apply_step_sample. */
int teuk_apply_step_tape(teuk_ctx *ctx, const void *d_in, void *d_out, int64_t n, int first, void *d_h,
                         void *d_tape, void *stream);

/* teuk_adjoint_step_spin with the forward stage values read from the
 * record teuk_apply_step_tape wrote for step n (same n and first) instead
 * of recomputed from s_n: the same lam_n and accumulators, bit for bit.
 * The record costs two states per step of device memory; keeping one per
 * step (a store-all forward run) removes both the checkpoint recompute and
 * the stage recompute from a backward sweep. */
int teuk_adjoint_step_tape(teuk_ctx *ctx, const void *d_lam_in, void *d_lam_out, const void *d_tape, int64_t n,
                           int first, const void *d_gseed, void *d_ws, void *stream);

/* d_out (one complex double, device) = sum conj(x) (y - z) over both
 * planes (z may be NULL: sum conj(x) y), in FP64 and a fixed order; the
 * difference is taken in FP64.  d_ws: the adjoint workspace. */
int teuk_dot(teuk_ctx *ctx, const void *d_x, const void *d_y, const void *d_z, void *d_ws, void *d_out,
             void *stream);

/* ---------------------------------------------------------------- batches
 * Many independent instances -- each a split-scheme context with its own
 * grid, spin, mode, source and buffers -- advanced together: one launch
 * covers every tile of every instance (a flattened tile list of
 * (instance, tile) entries) for one or two time steps, and long runs
 * replay a captured CUDA graph.
 * This is the data-parallel decomposition of the method over independent
 * problems (Sec. 4); each instance computes exactly what teuk_step computes
 * for it alone.  Instances must share the state precision and the theta
 * segment class (Ntheta <= 128, <= 256 or <= 1024).  The batch holds
 * pointers to the contexts, which must outlive it.  Every teuk_batch_step
 * reads each instance's current level, step and phase, so between batched
 * steps an instance may still be set, read, extracted or stepped alone. */
typedef struct teuk_batch teuk_batch;

/* Device workspace for a batch of `count` contexts (parameter tables and the
 * tile list), in *bytes.  TEUK_E_INVAL for a NULL context or count < 1. */
int teuk_batch_workspace_bytes(teuk_ctx *const *ctxs, int count, size_t *bytes);

/* Group contexts into a batch.  d_ws: caller-owned device memory of at
 * least teuk_batch_workspace_bytes, 256-byte aligned, for the lifetime of
 * the batch.  Steps per launch start at 2 where the kernel offers it
 * (Ntheta <= 256), else 1; tile heights start from a shared-memory model
 * (whole implicit passes, two CTAs per SM); teuk_batch_autotune measures
 * both.
 * TEUK_E_INVAL for mixed precision or segment class, a literal-scheme or
 * repeated context.  Synchronous (uploads the tile list). */
int teuk_batch_create(teuk_ctx *const *ctxs, int count, void *d_ws, size_t ws_bytes, teuk_batch **out);

/* Advance every instance by nsteps (instances whose state is physical take
 * the half implicit step first, as teuk_step does; with two steps per
 * launch an odd remainder takes a one-step launch).  Asynchronous on
 * `stream`; with a non-default stream and nsteps >= 128 chunks of 64 steps
 * replay one captured graph.  Work queued for an instance on another stream
 * (teuk_set_state, teuk_step) must be ordered before this call by the caller
 * (an event the stream waits on), and later work on other streams after it. */
int teuk_batch_step(teuk_batch *batch, int64_t nsteps, void *stream);

/* Tile height per instance (tile_rows: count entries), number of CTAs per
 * step and dynamic shared memory per CTA.  Any pointer may be NULL. */
int teuk_batch_tiling(const teuk_batch *batch, int *tile_rows, int *total_tiles, size_t *smem_bytes);

/* Set the tile height of every instance (count entries in [1, 254]);
 * TEUK_E_INVAL (and the previous tiling kept) if a tile does not fit. */
int teuk_batch_set_tiling(teuk_batch *batch, const int *tile_rows);

/* Time steps per launch: 1, or 2 (tiles carry two halo rows a side, both
 * steps run on them; Ntheta <= 256).  Results are bit for bit those of
 * single steps.  Setting it keeps the tile heights; TEUK_E_INVAL (and the
 * previous value kept) if 2 is unavailable or a tile no longer fits. */
int teuk_batch_steps_per_launch(const teuk_batch *batch, int *steps_per_launch);
int teuk_batch_set_steps_per_launch(teuk_batch *batch, int steps_per_launch);

/* Measured configuration: for each number of steps per launch the kernel
 * offers, a coordinate descent over the batch's Ntheta classes, each class
 * trying every whole number of implicit passes per tile that fits, timed
 * over trial_steps batched launches (CUDA events on `stream`); the faster
 * result per time step is kept.
 * The trials overwrite the states: afterwards every instance is zero at
 * step 0 with an empty waveform buffer (sources and weights kept).
 * Synchronous. */
int teuk_batch_autotune(teuk_batch *batch, int trial_steps, void *stream);

/* Message of the last error on the batch (or of the last failed create if
 * batch is NULL). */
const char *teuk_batch_last_error(const teuk_batch *batch);

/* Release the batch (not its contexts or workspace). */
int teuk_batch_destroy(teuk_batch *batch);

#ifdef __cplusplus
}
#endif
#endif
