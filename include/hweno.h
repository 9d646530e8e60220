/*
 * hweno.h -- C ABI of the GB300 (sm_103a) implementation of the moment-based
 * multi-resolution HWENO scheme of J. Li, C.-W. Shu and J. Qiu,
 * "Moment-based multi-resolution HWENO scheme for hyperbolic conservation
 * laws" (arXiv 2201.12193).  Section, equation and table names below are the
 * paper's.
 *
 * What one step computes (Sec. 2.1 for 1D, Sec. 2.2 for 2D): for every cell
 * and every conserved variable, point values at the Gauss-Lobatto points are
 * reconstructed from the zeroth and first moments of the 3-cell / 3x3-cell
 * stencil (Step 1: nested central polynomials q_1..q_4, WENO-Z weights of
 * eq. (non-linear-weight) with any positive linear weights); troubled cells
 * are found with the KXRCF indicator (eq. (KXRCF) / (KXRCF_)) and their first
 * moments replaced by eq. (vi) (Step 2); HLLC (Euler, eq. (f_HLLC)) or local
 * Lax-Friedrichs (scalar laws) fluxes and the Gauss-Lobatto quadratures of
 * eq. (F) / (integral1)-(integral3) give L(U) of eq. (1D-equ-int-approximation)
 * / (2D-equ-int-approximation), advanced by the SSP Runge-Kutta method of
 * eq. (Runge-Kutta) (Step 3).
 *
 * State layout everywhere: FP64 m[var][moment][j][i], contiguous in i, no
 * padding, j of size 1 in 1D.  Variables: (u) for scalar laws; (rho, rho*mu, E)
 * for 1D Euler; (rho, rho*mu, rho*nu, E) for 2D Euler.  Moments (eq. (1D-moment)
 * / (2D-moment)): 0 = cell average, 1 = first moment in x ((x-x_i)/dx
 * weighted), 2 = first moment in y (2D only).  count arguments are element
 * counts nvar * nmom * ny * nx and must match exactly.
 *
 * Ownership: the library allocates and frees all device memory it uses for a
 * handle; every pointer passed in belongs to the caller.  Device pointers
 * must be on the handle's device.  Errors never cross the ABI as exceptions:
 * each call returns an hweno_status and hweno_last_error() describes it.
 * A handle is not thread-safe; use one handle per host thread.
 *
 * Streams: work is enqueued on the handle's stream (hweno_set_stream; default
 * the legacy default stream).  hweno_step is asynchronous.  hweno_max_dt,
 * hweno_get_moments (host destination), hweno_troubled_mask, hweno_totals and
 * hweno_sync synchronise the stream; they also report a non-physical state
 * left by the last step (HWENO_ENONPHYSICAL), after which the state has been
 * rolled back to the one before that step.
 */
#ifndef HWENO_H
#define HWENO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hweno_s* hweno_t;

typedef enum {
  HWENO_OK = 0,
  HWENO_EINVAL = -1,        /* bad argument (size, pointer, grid, count) */
  HWENO_ECUDA = -2,         /* a CUDA runtime call failed */
  HWENO_ENONPHYSICAL = -3,  /* non-finite value, rho <= 0 or p <= 0 after a step */
  HWENO_ETIMEOUT = -4,      /* a bounded device wait gave up */
  HWENO_ESTATE = -5,        /* call out of order (e.g. no moments set) */
  HWENO_ENOMEM = -6         /* device allocation failed */
} hweno_status;

typedef enum { HWENO_ADVECTION = 0, HWENO_BURGERS = 1, HWENO_EULER = 2 } hweno_eq;
typedef enum {
  HWENO_BC_PERIODIC = 0, HWENO_BC_TRANSMISSIVE = 1, HWENO_BC_REFLECTIVE = 2, HWENO_BC_INFLOW = 3
} hweno_bc_kind;
typedef enum {
  HWENO_IND_NONE = 0, HWENO_IND_KXRCF = 1, HWENO_IND_ALL = 2, HWENO_IND_MLP = 3, HWENO_IND_TVB = 4
} hweno_indicator;

/* Uniform mesh and scheme options.
 *   dim 1 or 2; nx, ny >= 4 (ny ignored in 1D); 2D cells must be square
 *   (dx == dy to 1e-12 relative) because the smoothness indicators of
 *   eq. (2D-beta), eq. (2D-beta1) and h of eq. (KXRCF_) are stated for them.
 *   eq: advection (f = adv_a u, g = adv_b u), Burgers (f = g = u^2/2) or Euler.
 *   precision: 0 = FP64 throughout; 1 = FP32 reconstruction, indicator, flux
 *   and quadrature with FP64 state, FP64 Runge-Kutta accumulation and FP64
 *   differences of the face fluxes in the cell-average equation; 2 = the same
 *   split with double-float arithmetic (pairs of FP32 numbers, a 48-bit
 *   significand and FP32's exponent range; magnitudes below 2^-74 keep FP32
 *   precision) in place of FP32.
 *   indicator: HWENO_IND_KXRCF is the scheme (HWENO6-M5-I); NONE gives HWENO6
 *   (no modification); ALL gives HWENO6-M5-NI (every cell modified) (Sec. 3);
 *   MLP: the learned indicator with KXRCF fallback (see below; 2D Euler).
 *   TVB: the minmod-based TVB indicator of Remark 2 on the indicator variable
 *   (u, or rho for Euler), acting on the cell's linear polynomial of its
 *   moments: troubled when the modified minmod (identity for |a| <= tvb_m dx^2)
 *   changes a = 6 vbar (6 wbar in y), the polynomial's face deviation, against
 *   the forward and backward differences of the averages in that direction.
 *   gamma_bar: positive linear-weight seeds of eq. (linear-weight)
 *   (gamma_{l1,l2} = gamma_bar[l1-1] / sum_{l<=l2} gamma_bar[l-1]); the paper
 *   uses {1, 10, 100, 1000}.
 *   beta_of_q: 0 = smoothness indicators of p_l as eq. (beta) states (default);
 *   1 = of q_l (the variant for which Remark 1's expansion holds for every l).
 *   tvb_m: the TVB constant M (>= 0) of indicator TVB; ignored otherwise.
 *   charwise: 0 = reconstruct the conserved variables component by component
 *   (default); 1 = (1D Euler only) reconstruct in local characteristic
 *   variables: the stencil's moments projected on the eigenvectors of the flux
 *   Jacobian at the target cell's average, each field reconstructed by the
 *   scalar procedure, the point values mapped back.  The paper does not say
 *   which; its blast-wave example needs the characteristic form here. */
typedef struct {
  int dim;
  int nx, ny;
  double x0, x1, y0, y1;
  int eq;
  double adv_a, adv_b;
  int precision;
  int indicator;
  double gamma_bar[4];
  int beta_of_q;
  double tvb_m;
  int charwise;
} hweno_grid;

/* Boundary kinds of the four sides.  Periodic sides must come in pairs.
 * Transmissive = the mirror image about the boundary face (the cell average
 * and the tangential first moment are copied, the normal first moment changes
 * sign); ghost cells are images of interior cells throughout a stage.
 * Reflective (Euler) = the transmissive image with the wall-normal momentum
 * negated.  Inflow (2D Euler, FP64, not with the learned indicator) = ghost
 * cells of fixed states set by hweno_set_fixed_state (the inflow and
 * post-shock boundaries of Sec. 3's double Mach reflection and forward step):
 * that cell average, zero first moments, the same value at every
 * Gauss-Lobatto point, never troubled.  In a corner the y side's rule applies
 * to the cell the x side's rule gives (a fixed y ghost wins; the y wall image
 * of a fixed x ghost negates its y momentum). */
typedef struct { int xlo, xhi, ylo, yhi; } hweno_bc;

/* Create a solver.  gamma: ratio of specific heats (Euler; ignored otherwise).
 * Allocates all device buffers on the current device.  Returns EINVAL for a bad
 * grid, ENOMEM if allocation fails.  *out is NULL on failure. */
hweno_status hweno_create(const hweno_grid* grid, const hweno_bc* bc, double gamma, hweno_t* out);

/* Release everything the handle owns (waits for its stream first). */
void hweno_destroy(hweno_t h);

/* Use cuda_stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream). */
hweno_status hweno_set_stream(hweno_t h, void* cuda_stream);

/* Copy moments in (on_device = 0: pageable or pinned host; 1: device pointer).
 * Sets the solution time to 0. */
hweno_status hweno_set_moments(hweno_t h, const double* m, size_t count, int on_device);

/* Fixed-state ghost cells of one side (0 x-lo, 1 x-hi, 2 y-lo, 3 y-hi) of a
 * single-problem 2D Euler FP64 handle.  With segment = 1, the ghost cells
 * whose centre coordinate along the side (y on the x sides, x on the y sides;
 * ghost cells one position beyond each end included) is below c0 + speed * t,
 * t the time of the stage input, hold the conserved state a; the other ghost
 * cells of an HWENO_BC_INFLOW side hold b, those of another kind follow that
 * kind.  An inflow side needs this call before the first step (else step,
 * advance and rhs return ESTATE); a segment may also sit on a transmissive or
 * reflective side (the double Mach reflection's floor: post-shock before the
 * wedge, wall after it).  States need rho > 0 and p > 0 (else EINVAL).  Stage
 * times are t, t + dt and t + dt/2; positions and thresholds are rounded as
 * written (no fused multiply-add). */
typedef struct {
  int segment;
  double c0, speed;
  double a[4];     /* (rho, rho u, rho v, E) inside the segment */
  double b[4];     /* (rho, rho u, rho v, E) elsewhere on an inflow side */
} hweno_fixed_state;
hweno_status hweno_set_fixed_state(hweno_t h, int side, const hweno_fixed_state* f);

/* Solution time of a single-problem handle (read by moving segments):
 * hweno_step advances it by dt (restored when a step is rolled back),
 * hweno_advance by the time it reached, hweno_set_moments resets it to 0. */
hweno_status hweno_set_time(hweno_t h, double t);
hweno_status hweno_get_time(hweno_t h, double* t);

/* Copy the current moments out (synchronises when the destination is host memory). */
hweno_status hweno_get_moments(hweno_t h, double* m, size_t count, int on_device);

/* One SSP-RK3 step of size dt (three stages, eq. (Runge-Kutta)); asynchronous.
 * Reading (default, hweno_set_persistence): the first moments modified in
 * troubled cells replace the stage input and enter the Runge-Kutta
 * combination. */
hweno_status hweno_step(hweno_t h, double dt);

/* Row-slab decomposition of one 2D grid (no counterpart in the paper: the
 * update of a cell in one stage depends on the stage input of the cells up to
 * 4 rows and columns away (moments -> point values -> troubled flags ->
 * re-reconstruction -> fluxes), so a slab that holds 4 halo rows on each
 * internal side, refilled from its neighbours before every stage, advances its
 * own rows exactly as the whole grid would).
 * hweno_set_owned_rows: the rows [jlo, jhi) this handle owns; only they enter
 *   the status checks, the CFL wave speeds and hweno_totals (default: all).
 * hweno_stage: stage k (0, 1, 2, in this order, the same dt) of one SSP-RK3
 *   step; the three stages equal hweno_step bit for bit.  Asynchronous.
 * hweno_copy_rows: rows [j0, j0 + nrows) of every (variable, moment) plane of
 *   the state the next stage reads (U^n before stage 0, U^(1), U^(2) between
 *   stages) to (to_state = 0) or from (1) the device buffer buf, laid out
 *   [nvar * nmom][nrows][nx].  Asynchronous on the handle's stream.
 * hweno_wave_speeds: max a_x, max a_y over the owned rows (the quantities of
 *   hweno_max_dt's rule, +inf for a non-physical average), host array of 2.
 *   Synchronises.
 * Single 2D handles (else ESTATE); EINVAL for rows out of range or a stage out
 * of order. */
hweno_status hweno_set_owned_rows(hweno_t h, int jlo, int jhi);
hweno_status hweno_stage(hweno_t h, int k, double dt);
hweno_status hweno_copy_rows(hweno_t h, int j0, int nrows, double* buf, int to_state);
hweno_status hweno_wave_speeds(hweno_t h, double* ax_ay);

/* dt for the next step from the cell averages (CFL rule of Sec. 3, formula not
 * printed there; reading): 1D dt = cfl dx / max(|f'|) or max(|mu| + c);
 * 2D dt = cfl / (max(a_x)/dx + max(a_y)/dy).  Synchronises. */
hweno_status hweno_max_dt(hweno_t h, double cfl, double* dt_out);

/* Troubled-cell flags of the three stages of the last step, [3][ny][nx] bytes
 * (0/1), host memory.  Synchronises. */
hweno_status hweno_troubled_mask(hweno_t h, unsigned char* mask, size_t count);

/* Conservation totals sum(ubar) * dx * dy per variable (FP64), host array of
 * nvar doubles.  Synchronises. */
hweno_status hweno_totals(hweno_t h, double* sums);

/* Wait for the handle's stream; report a non-physical last step. */
hweno_status hweno_sync(hweno_t h);

/* One evaluation of the spatial operator with the troubled-cell steps on a
 * caller-given state (all device pointers, state layout):
 *   U    in : stage input;
 *   Umod out: U with the first moments of troubled cells replaced (eq. (vi));
 *   L    out: L(Umod);
 *   mask out: troubled flags [ny][nx] bytes;
 *   aleph out (may be NULL): KXRCF values [ny][nx] doubles.
 * Asynchronous on the handle's stream. */
hweno_status hweno_rhs(hweno_t h, const double* U, double* Umod, double* L, unsigned char* mask, double* aleph);

/* ---------------------------------------------------------------- learned indicator
 * (no counterpart in the paper: a small network trained on the paper's KXRCF
 * decisions, with KXRCF kept as the fallback and the judge)
 * Network: 108 -> 64 -> 64 -> 1, GELU hidden units, sigmoid output; inputs are
 * the 3x3 neighbourhood of a cell: per variable and cell k (paper label order)
 * (ubar_k - ubar_c, vbar_k, wbar_k) / D, D = max |ubar_k - ubar_c| +
 * dx^2 max |ubar_k| + 1e-12, except that the centre's average slot holds
 * ubar_c / (max |ubar_k| + 1e-12); clipped to [-8, 8] (108 = 4 variables x
 * 3 moments x 9 cells, order var, moment, cell).
 * Parameters: FP32 flat W1[64][108], b1[64], W2[64][64], b2[64], W3[64], b3[1]
 * (hweno_mlp_nparam() floats).  The contractions run on BF16 tensor cores with
 * FP32 accumulation.
 *
 * Indicator 3 in hweno_grid (2D Euler; single-problem handles): at the start of
 * each stage every cell's probability s comes from the network on the stage
 * input.  Where the confidence max(s, 1-s) >= conf, the network decides the flag
 * (s > 1/2) and a flagged cell's first moments are modified (eq. (vi)) before
 * Step 1, which reconstructs it from the modified moments (so only cells flagged
 * by the fallback are reconstructed twice).  The other cells are decided by
 * KXRCF from the Step-1 point values, as indicator 1 does.  With conf > 1 every
 * cell falls back and the results equal indicator 1's bit for bit.
 * hweno_set_mlp installs the parameters (host or device pointer, copied) and
 * conf (> 0); HWENO_ESTATE if the handle's indicator is not 3; a step before
 * hweno_set_mlp fails with HWENO_ESTATE.  hweno_mlp_fallbacks returns and resets
 * the number of cell decisions left to KXRCF since the last call.
 * hweno_mlp_probe: a device array of ny*nx floats that every later stage fills
 * with the network's probabilities (row-major j*nx+i), or NULL to stop.
 * hweno_features: the 108 features (float, row per cell) of the given cells
 * (device int array, j*nx+i) of a caller state U (device, state layout).
 * Training (device pointers; asynchronous on stream): hweno_mlp_loss_grad adds
 * the gradient of the weighted mean binary cross-entropy over n samples to grad
 * and the loss to *loss (caller zeroes both); w may be NULL (weights 1).
 * hweno_mlp_adam: one Adam step (beta 0.9, 0.999, eps 1e-8), step counts from 1.
 * hweno_mlp_forward: probabilities of n feature rows. */
int hweno_mlp_nparam(void);
hweno_status hweno_set_mlp(hweno_t h, const float* params, int on_device, float conf);
hweno_status hweno_mlp_fallbacks(hweno_t h, long long* cells);
hweno_status hweno_mlp_probe(hweno_t h, float* prob);
hweno_status hweno_features(hweno_t h, const double* U, const int* cells, int n, float* X);
hweno_status hweno_mlp_forward(const float* params, const float* X, int n, float* prob, void* stream);
hweno_status hweno_mlp_loss_grad(const float* params, const float* X, const float* y, const float* w, int n,
                                 float* grad, float* loss, void* stream);
hweno_status hweno_mlp_adam(float* params, const float* grad, float* m1, float* m2, int step, float lr,
                            void* stream);

/* Advance by t_end (>= 0) with the CFL step length (cfl > 0, the rule of
 * hweno_max_dt) computed on the device each step, the last step clipped so that
 * the run ends at t_end exactly, at most max_steps steps.  The solution time
 * (hweno_get_time) advances with it; moving fixed-state segments read their
 * stage times on the device.  No CFL step length (rho <= 0 or a non-finite wave
 * speed) fails the call with ENONPHYSICAL whatever the positivity switch.  Steps run in groups
 * of 12 replayed from a CUDA graph (no host round trip per step); steps left
 * over in the last group once t_end or max_steps is reached are skipped (the
 * state passes through unchanged).  Writes the time reached and the steps taken
 * (either pointer may be NULL).  The result equals hweno_max_dt + hweno_step
 * driven from the host, bit for bit.  A non-physical state stops the call with
 * HWENO_ENONPHYSICAL and is not rolled back (several steps per replay);
 * hweno_troubled_mask afterwards holds the flags of the group's last step, which
 * may be a skipped one.  Single-problem handles; synchronises. */
hweno_status hweno_advance(hweno_t h, double t_end, double cfl, long long max_steps, double* t_done,
                           long long* steps_done);

/* Positivity check of hweno_step / hweno_step_batch (no counterpart in the
 * paper, which has no positivity treatment): on (default), a stage whose new
 * cell averages have rho <= 0 or p <= 0 (Euler) fails the step with
 * HWENO_ENONPHYSICAL and the state is rolled back; off, only non-finite values
 * fail it (transient negative pressures are carried on, as the scheme itself
 * does).  Applies to single and batch handles. */
hweno_status hweno_set_positivity_check(hweno_t h, int on);

/* Solid block (the forward-facing step of Sec. 3, Example 3.10; no rule for it
 * in the paper): cells with i >= i0 and j < j1 are solid, bounded by a
 * vertical wall face at i = i0 (when i0 > 0) and a horizontal one at j = j1
 * (when j1 < ny).  Reading: a solid cell in the stencil of a fluid cell is
 * that cell's wall image -- mirrored across the vertical face when the
 * viewing cell lies left of it, across the horizontal face when it lies
 * above it, across both (through the corner) for the cell diagonal to the
 * corner -- each crossed face negating its wall-normal momentum and normal
 * first moment; a face shared with a solid cell carries the
 * reflective wall flux of the fluid side's own values and is never a KXRCF
 * inflow face; solid cells are not reconstructed, flagged or updated (their
 * state passes through) and take no part in the CFL rule or the totals.
 * j1 = 0 removes the block.  Single 2D Euler FP64 handles without the learned
 * indicator or the fused stage (else ESTATE); EINVAL unless 0 <= i0 < nx,
 * 1 <= j1 <= ny, at least 4 fluid cells lie beyond each face and the sides
 * the block touches (the right one when i0 > 0, the bottom one when j1 < ny)
 * are not periodic. */
hweno_status hweno_set_solid(hweno_t h, int i0, int j1);

/* One fused kernel per Runge-Kutta stage (on = 1) instead of the pipeline of
 * four launches (on = 0).  2D (Sec. 2.2; off by default): Steps 1-3
 * (reconstruction, eq. (KXRCF_), eq. (vi), the troubled re-reconstruction,
 * HLLC fluxes, eqs. (integral1)-(integral3), L and eq. (Runge-Kutta)) for a
 * strip of cells in one block, the point values kept in shared memory; single
 * 2D Euler handles without a solid block; sides with fixed states
 * (hweno_set_fixed_state) keep the pipeline; boundary images enter as
 * ordinary cells, so cells next to a non-periodic side may differ from the
 * pipeline by rounding, elsewhere the two agree to rounding of the quadrature
 * sums.  1D (Sec. 2.1; ON by default): the same steps for a segment of cells
 * and a 4-cell halo in shared memory, bitwise the pipeline's states, masks,
 * KXRCF values and counts (scalar laws and Euler, every side kind and
 * precision); component-wise reconstruction only (charwise handles keep the
 * pipeline).  Both: the KXRCF, none or all indicator (else ESTATE; TVB and the
 * learned indicator keep the pipeline).  Applies to hweno_step, hweno_stage,
 * hweno_advance and hweno_rhs. */
hweno_status hweno_set_fused(hweno_t h, int on);

/* TMA staging of the FP32-bulk update (off by default): each interior 32 x 4
 * tile loads its own point values (64 planes) into shared memory with one
 * cp.async.bulk.tensor completing on an mbarrier (the wait is bounded: past the
 * limit the step reports HWENO_ETIMEOUT); the one-cell halo, the stage states
 * and the tiles at the grid's edges read global memory.  The arithmetic is the
 * same code either way, so results are bitwise the same with on = 0 or 1.  Off
 * by default because the global-memory kernel, at 8 resident blocks per SM,
 * measured faster than the staged one at the 4 its shared memory allows.
 * Single 2D Euler FP32-bulk handles (else ESTATE for on = 1); EINVAL unless on
 * is 0 or 1. */
hweno_status hweno_set_tma(hweno_t h, int on);

/* How the first moments modified by eq. (vi) in troubled cells (Step 2.2) are
 * used; the paper does not say.  persist = 1 (default): they replace the
 * stage input, so the Runge-Kutta combination of eq. (Runge-Kutta) takes them
 * (stage 1 also modifies U^n); this reproduces Table 1's HWENO6-M5-NI errors
 * (Sec. 3, Example 3.1).  persist = 0: they serve the evaluation of L only and
 * the combination takes the stage states as they entered the stage.
 * hweno_rhs is unaffected (its Umod output holds the modified moments either
 * way).  EINVAL for other values.  Single and batch handles. */
hweno_status hweno_set_persistence(hweno_t h, int persist);

/* Troubled re-reconstruction work (Step 2.3): the number of cells reconstructed
 * a second time, from modified moments, since the last call (then reset to 0).
 * Single-problem handles; synchronises the handle's stream.  No counterpart in
 * the paper: a work counter. */
hweno_status hweno_rerecon_count(hweno_t h, long long* cells);

/* ---------------------------------------------------------------- batches
 * Many independent 2D Euler problems of different sizes in one handle; every
 * problem is the scheme above on its own grid and boundary kinds.  One batched
 * step is one SSP-RK3 step of every problem, run as one persistent cooperative
 * launch per Runge-Kutta stage (all problems' cells and tiles form one work
 * list), captured in a CUDA graph and replayed.  Phases inside a launch are
 * separated by a grid barrier whose waits are bounded; a wait that gives up
 * sets HWENO_ETIMEOUT (reported by the next synchronising call, which rolls the
 * step back).  All grids must be dim 2, eq Euler, and share precision,
 * indicator, gamma_bar and beta_of_q; cells square per problem.
 *
 * hweno_create_batch: n problems (grids[k], bcs[k]).
 * hweno_batch_set_moments / get_moments: problem k's moments in the state
 *   layout (count = 12 ny nx); get with a host destination synchronises.
 * hweno_step_batch: dt_device = device array of n doubles (one dt per problem)
 *   or NULL: each problem takes its CFL dt (reading of Sec. 3, as
 *   hweno_max_dt) from its own cell averages, computed on the device.
 * hweno_batch_dt: the dt each problem used in the last step (host, n doubles).
 * hweno_batch_troubled_mask: problem k's flags of the last step [3][ny][nx].
 * hweno_batch_set_tile: update-phase tile shape 0: 32x4, 1: 16x8, 2: 64x2
 *   (results do not depend on it; an autotuner picks the fastest). */
hweno_status hweno_create_batch(const hweno_grid* grids, const hweno_bc* bcs, int n, double gamma, hweno_t* out);
hweno_status hweno_batch_set_moments(hweno_t h, int k, const double* m, size_t count, int on_device);
hweno_status hweno_batch_get_moments(hweno_t h, int k, double* m, size_t count, int on_device);
hweno_status hweno_step_batch(hweno_t h, const double* dt_device, double cfl);
hweno_status hweno_batch_dt(hweno_t h, double* dt, int n);
hweno_status hweno_batch_troubled_mask(hweno_t h, int k, unsigned char* mask, size_t count);
hweno_status hweno_batch_set_tile(hweno_t h, int variant);
/* Bound of the grid barrier's waits (no counterpart in the paper): a wait
 * gives up after spin_limit polls (64 ns sleeps each; default 2^26, seconds),
 * sets HWENO_ETIMEOUT for the next synchronising call (which rolls the step
 * back) and lets the block continue, so no wait can hang the GPU.
 * extra_arrivals (0 normally, at most 1024) makes every barrier wait for that
 * many arrivals beyond the launched blocks, so every wait runs out: the way to
 * exercise the timeout path without faulting anything.  Takes effect from the
 * next hweno_step_batch. */
hweno_status hweno_batch_set_barrier(hweno_t h, long long spin_limit, int extra_arrivals);
/* 1 if the last batched step was replayed from a captured CUDA graph, 0 if its
 * launches were issued directly (capture unavailable), -1 for a non-batch handle. */
int hweno_batch_uses_graph(hweno_t h);
/* Per-problem status bits of the last failure a synchronising call reported
 * (1 = non-finite value, 2 = rho <= 0 or p <= 0; 0 = fine), n entries. */
hweno_status hweno_batch_status(hweno_t h, unsigned* bits, int n);

/* Per-kernel timing (instrumentation; no counterpart in the paper).  With
 * enable != 0, every kernel launch of later steps is bracketed by CUDA events
 * on the handle's stream.  hweno_profile_read synchronises and writes, for the
 * first nkinds (>= 4) kernel kinds {0 reconstruct, 1 indicator + modification
 * (KXRCF, or its fallback pass after the learned indicator), 2 reconstruct
 * troubled cells, 3 fluxes + quadrature + Runge-Kutta update, 4 learned
 * indicator network pass, 5 fused stage}, the summed device milliseconds and launch counts
 * since the last read (kinds past nkinds are dropped; slots past the last kind
 * are zeroed). */
hweno_status hweno_profile(hweno_t h, int enable);
hweno_status hweno_profile_read(hweno_t h, double* ms, int* launches, int nkinds);

/* Arithmetic throughput probe (measurement only; no counterpart in the
 * paper): the fused multiply-add rate of the current device in FLOP/s
 * (precision 0 = FP64, 1 = FP32), from `iters` iterations of 8 independent
 * FMA chains per thread over 4 blocks of 256 threads per multiprocessor, timed
 * with CUDA events on cuda_stream after a warm-up launch; an FMA counts 2 flop.
 * The roofline denominator of the reconstruction kernels, which are bound by
 * FP64 (or FP32) arithmetic, not by memory.  Synchronises.  EINVAL for bad
 * arguments, ECUDA if a launch fails. */
hweno_status hweno_alu_probe(int precision, long long iters, double* flop_per_s, void* cuda_stream);

/* The kernels' double -> float rounding (FP32-bulk precision; no counterpart
 * in the paper): out[t] = in[t] rounded to the nearest float, ties to even, by
 * integer operations (no FP64 instruction) for results in the normal float
 * range, by the FP64 conversion otherwise.  Device pointers, n values,
 * asynchronous on cuda_stream.  A check hook: the tests compare it with the
 * FP64 conversion bit for bit. */
hweno_status hweno_f32_round(const double* in, float* out, long long n, void* cuda_stream);

/* CFL reduction that allocates nothing (the paper has no counterpart; it
 * serves callers that cannot call cudaMalloc, e.g. code running under a frozen
 * memory budget or where the implicit synchronisation of an allocation is not
 * allowed, and that therefore cannot create a handle).
 *   grid : problem description as for hweno_create (dim, nx, ny, domain, eq,
 *          adv_a/adv_b); the boundary kinds do not matter here.
 *   gamma: ratio of specific heats (Euler).
 *   m    : device pointer, state in the layout above (no padding).
 *   cfl  : CFL number (> 0).
 *   out  : device pointer to 3 doubles, written {max a_x, max a_y, dt} with the
 *          wave speeds and dt of hweno_max_dt; dt = 0 if a cell average is
 *          non-physical.
 *   cuda_stream: the stream to run on (NULL = legacy default stream).
 * Asynchronous: out is valid once the stream has reached this work.  Scratch is
 * a static device array of 16384 x 2 doubles (256 KiB) per device that loads
 * the library, held until exit; grids beyond 4,194,304 cells (16384 blocks of
 * 256) are rejected with HWENO_EINVAL.  The first call on a device looks the
 * array up (cudaGetSymbolAddress, with that device current): make that first
 * call before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU race; order them on one stream.  Returns EINVAL for bad
 * arguments, ECUDA if a launch fails. */
hweno_status hweno_max_dt_noalloc(const hweno_grid* grid, double gamma, const double* m, double cfl, double* out,
                                  void* cuda_stream);

/* Message of the last error on this handle (never NULL). */
const char* hweno_last_error(hweno_t h);

/* Library version (major * 10000 + minor * 100 + patch). */
int hweno_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HWENO_H */
