/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the periodic lattice
 * Boltzmann scheme for quasi-static linear elasticity of Boolakee, Geier and
 * De Lorenzis, "A new lattice Boltzmann scheme for linear elastic solids:
 * periodic problems" (arXiv 2208.14870).
 *
 * The library advances one D2Q8 distribution function (the D2Q9 set without
 * its inert rest population, Sec. 3.3.2) on a doubly periodic nx-by-ny
 * lattice in pseudo-time until the displacement reaches the quasi-static
 * steady state of the damped Navier-Cauchy equation (Eq. linelasdamp), and
 * recovers displacement and Cauchy stress from the moments (Table 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lattice units: Delta x = Delta t = 1.  lambda and mu are the
 *    dimensionless Lame parameters (Sec. 2.2); K = lambda + mu
 *    (Eq. material_relations).  The body force g is the lattice force
 *    g = eps^2 g^(2) of Sec. 3.3.2 (for a problem posed on the unit square
 *    with E~ = 1, g = b / N^2).
 *  - Fields are row-major nx*ny arrays: node (x, y), 0 <= x < nx,
 *    0 <= y < ny, at index y*nx + x; the node sits at ((x+1/2), (y+1/2))
 *    (Sec. 5.1: the lattice is offset by half a spacing from the periodic
 *    boundary).
 *  - Population arrays are 8 planes of nx*ny doubles in the paper's
 *    one-index order (Sec. 4, population table):
 *      c = (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 *    They hold the pre-collision populations f_i(x, t) (input of
 *    Algorithm 1).
 *  - Stress is returned in lattice units: sigma_lat = eps * sigma~, i.e.
 *    sigma_xx = -(mbar_s + mbar_d)/2, sigma_yy = -(mbar_s - mbar_d)/2,
 *    sigma_xy = -mbar_11 (Table 2 without the 1/eps factor).
 *  - Host pointers are caller-owned; the library never keeps them after the
 *    call returns.  Device pointers ("_device" entry points) are CUDA global
 *    memory of the current device; the caller keeps ownership.
 *  - Every call returns a status (LBM_OK = 0 or a negative LBM_ERR_*), never
 *    aborts, and leaves a human-readable message for lbm_last_error().
 *  - Work is enqueued on the context's stream (lbm_set_stream; default: the
 *    legacy default stream).  Calls that read or write host buffers,
 *    lbm_set_force_device and lbm_solve synchronise that stream before
 *    returning; lbm_iterate, lbm_iterate_checked without output, lbm_reset and
 *    lbm_get_fields_device only enqueue.
 *  - A context belongs to the device that was current at lbm_create and
 *    must be used from one host thread at a time.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

/* Population storage type.  Collision arithmetic is FP64 for LBM_F64 and
 * FP32 for the other two.
 *  LBM_F64  : 8 FP64 planes.
 *  LBM_F32  : 8 FP32 planes.
 *  LBM_F16S : "shifted" FP16 storage: per node the first post-collision
 *             moments (m*_10, m*_01) in FP32 and, per population, the FP16
 *             deviation f*_i - E_i from an equilibrium-type part E_i that is
 *             M^-1 applied to (m*_10, m*_01, 0, 0, 0, theta m*_10,
 *             theta m*_01, 0); the deviations carry a power-of-two scale
 *             chosen from the force so they stay in FP16's normal range. */
enum lbm_dtype { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2 };

enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,            /* invalid argument (sizes, moduli, NaN, null pointer) */
    LBM_ERR_OOM = -2,            /* device or pinned host allocation failed */
    LBM_ERR_CUDA = -3,           /* a CUDA runtime call failed */
    LBM_ERR_DIVERGED = -4,       /* non-finite displacement seen by the residual check */
    LBM_ERR_NOT_CONVERGED = -5,  /* lbm_solve reached max_iters above tolerance */
    LBM_ERR_TIMEOUT = -6,        /* a bounded device-side wait gave up */
    LBM_ERR_STATE = -7           /* call not valid in the current state */
};

/* Optional scheme parameters (lbm_create_ex).  Zero-initialise, then set:
 *   theta : equilibrium constant of m_12^eq = theta*mbar_10 (Sec. 3.3.2);
 *           0 means the standard 1/3.  Must lie in (0, 1).
 *   tau12 : relaxation time of m_12 and m_21 (Eq. relaxation_time);
 *           0 means the standard 1/2 (rate 1).
 *   tau22 : relaxation time of m_22; 0 means 1/2.
 * Non-standard tau12/tau22 reproduce the fourth-order special case of
 * Sec. 6.3.3 / Appendix C. */
typedef struct lbm_options {
    double theta;
    double tau12;
    double tau22;
} lbm_options;

/* Relaxation rates in use (Table 1 with Eq. relaxation_rate:
 * w = 1/(tau + 1/2), theta tau_11 = mu, (1 - theta)/2 tau_d = mu,
 * (1 + theta)/2 tau_s = K). */
typedef struct lbm_rates {
    double w11, ws, wd, w12, w21, w22, theta;
} lbm_rates;

/* Create a context: allocates the population buffers (two, ping-pong), the
 * force, the displacement snapshot of the residual check and the reduction
 * scratch on the current device, and sets the state to the equilibrium of
 * u_0 = 0, i.e. all populations zero (Eq. init_cond), with zero force.
 * nx, ny >= 1; mu > 0; lambda + mu > 0; dtype one of lbm_dtype.
 * Errors: LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_create(int nx, int ny, double lambda, double mu, int dtype, lbm_ctx **out);
int lbm_create_ex(int nx, int ny, double lambda, double mu, int dtype,
                  const lbm_options *opt, lbm_ctx **out);

/* Free everything the context owns (synchronises its stream first).  Null is
 * ignored. */
void lbm_destroy(lbm_ctx *ctx);

/* Use `stream` (a cudaStream_t, may be null for the legacy default stream) for
 * all later work of this context.  The caller keeps ownership of the stream. */
int lbm_set_stream(lbm_ctx *ctx, void *stream);

/* How the calls that take host arrays (lbm_set_force, lbm_get_displacement,
 * lbm_get_stress) move them; no counterpart in the paper.
 *  LBM_HOST_DIRECT (default): pinned host arrays the device can address are
 *    read or written by the library's kernels directly over the host link (no
 *    device staging); other host arrays go through device staging by copies.
 *  LBM_HOST_COPY: every host array goes through device staging by copies, which
 *    the GPU's copy engines carry: a transfer then occupies no SM and overlaps
 *    the kernels that other contexts run on other streams (several lattices
 *    solved side by side).  Staging: up to 5 nx*ny doubles of device memory.
 * Both give the same values.  On GB300 (16384^2, FP32) the direct route was
 * the faster one both for one lattice and for two solved side by side: the
 * staged field copies add a device pass, and the copies slow down beside the
 * other lattice's kernels about as much as the direct transfers do.
 * Errors: LBM_ERR_ARG (mode not one of lbm_host_transfer). */
enum lbm_host_transfer { LBM_HOST_DIRECT = 0, LBM_HOST_COPY = 1 };
int lbm_set_host_transfer(lbm_ctx *ctx, int mode);
int lbm_get_host_transfer(lbm_ctx *ctx, int *mode);

/* Pseudo-time steps per stream-collide launch: 1 to 4.  With k > 1, one
 * launch runs k consecutive steps of Algorithm 1 (Sec. 3.3, Eqs. collision and
 * streaming): the intermediate post-collision states stay on chip in FP32, so
 * the populations cross device memory once per k steps.  Up to three steps
 * this runs on tiles (the tile and a halo of one node per extra step in shared
 * memory); four steps need the wavefront schedule (lbm_set_wavefront), and
 * without it k = 4 runs as k = 3.  A residual check (lbm_iterate_checked,
 * lbm_solve) falls on the last step of a launch: of a four-step wavefront
 * launch where that schedule runs, else of a launch of at most two steps;
 * steps left over when n is not a multiple of k run in shorter launches.  With LBM_F32 storage the
 * arithmetic per node is unchanged and the state after every launch equals
 * that of the same steps taken one per launch, bit for bit.  With LBM_F16S
 * storage the intermediate states are not rounded to the FP16 storage format,
 * so results differ from one step per launch by less than that format's
 * rounding (and lie closer to the FP64 result).  Available for LBM_F32 and
 * LBM_F16S storage on any lattice; the default is 4 (wavefront schedule) from
 * nx >= 256 and ny >= 8 on, else 3 from nx >= 64 and ny >= 16 on (a smaller
 * lattice fills the on-chip tile more than once and is faster one step per
 * launch).  LBM_F64 storage always runs one step per
 * launch.  Paper: the scheme advances one step at a time; grouping steps into
 * launches is a schedule of the same steps, not part of the method.
 * Errors: LBM_ERR_ARG (k outside 1..4, or k > 1 with LBM_F64 storage). */
int lbm_set_steps_per_launch(lbm_ctx *ctx, int k);
int lbm_get_steps_per_launch(lbm_ctx *ctx, int *k);

/* Wavefront schedule of launches of three or four steps (rows > 0: segments
 * of `rows` rows; rows = -1: segments chosen per launch), or the tile schedule
 * (rows = 0).  On the wavefront schedule a block owns a strip of 256 slot
 * columns and a segment of lattice rows and walks down the segment one row per
 * iteration at every step level at once, step j trailing step j - 1 by two
 * rows, each level keeping four rows in shared memory: the halo is 2(k - 1)
 * columns per strip instead of a ring of nodes around every tile.  Same steps
 * and, for LBM_F32, the same bits as one step per launch (see
 * lbm_set_steps_per_launch).  Used where nx >= 256 and ny >= 8; smaller
 * lattices keep the tile schedule.  With rows = -1 a segment is 256 rows,
 * halved (down to 16) while the grid would have fewer than four waves of
 * resident blocks.  Default -1 for LBM_F32 and LBM_F16S storage, 0 for
 * LBM_F64.
 * Errors: LBM_ERR_ARG (rows outside -1..2^20, or rows != 0 with LBM_F64
 * storage). */
int lbm_set_wavefront(lbm_ctx *ctx, int rows);
int lbm_get_wavefront(lbm_ctx *ctx, int *rows);

/* Body force (constant in pseudo-time, Sec. 2.1).  gx, gy: host arrays of
 * nx*ny doubles (lattice units), copied.  Pinned host arrays the device can
 * address (cudaHostAlloc / cudaMallocHost, or registered mapped memory) are
 * read by the conversion kernel directly over the host link, unless
 * lbm_set_host_transfer chose LBM_HOST_COPY; other host arrays go through a
 * device staging copy.  The force must be finite; the
 * steady state exists for a zero-mean force (the mean of u is conserved,
 * Sec. 6.2), which is the caller's responsibility.  For LBM_F16S a change of
 * the force magnitude rescales the stored deviations.  Synchronous. */
int lbm_set_force(lbm_ctx *ctx, const double *gx, const double *gy);

/* Same, from device arrays of nx*ny doubles.  Synchronises the context's
 * stream (the force is checked for non-finite values and, for LBM_F16S, its
 * maximum sets the storage scale). */
int lbm_set_force_device(lbm_ctx *ctx, const double *gx, const double *gy);

/* Body force with the higher-order correction of Sec. 4 (Eqs.
 * force_correction_x/y, "improved scheme" of Sec. 6.3.2) applied on the device
 * in lattice units with periodic central differences:
 *   gx' = gx - (D1 dxx gx + D2 dxy gy + D3 dyy gx),
 *   gy' = gy - (D3 dxx gy + D2 dxy gx + D1 dyy gy),
 * dxx g = g(x+1) - 2g(x) + g(x-1), dxy g = (g(x+1,y+1) - g(x+1,y-1) - g(x-1,y+1)
 * + g(x-1,y-1))/4.  d = {D1, D2, D3} (host, finite).  gx, gy as in
 * lbm_set_force.  Synchronous.  The caller chooses D: the constants printed in
 * Appendix B (lbm_error_constants) do not cancel the force-driven leading
 * error of this scheme as printed (D1 and D2 carry misprints, and the printed
 * constants have the opposite sign of the error equation as written), so they
 * are an input here rather than computed; d = -(D1, D2, D3) of lbm_error_constants_scheme
 * cancels it (about ten times smaller errors at nu = 0.8, E = 0.085, Sec. 6.3.2). */
int lbm_set_force_corrected(lbm_ctx *ctx, const double *gx, const double *gy, const double *d);

/* The leading-order error constants as printed in Appendix B:
 * out[0..4] = C1..C5, out[5..7] = D1..D3, for dimensionless Young's modulus E
 * (> 0), Poisson's ratio nu (-1 < nu < 1), theta (0 = 1/3) and relaxation
 * times tau12 = tau21 (0 = 1/2) and tau22 (0 = 1/2).  Host-only arithmetic. */
int lbm_error_constants(double E, double nu, double theta, double tau12, double tau22,
                        double *out);

/* The same constants of the scheme itself: Appendix B with three misprints
 * read, so that they equal the exact discrete leading error of this scheme
 * (extracted from its one-step operator: decay rates and eigenvectors of
 * free plane waves for C1..C5, steady states for D1..D3).  C2's E^3 term is
 * divided by 8 theta (1 - theta^2)(1 - nu^2)^3 as are those of C3 and C4
 * (printed: 8 (1 - theta^2)(1 - nu^2)^3); the E terms of D1 and D2 are divided
 * by (1 - theta^2)(1 - nu^2) and 2 (1 - theta^2)(1 - nu^2) (printed:
 * (1 - nu^2)^2).  The other five are the printed ones.  As printed, the
 * constants carry the opposite sign of the error source of Eq. ux_order2, so
 * the correction that cancels the force-driven leading error (the improved
 * scheme of Sec. 6.3.2) is lbm_set_force_corrected with d = -(D1, D2, D3).
 * Arguments and errors as lbm_error_constants.  Host-only arithmetic. */
int lbm_error_constants_scheme(double E, double nu, double theta, double tau12, double tau22,
                               double *out);

/* Relaxation times of the fourth-order special case (Sec. 6.3.3): tau12 =
 * tau21 as in Appendix C, which zeroes C5, and tau22 such that C1 of Appendix
 * B vanishes too (C1 is linear in tau22; the tau22 printed in Appendix C does
 * not zero it).  With both zero and the force correction d = -(D1, D2, D3) of
 * lbm_error_constants_scheme, a displacement field without mixed fourth
 * derivatives converges at fourth order.  Pass them in lbm_options; check
 * stability with lbm_spectral_radius (large regions of (E, nu) are unstable,
 * Sec. 6.3.3).  theta 0 = 1/3.  Host-only; LBM_ERR_ARG for E <= 0, nu outside
 * (-1, 1), theta outside (0, 1) or nu = theta. */
int lbm_fourth_order_taus(double E, double nu, double theta, double *tau12, double *tau22);

/* Von Neumann stability (Sec. 4): sup over sampled wave vectors
 * k = khat (cos phi, sin phi), khat in [0, pi] (nk >= 2 points), phi in
 * [0, pi/4] (nphi >= 1 points), of the spectral radius of the one-step
 * amplification matrix L(k) = diag(exp(-i k.c)) A, A of Eq. lbmvector with
 * the Table 1 equilibria.  theta, tau12 (= tau21), tau22 as in lbm_options
 * (0 = standard).  The scheme is stable when *rho <= 1 (the conserved
 * k = 0 modes give exactly 1); the paper samples nk = 50, nphi = 5.
 * Host-only; LBM_ERR_ARG for invalid parameters. */
int lbm_spectral_radius(double lambda, double mu, double theta, double tau12, double tau22,
                        int nk, int nphi, double *rho);

/* Back to the zero state (Eq. init_cond with u_0 = 0); step counter 0; the
 * residual snapshot is invalidated.  The force is kept.  Enqueued only. */
int lbm_reset(lbm_ctx *ctx);

/* n >= 0 pseudo-time steps of Algorithm 1 (collision + streaming, periodic
 * wrap by index arithmetic).  Enqueued only. */
int lbm_iterate(lbm_ctx *ctx, int64_t n);

/* n steps in which every check_every-th step also evaluates the steady-state
 * residual (fused into that step).  A check fused into the step that takes
 * the state from time t to t + 1 measures the displacement u^t of its input
 * state; checks run in the steps with (t + 1) % check_every == 0, so the
 * window between two checks is check_every steps.  The last residual is
 * written to
 * out[0..4] if out is non-null: r_inf, r_2, max|u|, ||u||_2, nonfinite flag
 * (see lbm_solve).  Synchronous when out is non-null. */
int lbm_iterate_checked(lbm_ctx *ctx, int64_t n, int check_every, double *out);

/* Iterate until the steady-state residual drops below tol (Sec. 2.1:
 * ||d u/dt|| < TOL "in some norm").  Reading used: every check_every (= k)
 * steps, r = max_x |u^n - u^(n-k)|_inf / (k max_x |u^n|_inf), accumulated in
 * FP64 (r = 0 when u = 0; for FP32 and FP16S storage u of the check step's
 * input state is evaluated exactly as an FP32 pair).  The first check after a
 * reset only takes the snapshot.  The window starts at a multiple of k long
 * enough for the storage's estimated rounding floor and doubles (up to 64 k)
 * after every check whose r is not below 0.95 of the previous one (see
 * lbm_batch_solve), so a residual held up by rounding or decaying very slowly
 * is measured over longer windows.  Stops when r < tol (LBM_OK), when a non-finite displacement
 * appears (LBM_ERR_DIVERGED) or after max_iters steps
 * (LBM_ERR_NOT_CONVERGED).  iters_out / residual_out (nullable) receive the
 * steps taken in this call and the last r.  Synchronous. */
int lbm_solve(lbm_ctx *ctx, double tol, int64_t max_iters, int check_every,
              int64_t *iters_out, double *residual_out);

/* Displacement u_x = mbar_10, u_y = mbar_01 (Table 2, Eq. coll10) of the
 * current state, FP64, into host arrays of nx*ny doubles.  Pinned host arrays
 * the device can address are written by the recovery kernel directly; into
 * other host arrays the fields are copied from a device staging buffer (one
 * recovery per state, shared with lbm_get_stress).  Synchronous. */
int lbm_get_displacement(lbm_ctx *ctx, double *ux, double *uy);

/* Cauchy stress in lattice units (Table 2 times eps, Eq. compute_bared with
 * the Table 1 equilibria), FP64, into host arrays of nx*ny (pinned host
 * arrays written directly, as for lbm_get_displacement).  Synchronous. */
int lbm_get_stress(lbm_ctx *ctx, double *sxx, double *syy, double *sxy);

/* All five fields (u_x, u_y, sigma_xx, sigma_yy, sigma_xy) into a device
 * array of 5*nx*ny doubles (plane-major).  Enqueued only. */
int lbm_get_fields_device(lbm_ctx *ctx, double *out);

/* Pre-collision populations of the current state (8 planes, see above) into
 * a host array of 8*nx*ny doubles.  Synchronous.  Checkpoint / test hook. */
int lbm_get_populations(lbm_ctx *ctx, double *f);

/* Overwrite the state with pre-collision populations f (host, 8*nx*ny
 * doubles, must be finite); rounded to the storage type.  Synchronous. */
int lbm_set_populations(lbm_ctx *ctx, const double *f);

/* Steps taken since the last reset (or set_populations). */
int lbm_get_step(lbm_ctx *ctx, int64_t *step);

/* Relaxation rates and theta in use. */
int lbm_get_rates(lbm_ctx *ctx, lbm_rates *out);

/* Bytes of device memory the context holds. */
int lbm_get_device_bytes(lbm_ctx *ctx, size_t *bytes);

/* Message of the last failing call on this host thread ("" if none). */
const char *lbm_last_error(void);

/* ---------------------------------------------------------------------------
 * Batched solves.  Many independent periodic problems (each the setting of
 * Sec. 2 with its own size, Lame parameters and body force) are solved in one
 * packed device arena by a persistent cooperative kernel: every step walks the
 * tiles of all running problems, a grid-wide barrier separates steps, and the
 * residual check of Sec. 2.1 (reading of lbm_solve) is fused into the last step
 * of each chunk of check_every steps, per problem.  Converged problems drop
 * out of the tile list between chunks.  The chunk (accumulator reset, kernel,
 * read-back) is replayed from a CUDA graph.  The tile shape is chosen by an
 * autotuner that times the first chunks and caches the choice per workload
 * signature in $LBM_AUTOTUNE_CACHE (default ~/.cache/lbm_gb300/autotune.txt;
 * LBM_AUTOTUNE=0 ignores the cache): tiles 32, 64 or 128 columns wide (tile
 * code 1, 2, 4: warps of 32 columns, one step per barrier) or, when
 * check_every is even, LBM_TILE_TWO_STEP tiles (62 x 22 nodes, two steps per
 * tile visit with the intermediate state on chip and one grid barrier per
 * pair of steps; lbm_set_steps_per_launch describes the arithmetic) or, when
 * check_every is a multiple of 4, the wavefront chunk LBM_TILE_WAVE: problems
 * at least 256 columns wide and 8 rows high advance four steps per visit of a
 * wavefront item (a 256-column strip by up to 256 rows on the schedule of
 * lbm_set_wavefront; the rows are halved, down to 16, while the work list
 * would hold fewer than four waves of resident blocks), narrower ones two steps per two-step tile, with two grid
 * barriers per four steps and items taken from a work counter, wavefront
 * items first.  Every tile code computes the same per-node arithmetic; FP32
 * results are the same bits under every code.  A problem that fits these
 * tiles clearly better with x and y exchanged (narrow and tall, or a width just
 * past a multiple of the strip's 250 output columns) is solved on its
 * transpose: the scheme is symmetric under the exchange (u_x <-> u_y, sigma_xx
 * <-> sigma_yy), the outputs are returned in the caller's orientation and
 * lbm_result.transposed reports it; the result then equals the problem solved
 * as given up to rounding.
 * ------------------------------------------------------------------------- */
/* Tile codes in lbm_batch_report.tile_v and lbm_stats.tile_v besides the
 * widths 1, 2, 4: two-step tiles, and the wavefront chunk. */
#define LBM_TILE_TWO_STEP 3
#define LBM_TILE_WAVE 5

typedef struct lbm_problem {
    int nx, ny;                 /* lattice size, >= 1 */
    double lambda, mu;          /* Lame parameters, lattice units; theta = 1/3,
                                   w_12 = w_21 = w_22 = 1 */
    const double *gx, *gy;      /* host, nx*ny each: body force (copied) */
} lbm_problem;

typedef struct lbm_result {
    int status;                 /* LBM_OK, LBM_ERR_NOT_CONVERGED or LBM_ERR_DIVERGED */
    int64_t iters;              /* steps taken (a multiple of check_every) */
    double residual;            /* last r_inf of the problem */
    double *ux, *uy;            /* host outputs, nx*ny each, caller-owned; may be null */
    double *sxx, *syy, *sxy;    /* host outputs (lattice-unit stress); may be null */
    int transposed;             /* out: 1 if the problem was solved on its transpose (x and y
                                   exchanged, a schedule choice for lattices that fit the
                                   arena's tiles better that way; the outputs are in the
                                   caller's orientation and differ only in rounding) */
} lbm_result;

typedef struct lbm_batch_report {
    int tile_v;                 /* tile code used: 1, 2, 4 (warps of 32 columns), LBM_TILE_TWO_STEP or LBM_TILE_WAVE */
    int blocks;                 /* grid of the persistent chunk kernel */
    int64_t chunks;             /* chunk launches */
    int64_t lattice_updates;    /* sum over problems of nodes x steps */
    double device_ms;           /* device time of the chunks (CUDA events) */
    double wall_ms;             /* whole call */
} lbm_batch_report;

/* Solve `count` problems to residual tol (checked every check_every >= 2
 * steps; a problem stops at the first check below tol, at divergence, or at
 * the first check at or beyond max_iters steps).  Rounding keeps a stored
 * state jittering by about J |u| (measured on converged states: J ~ 1.3e-7 to
 * 4.3e-7 for FP32; 2.5e-7 to 1e-5 for FP16-shifted storage, larger for a
 * shorter side and a larger nu), which floors a w-step residual near J / w.
 * Each problem starts with windows of check_every * min(64, max(1, ceil(2 J /
 * (tol * check_every)))) steps, J = 4e-7 (FP32) or 6e-4 / min(nx, ny) (FP16S),
 * and its window doubles (up to 64 check_every) after every check whose
 * residual is not below 0.95 of the previous one, as lbm_solve does.  dtype:
 * LBM_F32 or LBM_F16S.
 * results[i] receives status, steps, residual and, where the pointers are
 * non-null, the FP64 displacement and stress (Table 2).  report may be null.
 * Synchronous.  Returns LBM_OK when every problem was run (per-problem
 * outcomes are in results), LBM_ERR_ARG / LBM_ERR_OOM / LBM_ERR_CUDA otherwise. */
int lbm_batch_solve(int count, const lbm_problem *probs, int dtype, double tol, int check_every,
                    int64_t max_iters, lbm_result *results, lbm_batch_report *report);

/* ---------------------------------------------------------------------------
 * Continuous-batching solve server.  A worker thread owns two packed arenas
 * (FP32 and FP16-shifted storage, half of the HBM budget each).  Submitted
 * requests are copied and queued; between chunks of check_every steps the
 * worker admits queued requests whose lattice fits the free arena memory
 * (oldest first; a request bypassed for more than 50 chunks stops later
 * admissions to its arena until it fits), runs one chunk of every resident
 * problem (lbm_batch_solve's kernel and residual check), and retires problems
 * that converged, diverged or hit max_iters: their fields are recovered into
 * server-owned host memory and their arena memory is reused.  Requests that
 * arrive while others run are therefore solved concurrently with them; a
 * problem's arithmetic does not depend on what else is resident, so its result
 * is the same alone and in the mix.
 * ------------------------------------------------------------------------- */
typedef struct lbm_server lbm_server;

/* Returned by lbm_server_poll / lbm_server_wait while a request is not done. */
#define LBM_PENDING 1

typedef struct lbm_stats {
    int64_t submitted, completed, queued, running;
    double p50_ms, p95_ms, p99_ms, mean_ms;  /* submission -> completion latency */
    double solves_per_s;       /* completed / (last completion - first submission) */
    int64_t lattice_updates;   /* sum of nodes x steps of completed problems */
    double device_ms;          /* device time of all chunks */
    int64_t chunks;
    size_t hbm_bytes;          /* device memory held by the arenas */
    int peak_running;          /* most problems resident at once */
    int tile_v;                /* tile code: 1, 2, 4 (warps of 32 columns), LBM_TILE_TWO_STEP or LBM_TILE_WAVE */
    int failed;                /* LBM_OK, or the error that stopped the worker */
    int64_t memory_waits;      /* admission attempts refused because the request's arena lacked
                                  free memory (one per queued request and chunk) */
    size_t peak_resident_bytes;/* most arena memory held by resident problems at once (both arenas) */
} lbm_stats;

/* Start a server on the current device with an HBM budget (bytes, >= 1 MiB)
 * for the two arenas; residual checked every check_every >= 2 steps. */
int lbm_server_create(size_t hbm_budget_bytes, int check_every, lbm_server **out);

/* Stop the worker (requests still running are abandoned) and free
 * everything.  Null is ignored. */
void lbm_server_destroy(lbm_server *srv);

/* Queue one solve: problem (copied; its host arrays may be freed after the
 * call), dtype LBM_F32 or LBM_F16S, tolerance, step cap.  *ticket identifies
 * it.  LBM_ERR_ARG for a malformed request or a lattice that cannot fit the
 * arena's half of the budget. */
int lbm_server_submit(lbm_server *srv, const lbm_problem *prob, int dtype, double tol,
                      int64_t max_iters, uint64_t *ticket);

/* Non-blocking: LBM_PENDING while the request is queued or running;
 * otherwise fills out (status, iters, residual, and the fields into its
 * non-null host arrays of nx*ny doubles each), forgets the ticket and returns
 * LBM_OK.  LBM_ERR_ARG for an unknown ticket. */
int lbm_server_poll(lbm_server *srv, uint64_t ticket, lbm_result *out);

/* Like lbm_server_poll but waits up to timeout_s seconds. */
int lbm_server_wait(lbm_server *srv, uint64_t ticket, double timeout_s, lbm_result *out);

/* Drop a request (queued: removed; running: released at the next chunk
 * boundary; done: result discarded).  The ticket becomes unknown. */
int lbm_server_cancel(lbm_server *srv, uint64_t ticket);

/* Counters and latency percentiles of the requests completed so far. */
int lbm_server_stats(lbm_server *srv, lbm_stats *out);

/* ---------------------------------------------------------------------------
 * Allocation-free residual-checked step.  The paper has no counterpart: this
 * is a service of the library for callers that may not allocate device
 * memory -- plug-ins whose host application owns every device byte through
 * its own pool, and latency-critical loops that cannot afford cudaMalloc /
 * cudaFree, which may synchronise the whole device.
 *
 * One pseudo-time step with the fused steady-state residual (the kernel of
 * lbm_iterate_checked) on buffers the caller owns.  No memory is allocated:
 * the residual reduction's scratch (one slot of partial sums per block plus a
 * completion counter, about 40 KB) is a static device array of the library,
 * held by every GPU that loads the library until the process exits.
 *
 *  dtype     LBM_F64 or LBM_F32 (LBM_F16S is not supported here).
 *  lambda,mu Lame parameters as in lbm_create; standard theta = 1/3 and
 *            w_12 = w_21 = w_22 = 1.
 *  f_src     device, 8 planes of nx*ny values of the storage type, plane
 *            stride nx*ny, population order of this header: the stored state,
 *            i.e. the post-collision populations f*_i(x) of the previous step
 *            (all zeros is the zero state).
 *  f_dst     device, same layout, receives the state after the step; must not
 *            alias f_src.
 *  gx, gy    device, nx*ny values of the storage type (lattice force).
 *  snapshot  device, 2 planes of nx*ny entries of 8 bytes each: u_x, u_y of
 *            the previous check on input (zeros before the first); on output
 *            the displacement of this step's input state.  LBM_F64: doubles;
 *            LBM_F32: (hi, lo) pairs of floats whose sum is the displacement
 *            to about 2^-44 relative (the layout lbm_iterate_checked keeps).
 *  result    device, 5 doubles: max|du|, max|u|, sum du^2, sum u^2 and a
 *            non-finite flag, du being the change of u since the snapshot;
 *            r_inf = result[0] / (k * result[1]) for a window of k steps.
 *  grid_blocks  blocks of the launch, 0 = one per resident slot of the device
 *            (capped at LBM_NOALLOC_MAX_BLOCKS and at the number of tiles).
 *  stream    cudaStream_t (null: legacy default stream).  Enqueued only.
 *
 * Returns LBM_OK; LBM_ERR_ARG for nx or ny < 1, nx*ny > 2^31, another dtype,
 * non-finite or non-positive moduli, a null or aliased buffer, or
 * grid_blocks outside [0, LBM_NOALLOC_MAX_BLOCKS] (more blocks than the static
 * scratch has slots); LBM_ERR_CUDA if a CUDA call fails.  No message is left
 * for lbm_last_error.
 *
 * The first call on each device looks up the device address of the static
 * scratch (with that device current); make that first call before any stream
 * capture.  All calls share the one scratch array and it keeps the last
 * call's contents; each call clears the counter before its launch.  Calls
 * whose launches overlap on the GPU (different streams, or several host
 * threads) race on the scratch and give wrong residuals: serialise them. */
#define LBM_NOALLOC_MAX_BLOCKS 1024
int lbm_step_checked_noalloc(int nx, int ny, double lambda, double mu, int dtype,
                             const void *f_src, void *f_dst, const void *gx, const void *gy,
                             void *snapshot, double *result, int grid_blocks, void *stream);

/* Measured FP64 FMA throughput of the current device, in G thread-level FP64
 * instructions per second (every SM full of threads running independent
 * dependent-FMA chains, CUDA-event timed, about a quarter of a second).  The
 * FP64 storage path is bound by the FP64 pipe, and this is its roofline
 * denominator.  No counterpart in the paper.  Allocates and frees a small
 * device buffer; synchronous.  LBM_ERR_ARG for a null pointer, LBM_ERR_CUDA
 * if a CUDA call fails. */
int lbm_fp64_fma_rate(double *ginst_per_s);

/* Library version string. */
const char *lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
