/*
 * nrr.h -- C ABI of libnrr, a GB300 (sm_103a) solver for binary-black-hole
 * puncture initial data by hyperbolic relaxation (arXiv 2501.14030).
 *
 * The method (paper Sec. 2): the non-singular part u of the conformal factor
 * psi = psi_singular + u satisfies the Hamiltonian constraint
 *     lap(u) + (1/8) A~_ij A~^ij (psi_singular + u)^-7 = 0,
 * which is relaxed as the damped wave system
 *     du/dt = v - eta u,   dv/dt = c^2 [lap(u) + (1/8) A~A~ (psi_s + u)^-7],
 * with c proportional to the local grid spacing, by the method of lines with
 * RK4 on a curvilinear reference-metric grid, until the L2 norm of the
 * residual H (the left-hand side of the constraint) drops below a threshold
 * (paper Alg. 1: RHS -> BC -> RK substeps, H and its norm, stop test).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an nrr_status.  On failure nrr_last_error() gives a
 *    message for the calling thread.  No call aborts or prints.
 *  - Grid functions are padded 3-D arrays of s0*s1*s2 values, flat index
 *    p = i0 + s0*(i1 + s1*i2) (i0 fastest), s_d = n_d + 2*ng, ng = fd_order/2.
 *    Sampling is cell-centred: xx_d = xxmin_d + (i_d - ng + 1/2) dxx_d.
 *  - "Evolved" points are the interior plus the outer ghost shell (points
 *    beyond the outer boundary, evolved by the radiation condition).  Inner
 *    ghosts (xx0 < 0, theta outside [0,pi], phi outside [-pi,pi)) are images
 *    of evolved points; the kernels read them through the image map and only
 *    the calls that copy a grid function out fill them.
 *  - Pointers flagged "on_device" are CUDA device pointers on the current
 *    device; otherwise they are host pointers.  The caller owns every pointer
 *    it passes; the library copies what it keeps.
 *  - Each grid owns a non-blocking work stream.  Every call first orders
 *    that stream after the work already queued on the caller's stream (the
 *    one given to nrr_create_grid; NULL = the legacy default stream), and
 *    returns after its device work is complete.
 */
#ifndef NRR_H
#define NRR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NRR_OK = 0,
  NRR_ERR_INVALID_ARG = 1,   /* bad argument; nothing was changed          */
  NRR_ERR_OOM = 2,           /* device memory would not fit; checked before */
                             /* any allocation                              */
  NRR_ERR_CUDA = 3,          /* a CUDA runtime call failed                  */
  NRR_ERR_NOT_CONVERGED = 4, /* iteration limit reached above tolerance     */
  NRR_ERR_DIVERGED = 5,      /* residual norm became non-finite             */
  NRR_ERR_TIMEOUT = 6,       /* wall-clock limit of the solve reached       */
  NRR_ERR_STATE = 7          /* call out of order (e.g. relax before        */
                             /* punctures are set)                          */
} nrr_status;

enum { NRR_SINHSYMTP = 0, NRR_SPHERICAL = 1, NRR_CARTESIAN = 2, NRR_SINHSPHERICAL = 3,
       NRR_SINHCYLINDRICAL = 4 };
enum { NRR_FP64 = 0, NRR_FP32 = 1, NRR_FP32_DC = 2 };
enum { NRR_INIT_ZERO = 0, NRR_INIT_CURRENT = 1, NRR_INIT_HOST = 2,
       NRR_INIT_DEVICE = 3 };

/* Grid description (paper Sec. 2: SinhSymTP coordinates; Sec. 6: other
 * coordinate families; Sec. 4: centred finite differences of selectable
 * order).
 *   coord     NRR_SINHSYMTP: xx0 in [0,1], xx1 = theta in [0,pi],
 *             xx2 = phi in [-pi,pi); A = amax sinh(xx0/w)/sinh(1/w),
 *             x = A sin(th) cos(ph), y = A sin(th) sin(ph),
 *             z = sqrt(A^2 + bscale^2) cos(th), w = sinhwaa.
 *             NRR_SPHERICAL: xx0 = r in [0,rmax].
 *             NRR_CARTESIAN: [-xmax, xmax]^3.
 *             NRR_SINHSPHERICAL: xx0 in [0,1], r = amax sinh(xx0/w)/sinh(1/w),
 *             theta and phi as above (a sinh-stretched spherical grid, one of
 *             the further families of Sec. 6).
 *             NRR_SINHCYLINDRICAL (the cylindrical-like family of Sec. 6),
 *             stored as (rho, z, phi): xx0 in [0,1],
 *             rho = amax sinh(xx0/w)/sinh(1/w); xx1 in [-1,1],
 *             z = zmax sinh(xx1/wz)/sinh(1/wz), wz = sinhwz; xx2 = phi in
 *             [-pi,pi).  Points beyond rho = amax and beyond both ends
 *             |z| = zmax are outer (radiation) points; rho < 0 is imaged.
 *   n[3]      interior points per direction (n[2] even for curvilinear grids).
 *   fd_order  4, 8 or 10.
 *   zmax, sinhwz  SinhCylindrical only (ignored otherwise).                  */
typedef struct {
  int coord;
  int n[3];
  int fd_order;
  double amax, bscale, sinhwaa;
  double rmax;
  double xmax;
  double zmax, sinhwz;
} nrr_grid_desc;

/* One puncture (paper Sec. 2, Brandt-Bruegmann data with Bowen-York
 * curvature): bare mass m > 0, position x, momentum P, spin S. */
typedef struct {
  double m;
  double x[3];
  double P[3];
  double S[3];
} nrr_puncture;

/* Options of one solve (paper Sec. 2 relaxation system; Alg. 1 loop).
 *   mode         NRR_FP64, NRR_FP32 (whole relaxation in single precision)
 *                or NRR_FP32_DC (defect correction: every outer iteration
 *                evaluates in FP64 the relaxation system's right-hand side
 *                at the current state, then integrates in FP32 the
 *                increment of the state under the system linearised there
 *                and forced by that FP64 defect, adds the increment in FP64
 *                and checks the FP64 residual norm).
 *   tol          stop when the residual norm < tol (e.g. 1e-10).
 *   max_iters    RK4 steps allowed (all inner steps for NRR_FP32_DC).
 *   check_every  residual norm evaluated every this many steps (>= 1).
 *   cfl          dt = cfl * min over interior of the local spacing.
 *   eta          damping factor; <= 0 selects 2 pi cfl / (n0 dt).
 *   r_int        the norm integrates over interior points with r < r_int.
 *   initial      NRR_INIT_ZERO (u = v = 0), NRR_INIT_CURRENT (continue from
 *                the grid's state), NRR_INIT_HOST / NRR_INIT_DEVICE (u from
 *                u0, padded FP64 layout; v = eta u).
 *   u0           initial u for NRR_INIT_HOST/DEVICE, else ignored.
 *   timeout_ms   wall-clock limit (<= 0: none); checked between norm checks.
 *   inner_steps  NRR_FP32_DC: FP32 RK4 steps per outer iteration (0: use
 *                check_every).
 *   max_outer    NRR_FP32_DC: outer iterations allowed (0: no limit other
 *                than max_iters, which counts FP32 steps).                 */
typedef struct {
  int mode;
  double tol;
  int64_t max_iters;
  int check_every;
  double cfl;
  double eta;
  double r_int;
  int initial;
  const double *u0;
  int64_t timeout_ms;
  int64_t inner_steps;
  int max_outer;
} nrr_relax_opts;

/* Result of one solve: RK4 steps taken, outer defect-correction iterations,
 * last residual norm, wall seconds of the call, and its status code. */
typedef struct {
  int64_t iters;
  int64_t outer_iters;
  double final_norm;
  double seconds;
  int status;
} nrr_relax_result;

typedef struct nrr_grid nrr_grid;

/* Fills *o with the defaults: FP64, tol 1e-10, max_iters 10^6,
 * check_every 50, cfl 0.5, eta 0 (automatic), r_int 100, zero initial data,
 * no timeout, inner_steps 0 (= check_every), max_outer 0 (no limit). */
nrr_status nrr_default_opts(nrr_relax_opts *o);

/* Creates a grid: computes the full device footprint, fails with
 * NRR_ERR_OOM before allocating if it does not fit, allocates, and runs the
 * coordinate and reference-metric set-up on the device (paper Alg. 1, its
 * set-up: coordinate arrays, reference-metric precompute, boundary
 * containers, storage).  stream: a cudaStream_t, caller-owned, must outlive
 * the grid.  *out receives a handle owned by the caller (nrr_destroy_grid).
 * The kernels index a grid's arrays with 32-bit offsets, so a padded grid
 * holds at most 2^31 points.
 * Errors: NRR_ERR_INVALID_ARG (unsupported coord/order, n < 1, odd n2 on a
 * curvilinear grid, n1 < fd_order/2, more than 2^31 padded points),
 * NRR_ERR_OOM, NRR_ERR_CUDA. */
nrr_status nrr_create_grid(const nrr_grid_desc *d, void *stream,
                           nrr_grid **out);
nrr_status nrr_destroy_grid(nrr_grid *g);

/* Padded dims s[3] (interior plus NG ghost zones on each side, paper Sec. 4
 * memory layout), ghost width NG = fd_order/2, and interior point count of
 * a grid; outputs are caller-owned host memory.
 * Errors: NRR_ERR_INVALID_ARG for a null grid. */
nrr_status nrr_grid_dims(const nrr_grid *g, int s[3], int *ng,
                         int64_t *interior_points);

/* Sets the punctures (1..8) and computes the constant source terms on the
 * device (paper Sec. 2; Alg. 1 "compute constant source terms"):
 * alpha = 1/psi_singular, beta = (1/8) A~_ij A~^ij alpha^7 at every padded
 * point, with psi_singular = 1 + sum m_a/(2 r_a) and Bowen-York A~^ij.
 * p: caller-owned host array, copied.  Errors: NRR_ERR_INVALID_ARG (n out of
 * range, m <= 0, a puncture on a grid point). */
nrr_status nrr_set_punctures(nrr_grid *g, int n, const nrr_puncture *p);

/* Relaxes to tol (paper Alg. 1 relaxation loop).  Returns NRR_OK when the
 * norm fell below tol, else NRR_ERR_NOT_CONVERGED / NRR_ERR_DIVERGED /
 * NRR_ERR_TIMEOUT (also when a stage kernel's bounded wait expired);
 * *r (optional, caller-owned) is filled in every case.  The final state
 * stays on the grid (nrr_get_state).
 * Errors: NRR_ERR_INVALID_ARG (null grid or options, tol <= 0, cfl <= 0,
 * r_int <= 0, check_every < 1, a negative max_iters, inner_steps or
 * max_outer, an unknown mode or initial, a null u0 for
 * NRR_INIT_HOST/DEVICE), NRR_ERR_STATE (punctures not set), NRR_ERR_CUDA. */
nrr_status nrr_relax(nrr_grid *g, const nrr_relax_opts *o,
                     nrr_relax_result *r);

/* Residual H of the current u in FP64 (paper Eq. for u, the "H" of Alg. 1)
 * and its L2 norm over r < r_int: sqrt(sum H^2 J / sum J) over interior
 * points, J = h0 h1 h2 the reference-metric volume factor.
 * h_out (nullable): padded array of s0*s1*s2 doubles, zero off the interior;
 * device pointer when h_on_device, else host; caller-owned.  norm_out
 * (host) nullable.  Errors: NRR_ERR_INVALID_ARG (null grid), NRR_ERR_STATE
 * (punctures not set), NRR_ERR_CUDA. */
nrr_status nrr_residual(nrr_grid *g, double r_int, double *norm_out,
                        double *h_out, int h_on_device);

/* Copies the current state u (and v) of the relaxation system (paper Sec. 2)
 * out, padded layout with inner ghosts filled, FP64 whatever the solve mode;
 * u and v nullable (NULL: not copied); caller-owned arrays of s0*s1*s2
 * doubles, device pointers when on_device.
 * Errors: NRR_ERR_INVALID_ARG (null grid), NRR_ERR_CUDA. */
nrr_status nrr_get_state(nrr_grid *g, double *u, double *v, int on_device);

/* Replaces the state (u, v) of the relaxation system (paper Sec. 2) from
 * padded FP64 arrays (inner ghosts ignored), copied; v may be NULL (v = 0);
 * device pointers when on_device.  Used for checkpoint/resume and warm
 * starts.  Errors: NRR_ERR_INVALID_ARG (null grid or u), NRR_ERR_CUDA. */
nrr_status nrr_set_state(nrr_grid *g, const double *u, const double *v,
                         int on_device);

/* One evaluation of the relaxation right-hand side with its boundary
 * conditions (paper Sec. 2 system; Alg. 1 RHS then BC) on the given state,
 * in the precision of `mode` (NRR_FP64 / NRR_FP32), with damping eta.
 * u, v in: padded FP64; ku, kv out: padded FP64, values at evolved points
 * and inner ghosts (copied from their images).  All device pointers,
 * caller-owned.  Errors: NRR_ERR_INVALID_ARG (null pointer, unknown mode),
 * NRR_ERR_STATE (punctures not set), NRR_ERR_TIMEOUT (a bounded wait
 * expired), NRR_ERR_CUDA. */
nrr_status nrr_rhs(nrr_grid *g, int mode, double eta, const double *u,
                   const double *v, double *ku, double *kv);

/* Takes `steps` RK4 steps (paper Alg. 1 inner loop) from the current state
 * in precision `mode` with time step dt and damping eta, without norm checks.
 * For trajectory comparisons and benchmarks.
 * Errors: NRR_ERR_INVALID_ARG (steps < 0, dt <= 0, unknown mode),
 * NRR_ERR_STATE (punctures not set), NRR_ERR_TIMEOUT if a stage kernel's
 * bounded wait (tensor copies, grid barrier) expired, NRR_ERR_CUDA. */
nrr_status nrr_step(nrr_grid *g, int mode, double dt, double eta,
                    int64_t steps);

/* The time step the solver uses for a given CFL factor (paper Sec. 2: the
 * wave speed follows the local spacing so that one dt satisfies the CFL
 * condition everywhere), and the default damping: dt = cfl * min ds over
 * the interior, eta = 2 pi cfl / (n0 dt).  Host outputs, nullable.
 * Errors: NRR_ERR_INVALID_ARG (null grid, cfl <= 0). */
nrr_status nrr_timestep(const nrr_grid *g, double cfl, double *dt,
                        double *eta_default);

/* Host-side image map of the inner boundary (paper Sec. 2 inner boundary
 * conditions; Alg. 1 BC): out[p] = flat index of the evolved point whose
 * value ghost p copies, or p itself for evolved points.
 * out: caller-owned host array of s0*s1*s2 int32.  Pure host computation,
 * no device.  Errors: NRR_ERR_INVALID_ARG (bad descriptor, null out). */
nrr_status nrr_image_map(const nrr_grid_desc *d, int32_t *out);

/* Measurement hook (the per-kernel timings of paper Sec. 5, taken with CUDA
 * events here): takes `steps` RK4 steps exactly as nrr_step does, with
 * CUDA events recorded on the grid's work stream around them, and returns
 * the average device time of one fused stage launch in *ms_per_launch
 * (4 launches per step).  The state advances.
 * Errors: as nrr_step, and NRR_ERR_INVALID_ARG for steps < 1 or a null
 * output. */
nrr_status nrr_profile_stages(nrr_grid *g, int mode, double dt, double eta,
                              int64_t steps, double *ms_per_launch);

/* Launch shape of the fused stage kernels for the precision of `mode` (NRR_FP64
 * / NRR_FP32); the paper fixes one thread block shape (Sec. 4, parallelization
 * strategy), this library offers several. Curvilinear grids: variant 0 = one
 * thread per (i0, i1) column and zc (1, 2 or 4) phi planes, neighbours read
 * through the caches, in blocks of `block` threads (32, 64, 128 or 256; 0 keeps the
 * current size); variant 1 = tiles of 32 x 4 columns staged plane by plane
 * through registers into shared memory, zc (2, 4, 8 or 16) planes per block;
 * variant 2 = one (column, plane) per step of a grid that exactly fills every
 * SM (zc = 1); variant 3 = 32 x 4 tiles whose planes stream through a shared-
 * memory ring filled by tensor (TMA) copies, zc (2, 4, 8 or 16) planes per
 * block, for FD order 8 with n0 % 32 == 0 and n1 % 4 == 0 (other grids run
 * variant 1 instead; in FP32, block 256 selects 32 x 8 tiles where n1 % 8 ==
 * 0); variant 4 = the RK4 steps between two norm checks in one cooperative
 * launch of a column kernel with grid barriers between stages (zc = 1); variant
 * 5 = the same multi-stage launch over variant 3's tensor-copy tiles, zc (2, 4,
 * 8 or 16) planes per tile, under variant 3's conditions (other grids run
 * variant 4 instead). Single stage launches of variants 4 and 5 run variants 0
 * and 3; variant 6 = two RK4 stages per launch (zc = 1; FP32 stages of
 * SinhSymTP grids of FD order 8 with n0 % 32 == 0, n1 % 4 == 0 and n2 <= 16;
 * one block per 32 x 4 column tile with every phi plane, the first stage on
 * the tile and a halo in shared memory; its single-stage launches run
 * variant 0). Cartesian grids: variant 1 = the tensor-copy kernel under the same
 * conditions, any other variant the column kernel (zc planes per thread,
 * `block` threads). SinhCylindrical grids: variant 0 only. Results do not
 * depend on the shape beyond rounding order.
 * Errors: NRR_ERR_INVALID_ARG for other values. */
nrr_status nrr_set_launch(nrr_grid *g, int mode, int variant, int zc, int block);

/* The current launch shape for `mode` (as set by nrr_set_launch or chosen by
 * nrr_autotune; no paper counterpart); host outputs, nullable.
 * Errors: NRR_ERR_INVALID_ARG (null grid, unknown mode). */
nrr_status nrr_get_launch(const nrr_grid *g, int mode, int *variant, int *zc,
                          int *block);

/* Programmatic dependent launch (no paper counterpart; the paper launches
 * its kernels in sequence, Sec. 4) of the fused stage kernels, both precisions
 * (on = 1, the default): each stage kernel is launched so that its blocks
 * may be scheduled while the preceding kernel on the stream drains; they
 * read only solve-constant data (column weights, geometry) until that kernel
 * has completed and its writes are visible, so results are identical either
 * way.  on = 0 restores plain stream ordering.  Drops the grid's captured
 * relaxation graphs (rebuilt on the next nrr_relax).
 * Errors: NRR_ERR_INVALID_ARG for a null grid or on not 0/1. */
nrr_status nrr_set_pdl(nrr_grid *g, int on);

/* Where the stop test of the relaxation loop runs (paper Alg. 1: the norm is
 * evaluated every check_every steps and the loop stops below tol).  on = 1
 * (the default): on the device -- each nrr_relax is one graph launch in
 * which a conditional WHILE node repeats chunks of check_every RK4 steps (or
 * defect-correction outer iterations) followed by the norm and a control
 * kernel, and the host reads the outcome once at the end; the wall-clock
 * limit is then measured on the device.  on = 0: the host launches one
 * chunk's graph at a time and reads the norm after each.  Both take the same
 * steps and give identical states.
 * Errors: NRR_ERR_INVALID_ARG for a null grid or on not 0/1. */
nrr_status nrr_set_device_loop(nrr_grid *g, int on);

/* The autotuner's cache as a file (JSON; no paper counterpart): every launch
 * shape chosen in this process by nrr_autotune (or loaded), keyed by
 * coordinates, interior sizes, FD order and precision. nrr_autotune_save writes
 * it to `path`; nrr_autotune_load adds the entries of such a file to the cache,
 * so that grids created afterwards with a matching key start with that shape
 * without tuning (grids that exist already keep theirs); nrr_autotune_clear
 * empties the cache. Host only; no GPU work. Errors: NRR_ERR_INVALID_ARG (null
 * path; an unreadable, malformed or invalid file, in which case nothing is
 * added), NRR_ERR_STATE (the file cannot be written). */
nrr_status nrr_autotune_save(const char *path);
nrr_status nrr_autotune_load(const char *path);
nrr_status nrr_autotune_clear(void);

/* Autotuner (project-written; the paper fixes its block shape, Sec. 4):
 * times `trial_steps` RK4 steps for each candidate launch shape with CUDA
 * events on the grid's work stream -- variant 0 with (zc, block) in
 * {(1, 32), (1, 64), (1, 128), (1, 256), (2, 64), (2, 128), (4, 128)}, variant 1 with
 * zc in {2, 4, 8, 16}, variant 2, variant 3 with zc in {2, 4, 8, 16} and
 * block 128 or 256, variant 4, variant 5 with zc in {4, 8, 16} -- skips
 * shapes the grid cannot launch, keeps the fastest for this grid and for
 * every later grid of the same coordinates, sizes, order and precision in
 * this process, and restores the state it started from, bit for bit and in
 * the precision it was held in.  Needs the punctures set.  *best_zc and
 * *best_ms_per_launch (nullable) report the choice and its average time per
 * stage launch.
 * Errors: NRR_ERR_INVALID_ARG (null grid, unknown mode, trial_steps < 1),
 * NRR_ERR_STATE (punctures not set), NRR_ERR_CUDA. */
nrr_status nrr_autotune(nrr_grid *g, int mode, int64_t trial_steps,
                        int *best_variant, int *best_zc,
                        double *best_ms_per_launch);

/* Wave-speed reference of a grid (paper Sec. 2: the wave speed c is
 * proportional to the local grid spacing so that one time step satisfies the
 * CFL condition everywhere): c = (local spacing) / ds_ref instead of
 * (local spacing) / (the grid's own smallest spacing), for a grid that is
 * one patch of a multi-patch system relaxed with one time step
 * dt = cfl ds_ref.  Recomputes the c^2-scaled stencil weights and, if the
 * punctures are set, the c^2-scaled source; the solution of the relaxation
 * does not depend on c.  nrr_timestep then reports dt = cfl ds_ref.
 * Errors: NRR_ERR_INVALID_ARG (null grid, ds_ref not positive), NRR_ERR_CUDA. */
nrr_status nrr_set_speed_reference(nrr_grid *g, double ds_ref);

/* ---- Two overlapping patches (paper Sec. 5: several patches of one solve;
 * Sec. 6: multipatch grids with interpolation between patches) ----------- */
typedef struct nrr_patchset nrr_patchset;

/* Couples an outer grid (any family) and an inner Cartesian grid (a box that
 * overlaps it) into one system.  Receivers: every ghost point of the box,
 * and every interior point of the outer grid with max(|x|,|y|,|z|) < hole.
 * A receiver's value is the tensor-product Lagrange interpolation, q points
 * per direction (q = 2, 4 or 6), of the other patch in that patch's
 * coordinates xx (inner-boundary ghosts of the donor read through their
 * images).  Both grids must have their punctures set; both get the wave-speed
 * reference min(smallest spacing of the two) (nrr_set_speed_reference), which
 * they keep after the patch set is destroyed.  The grids stay owned by the
 * caller and must outlive the patch set.
 * Errors: NRR_ERR_INVALID_ARG (null or equal grids, an inner grid that is not
 * Cartesian, q, hole <= 0, a receiver whose stencil leaves the donor, a donor
 * point that is a receiver of the other link -- a hole too large for the
 * box, a grid of 2^31 points or more), NRR_ERR_STATE (punctures not set),
 * NRR_ERR_OOM, NRR_ERR_CUDA.  nrr_patchset_relax replays each full chunk of
 * check_every steps (both patches' stages, the inner patch's on a side
 * stream, the links, the norm) as one CUDA graph, captured on first use and
 * again when dt, eta, r_int or a grid's launch shape changes. */
nrr_status nrr_patchset_create(nrr_grid *outer, nrr_grid *inner, double hole,
                               int q, nrr_patchset **out);
nrr_status nrr_patchset_destroy(nrr_patchset *ps);

/* Receiver counts of the two links and the common wave-speed reference
 * (host outputs, nullable).  Errors: NRR_ERR_INVALID_ARG for a null set. */
nrr_status nrr_patchset_info(const nrr_patchset *ps, int64_t *outer_receivers,
                             int64_t *inner_receivers, double *ds_ref);

/* The common time step dt = cfl ds_ref and the default damping
 * 2 pi cfl / (n0 dt) with n0 of the outer grid (paper Sec. 2).
 * Errors: NRR_ERR_INVALID_ARG (null set, cfl <= 0). */
nrr_status nrr_patchset_timestep(const nrr_patchset *ps, double cfl, double *dt,
                                 double *eta_default);

/* `steps` RK4 steps of the coupled system in FP64 (paper Alg. 1 inner loop):
 * each stage runs both grids' fused stage kernels, then sets every
 * receiver of the stage's output from the donor's output.  The state is that
 * of the two grids (nrr_get_state / nrr_set_state; a state set from outside
 * should hold interpolated values at the receivers).
 * Errors: NRR_ERR_INVALID_ARG (null set, dt <= 0, steps < 0), NRR_ERR_CUDA. */
nrr_status nrr_patchset_step(nrr_patchset *ps, double dt, double eta,
                             int64_t steps);

/* Norm of the coupled residual (paper Alg. 1 L2 norm): sqrt(sum H^2 J /
 * sum J) over the interior points of both grids with r < r_int that are not
 * receivers.  norm_out: host.  Errors: NRR_ERR_INVALID_ARG, NRR_ERR_CUDA. */
nrr_status nrr_patchset_residual(nrr_patchset *ps, double r_int,
                                 double *norm_out);

/* Relaxes the coupled system (paper Alg. 1 loop): initial NRR_INIT_ZERO or
 * NRR_INIT_CURRENT; dt and eta as nrr_patchset_timestep (o->eta > 0
 * overrides eta); returns as nrr_relax does.  *r (nullable) filled in
 * every case.  Modes:
 *   NRR_FP64: FP64 steps of both patches, norm every check_every steps;
 *   NRR_FP32_DC: defect correction as nrr_relax does it for one grid, on
 *   the coupled system.  Each outer iteration takes both patches' FP64
 *   defects, relaxes their FP32 increments together for inner_steps
 *   (default check_every) steps, with the links applied to the increments
 *   in FP32, then adds the increments to the FP64 state.  The coupled FP64
 *   norm is checked after each outer iteration; max_outer limits the
 *   iterations (0 = none).
 * Errors: NRR_ERR_INVALID_ARG (other modes or initial data, invalid
 * options), NRR_ERR_NOT_CONVERGED, NRR_ERR_DIVERGED, NRR_ERR_TIMEOUT,
 * NRR_ERR_CUDA. */
nrr_status nrr_patchset_relax(nrr_patchset *ps, const nrr_relax_opts *o,
                              nrr_relax_result *r);

/* ---- Batches of independent solves (paper Sec. 5, N independent grids,
 * there on several streams; here one graph launch for all of them) ------- */
typedef struct nrr_batch nrr_batch;

/* Creates a batch of n solves of uneven sizes: descs[i] (SinhSymTP, Spherical
 * or SinhSpherical, one fd_order for the whole batch), npunct[i] punctures at
 * punct[i] (host arrays, copied). Computes the footprint first (NRR_ERR_OOM
 * before any allocation), then allocates one arena per field and runs the set-
 * up of every solve on the device. flags bit 0: also allocate FP64 stage
 * buffers so that NRR_FP64 batch relaxations are possible (NRR_FP32_DC needs no
 * extra storage). stream: as for nrr_create_grid. The paper runs independent
 * patches on separate streams (Sec. 4 scalability, Sec. 5); here one batch
 * object and one graph. Errors: NRR_ERR_INVALID_ARG (n < 1, a bad descriptor,
 * mixed orders or a Cartesian grid, bad punctures), NRR_ERR_OOM, NRR_ERR_CUDA. */
nrr_status nrr_batch_create(int n, const nrr_grid_desc *descs,
                            const int *npunct, const nrr_puncture *const *punct,
                            int flags, void *stream, nrr_batch **out);
nrr_status nrr_batch_destroy(nrr_batch *b);
/* Padded and interior points summed over the solves (host outputs, nullable;
 * the storage of paper Sec. 4 per solve). Errors: NRR_ERR_INVALID_ARG for a
 * null batch. */
nrr_status nrr_batch_info(const nrr_batch *b, int64_t *total_points,
                          int64_t *interior_points);

/* Relaxes every solve of the batch to o->tol (modes NRR_FP64 or
 * NRR_FP32_DC; initial NRR_INIT_ZERO or NRR_INIT_CURRENT) as one CUDA graph
 * launch: each RK4 stage is one kernel over all solves still above tol; the
 * per-solve norms and the stop test run on the device every check_every
 * steps (every inner_steps for NRR_FP32_DC) and a conditional WHILE node
 * repeats the chunk until no solve is left, max_iters steps have been taken
 * or timeout_ms has passed (measured on the device).  per_solve (nullable,
 * n entries) receives each solve's steps, norm and status; total (nullable)
 * the largest step count, the number of chunks and the largest norm.
 * Returns NRR_OK when every solve converged (paper Alg. 1 per solve),
 * else NRR_ERR_NOT_CONVERGED / NRR_ERR_DIVERGED / NRR_ERR_TIMEOUT (also
 * when a stage kernel's bounded wait expired).
 * Errors: NRR_ERR_INVALID_ARG (null batch or options, a mode or initial
 * other than those above, NRR_FP64 without flags bit 0), NRR_ERR_CUDA. */
nrr_status nrr_batch_relax(nrr_batch *b, const nrr_relax_opts *o,
                           nrr_relax_result *per_solve,
                           nrr_relax_result *total);

/* Copies u of solve i (the relaxed field of paper Sec. 2) out (padded FP64
 * layout, inner ghosts filled) to a
 * caller-owned array, device pointer when on_device.
 * Errors: NRR_ERR_INVALID_ARG (null argument, i out of range),
 * NRR_ERR_CUDA. */
nrr_status nrr_batch_get_u(nrr_batch *b, int i, double *dst, int on_device);

/* Sets u of solve i (the field of paper Sec. 2; padded FP64 layout; inner
 * ghosts ignored) for a warm
 * start: a following nrr_batch_relax with initial = NRR_INIT_DEVICE starts
 * from the u of every solve with v = eta u.  u: caller-owned, copied.
 * Errors: NRR_ERR_INVALID_ARG (null argument, i out of range),
 * NRR_ERR_CUDA. */
nrr_status nrr_batch_set_u(nrr_batch *b, int i, const double *u, int on_device);

/* Interior u (paper Sec. 2) of every solve as FP32, dst (device)
 * [n][n0*n1*n2] with i0
 * fastest; all solves must have the same size.  Training targets of the
 * surrogate.  Errors: NRR_ERR_INVALID_ARG (null argument, solves of
 * different sizes), NRR_ERR_CUDA. */
nrr_status nrr_batch_get_interior(nrr_batch *b, float *dst);

/* Stage kernel (paper Alg. 1 RHS, BC and RK substep, fused) of a batch for
 * `mode` (NRR_FP64, or NRR_FP32_DC for its FP32
 * stages; the FP64 defect evaluations of NRR_FP32_DC use the NRR_FP64
 * setting).  Variant 0 stages each plane of a 32 x 4 column tile through
 * registers into shared memory; variant 1 streams the planes of a block's
 * chunk through a ring of shared-memory slots filled by tensor (TMA) copies
 * from per-solve 4-D tensor maps, completing on mbarriers (only for FD order
 * 8 with every solve's n0 % 32 == 0 and n1 % 4 == 0); both take zc (2, 4, 8
 * or 16) phi planes per block and give bitwise identical results.  Variant
 * 2 = one thread per column of evolved points and zc (1, 2 or 4) planes.
 * Defaults: variant 2, zc 1 for FP64; for FP32 variant 1, zc 16 where the
 * batch allows variant 1, else variant 0, zc 4.
 * Errors: NRR_ERR_INVALID_ARG for other values or an ineligible batch. */
nrr_status nrr_batch_set_launch(nrr_batch *b, int mode, int variant, int zc);

/* Autotuner (no paper counterpart; the paper fixes the block, Sec. 4) for
 * the batch's stage kernel (variant and phi planes per block
 * chunk, as in nrr_batch_set_launch), timed over all solves on the current
 * state (restored afterwards); keeps the fastest for later relaxations.
 * Candidates: variant 0 with zc 2, 4, 8, 16; variant 1 with zc 4, 8, 16 (when
 * eligible); variant 2 with zc 1, 2.  Outputs nullable.  NRR_ERR_TIMEOUT if a
 * tensor-copy wait expired. */
nrr_status nrr_batch_autotune(nrr_batch *b, int mode, int64_t trial_steps,
                              int *best_zc, double *best_ms_per_launch,
                              int *best_variant);

/* BF16 tensor-core GEMM used by the surrogate network (no paper
 * counterpart: the paper has no learned component) (tcgen05 MMA with an
 * FP32 accumulator in tensor memory, TMA-fed 128-byte-swizzled tiles):
 * D[m][n] = sum_k A[m][k] B[n][k] for row-major BF16 A (M x K) and B
 * (N x K) -- both K-major -- and row-major FP32 D (M x N).  All device
 * pointers, 16-byte aligned; M % 128 == 0, N % 64 == 0, K % 64 == 0.
 * Tile width and K splits are chosen from the shape (as
 * nrr_gemm_bf16_tn_async with bn = splits = 0).  Synchronous on `stream`:
 * it ends with nrr_gemm_status, so NRR_ERR_TIMEOUT if a pipeline wait of
 * this or an earlier unchecked call expired.
 * Errors: NRR_ERR_INVALID_ARG (null or misaligned pointer, a size that is
 * not a multiple of the tile), NRR_ERR_OOM (split-K workspace),
 * NRR_ERR_CUDA. */
nrr_status nrr_gemm_bf16_tn(const void *A, const void *B, float *D, int M,
                            int N, int K, void *stream);

/* The same product, only enqueued on `stream` (no host synchronisation).
 * persistent: 1 = one CTA per SM walks all output tiles with two tensor-
 * memory accumulators (a tile's epilogue, stored by TMA, overlaps the next
 * tile's main loop); 2 = the same in clusters of two CTAs that take pairs of
 * vertically adjacent tiles and share their B tile by TMA multicast (M %
 * 256 == 0; bitwise equal results, measured 9% slower than 1 at
 * 8192x16384x512, never chosen); 0 = one CTA per output tile; -1 = choose
 * (persistent 1 when there are more 128 x 128 output tiles than SMs and K
 * is not split).
 * bn: output tile width 64, 128 or 256 (must divide N), 0 to choose
 * (persistent: 256 when it divides N, else 128, else 64; K split: 128 when
 * it divides N, else 64; otherwise the widest that divides N and gives at
 * least half as many tiles as SMs, else 64).  splits (one CTA per tile
 * only): number of equal K ranges computed by separate CTAs into a
 * stream-ordered FP32 workspace (splits x M x N, cudaMallocAsync on
 * `stream`, freed on it after use) and summed by a second kernel in a fixed
 * order, so results are deterministic; 1 = no split, 0 = choose (split only
 * when the 128-wide output tiles fill fewer than half the SMs and
 * K / 64 >= 32, into about one CTA per SM, at least eight k-blocks each);
 * at most K / 64.  A
 * pipeline wait that expires is only recorded in a device flag:
 * nrr_gemm_status reads it.
 * Errors (host-side, nothing enqueued): NRR_ERR_INVALID_ARG (as
 * nrr_gemm_bf16_tn, or bn / splits / persistent outside the ranges above,
 * or persistent 1 or 2 with splits > 1), NRR_ERR_OOM, NRR_ERR_CUDA. */
nrr_status nrr_gemm_bf16_tn_async(const void *A, const void *B, float *D, int M,
                                  int N, int K, int bn, int splits, int persistent,
                                  void *stream);

/* Waits for `stream` and reads the GEMM error flag, which every GEMM of the
 * library (nrr_gemm_*, the surrogate) sets when a pipeline wait expires;
 * clears it.  NRR_OK, NRR_ERR_TIMEOUT (a wait expired since the last
 * check: that call's output is incomplete), NRR_ERR_CUDA. */
nrr_status nrr_gemm_status(void *stream);

/* ---- Warm-start surrogate (trained on solutions the solver generates) ---- */
typedef struct nrr_surrogate nrr_surrogate;

/* A multilayer perceptron n_in -> hidden x depth (GELU) -> n_out (linear)
 * with BF16 weights and activations, FP32 accumulation on the tensor cores
 * and FP32 master weights (AdamW).  init_params: host array in the logical
 * packed layout -- for each layer l, W_l as [out][in] row-major then b_l
 * [out] -- of nrr_surrogate_num_params() floats (the caller draws them).
 * Limits: n_in <= 64, hidden and n_out multiples of 128, batch a multiple
 * of 128.  Output scaling starts as the identity (mean 0, std 1).  The
 * paper has no surrogate; this serves the warm start of nrr_relax
 * (NRR_INIT_HOST/DEVICE) and nrr_batch_relax.  init_params is copied.
 * Errors: NRR_ERR_INVALID_ARG (sizes outside the limits, null pointers),
 * NRR_ERR_OOM, NRR_ERR_CUDA. */
nrr_status nrr_surrogate_create(int n_in, int hidden, int depth, int n_out,
                                int batch, const float *init_params,
                                void *stream, nrr_surrogate **out);
nrr_status nrr_surrogate_destroy(nrr_surrogate *s);
int64_t nrr_surrogate_num_params(const nrr_surrogate *s);

/* Surrogate (no paper counterpart).  Sets the output scaling to the
 * per-output mean and standard deviation of
 * Y (device, [n][n_out] FP32); the network learns (Y - mean)/std.
 * Errors: NRR_ERR_INVALID_ARG (null argument, n < 1), NRR_ERR_CUDA. */
nrr_status nrr_surrogate_fit_scaling(nrr_surrogate *s, const float *Y,
                                     int64_t n);

/* Surrogate training (no paper counterpart): `steps` AdamW steps (beta
 * 0.9/0.999, eps 1e-8, decoupled weight decay on
 * weights) on minibatches of `batch` rows: step t uses the sample indices
 * order[t*batch .. (t+1)*batch) (device int32, each in [0, n), at least
 * steps*batch of them; the caller draws the shuffles and the library does
 * not read them back to check).  X: device [n][n_in], Y: device
 * [n][n_out].  loss_out (nullable, host, steps floats) receives each step's
 * mean squared error of the scaled outputs.  With steps >= 2 the first step
 * is launched from the host and the others replay it as one captured CUDA
 * graph (a device step counter selects the minibatch, the loss slot and the
 * AdamW bias corrections): the same kernels and arguments, so the same
 * results as one-step calls.
 * Errors: NRR_ERR_INVALID_ARG (null argument, n < batch, lr <= 0),
 * NRR_ERR_TIMEOUT (a GEMM pipeline wait expired), NRR_ERR_CUDA. */
nrr_status nrr_surrogate_train(nrr_surrogate *s, const float *X, const float *Y,
                               int64_t n, const int32_t *order, int64_t steps,
                               double lr, double weight_decay, float *loss_out);

/* Surrogate inference (no paper counterpart): out (device [n][n_out]) =
 * network(X) mapped back through the scaling;
 * X device [n][n_in]; any n >= 1 (processed in chunks of `batch` rows).
 * Errors: NRR_ERR_INVALID_ARG (null argument, n < 1), NRR_ERR_TIMEOUT,
 * NRR_ERR_CUDA. */
nrr_status nrr_surrogate_predict(nrr_surrogate *s, const float *X, int64_t n,
                                 float *out);

/* Surrogate (no paper counterpart): loss and parameter gradients of one
 * minibatch (the first `batch` rows of
 * X, Y; device) without updating: grads is a host array in the logical
 * packed layout.  For gradient checks.  Errors: NRR_ERR_INVALID_ARG (null
 * argument), NRR_ERR_TIMEOUT, NRR_ERR_CUDA. */
nrr_status nrr_surrogate_gradients(nrr_surrogate *s, const float *X,
                                   const float *Y, float *grads, double *loss);

/* Surrogate (no paper counterpart): current parameters in the logical
 * packed layout (caller-owned host array
 * of nrr_surrogate_num_params() floats).
 * Errors: NRR_ERR_INVALID_ARG (null argument), NRR_ERR_CUDA. */
nrr_status nrr_surrogate_get_params(nrr_surrogate *s, float *params);

/* Warm-start prolongation (no paper counterpart; it feeds the initial data
 * of paper Alg. 1's relaxation): u on the fine grid (device, padded FP64, every
 * point written) interpolated trilinearly in the coordinates xx from the
 * coarse interior values uc (device, [n2][n1][n0] FP32) of a grid of the
 * same curvilinear family and parameters; coarse neighbours across the inner
 * boundary come from their images, beyond the outer boundary the last
 * interior plane is used.  Synchronous on `stream`.
 * Errors: NRR_ERR_INVALID_ARG (null argument, grids of different families
 * or parameters, a bad descriptor, a fine grid above 2^31 points),
 * NRR_ERR_CUDA. */
nrr_status nrr_prolong(const nrr_grid_desc *coarse, const float *uc,
                       const nrr_grid_desc *fine, double *uf, void *stream);

/* Cumulative number of kernels this library has launched in this process
 * (graph replays count every kernel node); a measurement counter with no
 * paper counterpart.  Cannot fail. */
int64_t nrr_kernel_launches(void);

/* Diagnostic (the paper has no counterpart): runs one bounded wait of the
 * kind the stage kernels use on something that never happens -- which = 0:
 * an mbarrier phase that nothing completes (the tensor-copy pipeline's
 * wait); which = 1: a grid barrier that expects one block more than the grid
 * has (the multi-stage kernel's barrier) -- and reports in *expired (host)
 * whether the wait gave up and recorded its error, as it must.  The kernel
 * returns normally, so the context stays usable.  Takes up to a few seconds
 * (the poll limits of those waits).  Work on `stream` (NULL = legacy
 * default); blocks until done.  Allocates 8 bytes of device memory.
 * Errors: NRR_ERR_INVALID_ARG, NRR_ERR_OOM, NRR_ERR_CUDA. */
nrr_status nrr_selftest_wait_expiry(int which, void *stream, int *expired);

/* Diagnostic of the source term's reciprocal (paper Sec. 2 source
 * (psi_s + u)^-7, evaluated as (1 + alpha u)^-1 and products; the paper's
 * Sec. 4 intrinsics discussion is the counterpart): out[i] = the stage
 * kernels' reciprocal of s[i] -- the hardware approximation refined by one
 * third-order step in FP64 (fp32 = 0) or one Newton step in FP32 (fp32 = 1).
 * s, out: device arrays of n doubles (or floats), caller-owned.  Tests
 * compare it with correctly rounded division.  Synchronous on `stream`.
 * Errors: NRR_ERR_INVALID_ARG (null pointer, n < 0, fp32 not 0/1),
 * NRR_ERR_CUDA. */
nrr_status nrr_selftest_recip(const void *s, void *out, int64_t n, int fp32,
                              void *stream);

/* Address checks of the debug build (no paper counterpart; a stand-in for
 * a memory checker where none can run).  libnrr_debug.so, built with
 * NRR_DEBUG=1, checks every load and store of the stencil, boundary and
 * residual kernels against the device allocations the library owns (grids,
 * batches, patch systems, surrogates): an access outside all of them is
 * skipped (a load reads zero, a store is dropped) and recorded, and nothing
 * traps.  This call waits for the device, then reports *enabled = 1 for the
 * debug build (0 for the release build, whose kernels check nothing),
 * *first_bad = the first refused device address since the previous call
 * (0: none) and *refused = how many accesses were refused since then, and
 * clears the record.  Outputs host, nullable.  Errors: NRR_ERR_STATE if more
 * allocations were alive at once than the check's table holds (the check
 * was then incomplete), NRR_ERR_CUDA. */
nrr_status nrr_debug_check(int *enabled, unsigned long long *first_bad,
                           unsigned long long *refused);

/* Measurement hook for the rooflines (the paper's Sec. 5 roofline uses the
 * vendor's peaks; here they are measured): kernels of this library, timed
 * with CUDA events on `stream` (best of five), report
 *   fp64_tflops  FP64 FMA throughput (2 flops per FMA) with eight
 *                independent chains per thread on every SM;
 *   fp32_tflops  the same in FP32;
 *   l2_gbs       read bandwidth from a buffer of l2_bytes (0: 48 MiB) that
 *                stays in L2, read 20 times over.
 * Allocates and frees its buffer.  Outputs host, nullable.
 * Errors: NRR_ERR_INVALID_ARG (l2_bytes not 0 and outside [1 MiB, 4 GiB]),
 * NRR_ERR_OOM, NRR_ERR_CUDA. */
nrr_status nrr_probe_peaks(int64_t l2_bytes, void *stream, double *fp64_tflops,
                           double *fp32_tflops, double *l2_gbs);

/* Residual norm without any device allocation.  The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc,
 * for instance an application whose memory manager already owns the whole
 * device, or an embedding whose policy allows no allocation calls after
 * start-up.  No grid object is needed: for the grid described by d and the
 * punctures p (host array, 1..8), it evaluates H = lap(u) + (1/8) A~A~
 * (psi_s + u)^-7 at interior points of the caller's u (device pointer,
 * padded FP64 layout, inner ghosts ignored) and writes the L2 norm over
 * r < r_int, sqrt(sum H^2 J / sum J), to norm_out[0] (device pointer), and H
 * to h_out (device pointer, padded, nullable; only interior points are
 * written).  Geometry and source are recomputed per point.
 * Work is queued on `stream` (a cudaStream_t, NULL = legacy default); the
 * results are ready when that stream has reached this point.
 * Scratch: the per-block partial sums live in one static device array of
 * 32768 pairs of doubles (512 KiB), held by every GPU that loads the
 * library until exit.  Grids with n0*n1 > 32768*128 are rejected with
 * NRR_ERR_INVALID_ARG.  Every call reuses that array and each launch writes
 * every slot it reads, so nothing needs clearing between calls; calls that
 * overlap on the GPU (on different streams, or from several host threads)
 * race on it and must be serialised by the caller.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before capturing any stream.  The
 * address is remembered with the device's context and looked up again when
 * another context is current (after cudaDeviceReset, for instance).
 * The caller's buffers cannot be checked here: u and h_out must hold
 * s0*s1*s2 doubles and norm_out at least one.
 * Coordinates: SinhSymTP, Spherical and Cartesian (not SinhSpherical or
 * SinhCylindrical).
 * Errors: NRR_ERR_INVALID_ARG (null pointer, a descriptor the grid calls
 * reject -- see nrr_create_grid --, SinhSpherical, punctures, r_int <= 0,
 * n0*n1 beyond the scratch), NRR_ERR_CUDA (lookup or launch failure). */
nrr_status nrr_residual_noalloc(const nrr_grid_desc *d, int npunct,
                                const nrr_puncture *p, const double *u,
                                double r_int, double *norm_out, double *h_out,
                                void *stream);

const char *nrr_last_error(void);
const char *nrr_version(void);

#ifdef __cplusplus
}
#endif
#endif
