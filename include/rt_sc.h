/*
 * rt_sc.h -- C ABI of the GB300 short-characteristics radiative-transfer library.
 *
 * The library solves the time-independent, multi-frequency transfer equation
 *     n . grad I_nu = chi_nu (S_nu - I_nu),   S_nu = eps_nu B_nu + (1 - eps_nu) J_nu
 * (Davis, Stone & Jiang 2012, Eqs. 8-9) on a uniform 3D or 2D Cartesian grid with
 *   - the short-characteristics formal solution with linear upwind-face
 *     interpolation and exponential segment weights (Sec. 3.3, Eq. 20),
 *   - the discrete moments J, H, K (Eqs. 17-19) and the diagonal Lambda*
 *     (Sec. 3.4, Olson & Kunasz 1987),
 *   - Jacobi accelerated Lambda iteration (Sec. 3.4, Eq. 24) with the
 *     max |dS|/S convergence test (Eq. 25),
 *   - the integral-form heating rate and the Eddington tensor K/J (Sec. 4).
 *
 * Conventions shared by every call:
 *   - Status codes, never exceptions.  On failure rt_last_error() describes why.
 *   - Cell arrays are float64, C order [nf][nz][ny][nx] (x fastest).
 *   - Inputs are copied in; the caller keeps ownership of its pointers and
 *     allocates every output buffer.  The library owns all device state of a grid.
 *   - on_device = 0: pointers are host memory.  on_device = 1: pointers are device
 *     memory on the grid's device, read/written on the call's stream.
 *   - Calls that return host scalars (iteration counts, residuals) or write host
 *     buffers synchronise the stream before returning.
 *   - A grid is not thread-safe: one host thread at a time per grid.
 *   - All compute runs in the library's CUDA kernels; there is no CPU fallback.
 */
#ifndef RT_SC_H
#define RT_SC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_grid_s *rt_grid;   /* opaque handle; owns all device state */

typedef enum {
  RT_OK = 0,
  RT_ERR_ARG = -1,            /* invalid argument or input value */
  RT_ERR_OOM = -2,            /* device allocation failed */
  RT_ERR_CUDA = -3,           /* a CUDA call failed (message has the CUDA error) */
  RT_ERR_NOT_CONVERGED = -4,  /* max_iter formal solutions without meeting tol */
  RT_ERR_TIMEOUT = -5,        /* a wait gave up (rt_wait) */
  RT_ERR_STATE = -6           /* call out of order (e.g. solve before set_opacity_source) */
} rt_status;

/* Boundary type of one face (Sec. 3.5).
 *   PERIODIC: incoming intensity is the outgoing intensity of the opposite face
 *             from the previous formal solution (lagged by one iteration);
 *             both faces of an axis must be periodic together.
 *   VACUUM:   no incoming intensity.
 *   THERMAL:  incoming intensity I = B of the adjacent boundary layer.
 *   FIXED:    incoming intensity given per angle with rt_set_boundary_intensity.
 *   EXTERNAL: (z faces of FP64 3D grids of >= 2 planes, not combined with FIXED
 *             x or y faces) a subdomain face of the domain decomposition of
 *             Sec. 3.5: the ghost layer's opacity, source function and B, and the
 *             incoming intensities (the neighbouring subdomain's, from its previous
 *             formal solution), are set by rt_set_external_face.  Past such a face
 *             an out-of-range non-periodic x or y face decides the ghost intensity
 *             (thermal: the ghost layer's B), as it would in the undecomposed
 *             domain.  Such grids sweep one cell per thread (variant 1).
 * At every other non-periodic face the ghost opacity and source function copy
 * the adjacent boundary layer. */
typedef enum { RT_BC_PERIODIC = 0, RT_BC_VACUUM = 1, RT_BC_THERMAL = 2, RT_BC_FIXED = 3,
               RT_BC_EXTERNAL = 4 } rt_bc;

/* Arithmetic of the formal solution.
 *   FP64:  everything in double precision.
 *   MIXED: the sweep (interpolation, segment weights, intensities, the per-sweep
 *          angle sums) in float32 with a polynomial form of the segment weights
 *          for small optical depth; J summed across sweeps, Lambda*, the ALI
 *          update, its denominator and the convergence test in double precision.
 *          A Jacobi ALI solve with linear interpolation does its first formal
 *          solution in FP64 (on an internal FP64 copy of the grid, allocated by
 *          rt_set_opacity_source unless every eps is 1) and then sweeps only the
 *          change of S in float32, accumulating J in FP64, so that float32
 *          rounding scales with the update, not with S.  The Jacobi update still
 *          amplifies the increments' rounding by about 1/eps in optically thick
 *          cells (measured without the later FP64 iterations: max relative error
 *          of S about 1.6e-8 / eps), so each time the largest relative change of S
 *          has fallen 100-fold another iteration is done in FP64, whose J replaces
 *          the accumulated one (rt_set_fp64_anchors; the errors then fall to
 *          1e-9..1e-6 on the benchmark media), and frequency bins whose smallest
 *          eps among optically thick cells is below 1.2e-4 (unit roundoff / eps >
 *          5e-4, rt_set_fp64_bin_limit) are solved in FP64 by an internal FP64
 *          grid of those bins (rt_get_sweep_plan reports how many): there the
 *          FP64 iterations would have to come so often, to keep the iteration
 *          count within one of the FP64 solve's, that they would cost as much. */
typedef enum { RT_PREC_FP64 = 0, RT_PREC_MIXED = 1 } rt_precision;

typedef struct {
  int nx, ny, nz;        /* cells per axis; nz == 1 selects 2D (z-invariant) */
  double dx, dy, dz;     /* cell spacing (dz ignored in 2D) */
  int n_mu;              /* polar angles: 2, 4, 6, 8, 10 or 12 -> n_mu (n_mu + 2) rays (half in 2D) */
  int nfreq;             /* independent frequency bins, >= 1 */
  rt_bc bc_lo[3];        /* boundary of the low face of x, y, z */
  rt_bc bc_hi[3];        /* boundary of the high face of x, y, z */
  rt_precision prec;
} rt_grid_desc;

typedef struct {
  double tol;            /* delta_c of Eq. 25 (e.g. 1e-6) */
  int max_iter;          /* maximum formal solutions per solve */
  int check_every;       /* formal solutions enqueued between host checks; 0 = automatic */
  void *stream;          /* cudaStream_t to run on; NULL = the grid's own stream */
} rt_solve_opts;

/* Create a grid on the current CUDA device.  Builds the level-symmetric angle set
 * (Sec. 3.2) and allocates device state sized by desc.  *out is set on success.
 * Errors: RT_ERR_ARG (bad sizes, n_mu, or a half-periodic axis), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_create_grid(const rt_grid_desc *desc, rt_grid *out);

/* Release all device state of a grid.  NULL is accepted. */
rt_status rt_destroy_grid(rt_grid g);

/* Number of rays and the angle table: mu [n_angles][3] (direction cosines) and
 * w [n_angles] (weights, sum 1; Eq. 17 carries no 4 pi).  Either pointer may be
 * NULL.  Order: octant o = 0..7 with signs (-1 if o&1, -1 if o&2, -1 if o&4) for
 * (x, y, z), in 2D only the octants with mu_z > 0 (weights doubled); within an
 * octant level indices i outer, j inner, l = n_mu/2 + 2 - i - j. */
int rt_num_angles(rt_grid g);
rt_status rt_get_angles(rt_grid g, double *mu, double *w);

/* The same angle table without a grid (host only, no GPU needed): writes
 * n_angles rows into mu [n][3] and w [n] when they are non-NULL and returns
 * n_angles, or a negative rt_status for an unsupported n_mu.  Sec. 3.2. */
int rt_angle_table(int n_mu, int two_d, double *mu, double *w);

/* Set the medium (Sec. 2, step 1): total opacity chi_tot >= 0, photon destruction
 * probability 0 < eps <= 1, thermal source function B >= 0, all [nf][nz][ny][nx],
 * and the frequency quadrature weights freq_w [nf] used by the heating rate
 * (NULL = all 1).  No NaN/Inf allowed.  Copies the inputs, computes Lambda*
 * (depends on chi only) and resets S to B and the periodic ghosts to the image
 * cells' S.  Errors: RT_ERR_ARG for out-of-range or non-finite values. */
rt_status rt_set_opacity_source(rt_grid g, const double *chi_tot, const double *eps,
                                const double *B, const double *freq_w, int on_device);

/* Incident intensity for a face declared RT_BC_FIXED.  face = 2*axis + side
 * (0 x-lo, 1 x-hi, 2 y-lo, 3 y-hi, 4 z-lo, 5 z-hi).  I is
 * [nf][n_angles][face cells], face cells ordered x-face [nz][ny], y-face [nz][nx],
 * z-face [ny][nx]; only rays entering through the face are used.  Values are
 * used for the ghost vertex just outside each face cell (and, at edges and
 * corners, for the ghost whose first non-periodic out-of-range axis in the order
 * z, y, x is this face's).  Host pointer.  Errors: RT_ERR_ARG, RT_ERR_STATE if
 * the face is not RT_BC_FIXED. */
rt_status rt_set_boundary_intensity(rt_grid g, int face, const double *I);

/* One formal solution J = Lambda[S] (Sec. 3.4, Eq. 21) without an S update.
 * S: [nf][nz][ny][nx] or NULL to use the grid's current S; when S is given the
 * periodic ghosts are reset to the image cells' S (first-iteration semantics),
 * otherwise the lagged ghosts of the previous formal solution are used and
 * advanced.  J_out, lstar_out: [nf][nz][ny][nx] or NULL.  opts may be NULL.
 * Errors: RT_ERR_STATE before rt_set_opacity_source. */
rt_status rt_formal_solve(rt_grid g, const double *S, double *J_out, double *lstar_out,
                          int on_device, const rt_solve_opts *opts);

/* Jacobi ALI to max|dS|/S <= opts->tol (Eqs. 24-25) (or Gauss-Seidel, see
 * rt_set_iteration).  S_init [nf][nz][ny][nx] (device or host per on_device) or
 * NULL to start from S = B.  Periodic ghosts start as the image cells' S.  When
 * every eps == 1 the stopping test uses the change of J between consecutive
 * formal solutions.  iters_out: formal solutions performed; resid_out: the last
 * max relative change.  Iterations are enqueued in batches (opts->check_every,
 * or 4 doubling to 64) with one host check per batch; after the first batch of
 * a solve, a batch's launches are captured once as a CUDA graph and replayed
 * (not while timing is enabled, whose events need direct launches; a stream
 * that cannot be captured, such as the legacy default stream, keeps direct
 * launches).  Returns RT_ERR_NOT_CONVERGED (state kept) if max_iter is reached
 * first. */
rt_status rt_ali_solve(rt_grid g, const double *S_init, int on_device, const rt_solve_opts *opts,
                       int *iters_out, double *resid_out);

/* The Jacobi ALI solves (Eqs. 24-25) of n grids together, each from S = B with
 * the same iterates, results and iteration count as rt_ali_solve would give it
 * (bit for bit), with the sweeps of grids that can share a launch merged: every
 * iteration, one launch sweeps all grids with the pipelined sweep (variant 3:
 * the mixed default) of the same precision and cluster size (rt_set_sweep_config
 * sets it; rows of a multiple of 4 cells or not) -- up to 24 grids per launch --
 * and the other grids' sweeps are launched one by one; then each grid's update.
 * Grids leave as they finish; each keeps its own host-check schedule (as in
 * rt_ali_solve).  All work runs on opts->stream (NULL: the first grid's own
 * stream).  opts (may be NULL) applies to every grid.  iters, resid, status:
 * per grid (each may be NULL).  No counterpart in the paper: many small
 * problems then fill the GPU as one large one does.  Errors: RT_ERR_ARG for a
 * NULL grid; RT_ERR_STATE for a grid without medium, with the Gauss-Seidel
 * iteration or with quadratic interpolation (before any solve); otherwise the
 * first failing grid's status (RT_ERR_NOT_CONVERGED where max_iter ran out;
 * the other grids still finish). */
rt_status rt_ali_solve_many(rt_grid *grids, int n, const rt_solve_opts *opts, int *iters, double *resid,
                            int *status);

/* Outputs of the last formal solution of the latest solve (Sec. 4): J [nf][cells],
 * H [nf][3][cells], K [nf][6][cells] (xx, yy, zz, xy, xz, yz), the variable
 * Eddington tensor f = K/J [nf][6][cells], and the heating rate Q [cells] in the
 * form chosen by rt_set_heating_form (default: the integral form
 * Q = 4 pi sum_nu w_nu eps_nu chi_nu (J_nu - B_nu)).  Any pointer may be NULL.
 * Recomputes that formal solution with moment accumulation.
 * Errors: RT_ERR_STATE if no formal solution has run. */
rt_status rt_moments(rt_grid g, double *J, double *H, double *K, double *f, double *Q,
                     int on_device, const rt_solve_opts *opts);

/* Order of the interpolation on the crossed face (Sec. 3.3).
 *   RT_INTERP_LINEAR (default): bilinear I-, S-, chi- on the upwind face and S
 *     linear along the segment (Eq. 20 with Psi+ = 0).
 *   RT_INTERP_QUADRATIC: the second-order option -- I-, S-, chi- (and S+, chi+ at
 *     the downwind point, the same offsets on the next plane) from the 3 x 3 face
 *     vertices around the cell's column, along the lower canonical face axis
 *     first, each time the parabola through three values clamped to the two that
 *     bracket the point (no new extrema; exact for monotone quadratic data); S
 *     along the segment the quadratic Bezier curve whose control value
 *     S0 - dtau-/2 S'(tau0), S' from the parabola through S-, S0, S+, is clamped
 *     to [min(S-, S0), max(S-, S0)] where that parabola would overshoot.
 *     Lambda* is the local weight of S0 (the control value's dependence limited
 *     to [0, 1]); the clamps make it depend on S, so ALI solves take it from
 *     every formal solution, and RT_PREC_MIXED grids sweep S itself, not its
 *     increments (float32 rounding then limits tol to about 1e-7 / eps).  Uses
 *     the pipelined sweep (variant 3) only.
 * Replans the sweep.  Errors: RT_ERR_ARG for another value; RT_ERR_STATE for
 * quadratic interpolation on a Gauss-Seidel grid (rt_set_iteration). */
typedef enum { RT_INTERP_LINEAR = 1, RT_INTERP_QUADRATIC = 2 } rt_interp;
rt_status rt_set_interpolation(rt_grid g, int order);

/* Iteration scheme of rt_ali_solve (Sec. 3.4).
 *   RT_ITER_JACOBI (default): every S update uses the J of one formal solution
 *     of the previous S (Eq. 24).
 *   RT_ITER_GAUSS_SEIDEL: the Gauss-Seidel scheme (after Trujillo Bueno &
 *     Fabiani Bendicho 1995) in plane-wavefront form.  The reverse axis V is z
 *     (y for 2D grids); the reverse rays are those whose upwind face is normal
 *     to V (ties with V included) with mu_V < 0.  Each iteration solves every
 *     other ray with the current S, then sweeps the reverse rays from the top
 *     plane of V down; each plane's S is updated by Eq. 24 with
 *     J = (other rays' J) + (a first-order correction of the other rays for
 *     the plane above, whose S is already new: the Psi- weights of their
 *     upwind vertices there times its change) + (the reverse rays' J, which
 *     already see the new S above), and the reverse rays' intensities on that
 *     plane then take the change of the S they read from it (Psi0 dS, and on
 *     the top plane of a bounded V axis Psi- times the ghost layer's change).
 *     The fixed point is the Jacobi one; fewer iterations reach it.  As with
 *     Jacobi, RT_PREC_MIXED grids sweep changes after the first iteration
 *     (the forward rays' J and the reverse rays' J kept in FP64); a medium with
 *     eps = 1 everywhere uses the Jacobi test of Eq. 25 on J.  Needs linear
 *     interpolation.  The reverse phase is one cooperative launch whose planes
 *     are separated by grid barriers; a barrier wait that gives up makes the
 *     solve return RT_ERR_CUDA (device error code 60).
 * Rebuilds the rays' sweep groups (tied rays join the V groups) and replans.
 * Errors: RT_ERR_ARG for another value; RT_ERR_STATE for Gauss-Seidel on a
 * grid with quadratic interpolation. */
typedef enum { RT_ITER_JACOBI = 0, RT_ITER_GAUSS_SEIDEL = 1 } rt_iteration;
rt_status rt_set_iteration(rt_grid g, int scheme);

/* Polls (about 64 ns apart) after which a wait at the Gauss-Seidel reverse
 * phase's grid barrier gives up (default 2^22, a quarter of a second or more):
 * every block then returns, the solve returns RT_ERR_CUDA with device error
 * code 60 and the grid stays usable (the next solve clears the error).  No
 * counterpart in the paper: a bound on a device-side wait, which tests set to 0
 * to exercise the path.  Errors: RT_ERR_ARG for a negative limit. */
rt_status rt_set_wait_limit(rt_grid g, long long polls);

/* Mixed grids, Jacobi ALI solves with linear interpolation: after the first
 * (FP64) iteration, another iteration is done in FP64 from the current S each
 * time the largest relative change of S (Eq. 25) has fallen by the factor
 * `drop` since the last one (checked between batches of iterations; default
 * 1e-2; 0 disables).  Its J replaces the J accumulated in FP64 from the float32
 * increments, dropping the rounding they carried so far; without it that
 * rounding biases the converged S by about unit roundoff / eps in optically
 * thick cells, which the heating rate's cancellation J - B shows where J is
 * close to B.  The iteration count is unchanged (an FP64 iteration replaces a
 * float32 one).  Errors: RT_ERR_ARG for drop outside [0, 1). */
rt_status rt_set_fp64_anchors(rt_grid g, double drop);

/* Mixed grids: the limit on unit roundoff / (smallest eps among optically thick
 * cells) above which a frequency bin is solved by the internal FP64 grid of
 * such bins (see RT_PREC_MIXED; default 5e-4).  Takes effect at the next
 * rt_set_opacity_source.  INFINITY keeps every bin in float32; 0 moves every
 * bin with an optically thick cell to FP64.  Errors: RT_ERR_ARG for a negative
 * or NaN limit. */
rt_status rt_set_fp64_bin_limit(rt_grid g, double limit);

/* Form of the heating rate Q returned by rt_moments (Sec. 4).
 *   RT_HEAT_INTEGRAL:     Q = 4 pi sum_nu w_nu chi_abs,nu (J_nu - B_nu), chi_abs = eps chi.
 *   RT_HEAT_DIFFERENTIAL: Q = -4 pi sum_nu w_nu div H_nu, div H from centred
 *                         differences of the cell-centred H (wrapped on periodic
 *                         axes, one-sided at the first and last cell of a bounded
 *                         axis, zero along an axis of one cell).
 *   RT_HEAT_SWITCH:       per cell and frequency, the integral form where
 *                         chi_nu dx <= 1 and the differential form elsewhere, dx
 *                         the largest cell spacing along axes of more than one cell
 *                         (the paper's switch; the integral form loses accuracy in
 *                         optically thick cells, where J ~ B).
 * Errors: RT_ERR_ARG for another value. */
typedef enum { RT_HEAT_INTEGRAL = 0, RT_HEAT_DIFFERENTIAL = 1, RT_HEAT_SWITCH = 2 } rt_heating_form;
rt_status rt_set_heating_form(rt_grid g, int form);

/* Ghost layer of a subdomain (RT_BC_EXTERNAL) z face, side 0 = low, 1 = high
 * (Sec. 3.5): the neighbouring subdomain's opacity chi, source function S and
 * B on its plane next to the face, [nf][ny][nx], and the intensity of every ray
 * there from its previous formal solution, I [nf][n_angles][ny][nx] (only rays
 * entering through the face are read).  Any pointer may be NULL (that part is
 * kept).  A new chi recomputes Lambda*.  Errors: RT_ERR_STATE if the face is not
 * a subdomain face. */
rt_status rt_set_external_face(rt_grid g, int side, const double *chi, const double *S, const double *B,
                               const double *I, int on_device, const rt_solve_opts *opts);

/* The intensities the latest formal solution left on the grid's first (side 0)
 * or last (side 1) z plane, I [nf][n_angles][ny][nx]: what the neighbouring
 * subdomain beyond that face needs for its next formal solution.  Errors:
 * RT_ERR_STATE if the face is not a subdomain face. */
rt_status rt_get_face_intensity(rt_grid g, int side, double *I, int on_device, const rt_solve_opts *opts);

/* A Jacobi ALI solve (Eq. 24) taken one step at a time, for callers that
 * coordinate several grids (the subdomains of a domain decomposition) between
 * iterations.  rt_ali_begin starts it (S = S_init, or B when NULL; periodic
 * ghosts from S) with no stopping rule of its own; rt_ali_iterate performs n
 * iterations (formal solution of the current S, update) and returns the
 * iterations since rt_ali_begin and the max relative change of the last one
 * (Eq. 25; of J when every eps = 1).  Jacobi iteration only.  Errors:
 * RT_ERR_STATE before rt_set_opacity_source, for a Gauss-Seidel grid, or when
 * another solve or formal solution has run since rt_ali_begin. */
rt_status rt_ali_begin(rt_grid g, const double *S_init, int on_device, const rt_solve_opts *opts);
rt_status rt_ali_iterate(rt_grid g, int n, const rt_solve_opts *opts, int *iters_out, double *resid_out);

/* Current source function S [nf][nz][ny][nx]. */
rt_status rt_get_S(rt_grid g, double *S, int on_device, const rt_solve_opts *opts);

/* Device-time record of the latest rt_ali_solve / rt_formal_solve call, taken
 * with CUDA events on the launching stream when enabled.  sweep_ms: summed
 * duration of the formal-solution kernel launches that did work; sweep_launches:
 * how many; total_ms: the whole solve; kernel_launches: all kernels this grid has
 * launched since it was created (cumulative); updates: cell * ray * frequency
 * updates of the latest call; graph_launches: ALI batches replayed as CUDA
 * graphs since the grid was created. */
typedef struct {
  int iters;
  double resid;
  double sweep_ms;
  int sweep_launches;
  double total_ms;
  long long kernel_launches;
  long long updates;       /* cell * ray * frequency updates performed */
  long long graph_launches; /* ALI batches replayed as CUDA graphs (cumulative) */
  int first_fp64;           /* 1 if the latest ALI solve (mixed grid) did its first formal
                               solution in FP64 (see RT_PREC_MIXED) */
  int fp64_anchors;         /* later iterations of that solve done in FP64
                               (rt_set_fp64_anchors) */
  long long shared_launches; /* sweeps launched together with other grids' sweeps
                               (rt_ali_solve_many, the server's shared mode; cumulative) */
} rt_stats;
rt_status rt_enable_timing(rt_grid g, int enable);
rt_status rt_get_stats(rt_grid g, rt_stats *out);

/* Tuning of the formal-solution launch (0 = automatic for each): rays per sweep
 * group (1..8), CTAs per thread-block cluster = strips per plane (1..16),
 * threads per CTA (multiple of 32, <= 512; FP64 grids use at most 256 for
 * variants 2 and 3) and the kernel variant (1 = one cell per thread with direct
 * loads, 2 = shared-memory staged planes with four cells per thread,
 * 3 = pipelined: chi and S staged one plane ahead by asynchronous copies, strip
 * edges exchanged through distributed shared memory).  Automatic choice:
 * variant 3 for RT_PREC_MIXED, 1 for FP64; rays per group and strips from the
 * runtime's count of co-resident clusters (rt_autotune measures instead).
 * Results do not depend on the configuration beyond rounding order.
 * Errors: RT_ERR_ARG for out-of-range values or no feasible configuration. */
rt_status rt_set_sweep_config(rt_grid g, int angles_per_group, int cluster_ctas, int threads,
                              int variant);

/* The sweep plan in use (7 ints): plan[0] variant, [1] groups per frequency,
 * [2] rays per group (max), [3] strips per plane (cluster size), [4] threads per
 * CTA, [5] dynamic shared memory bytes per CTA, [6] frequency bins a mixed grid
 * solves in FP64 (see RT_PREC_MIXED). */
rt_status rt_get_sweep_plan(rt_grid g, int *plan);

/* Time candidate sweep configurations (variant x rays per group x strips) with
 * formal solutions of the current medium, keep the fastest for this grid and
 * remember it for every later grid of the same shape, rays, frequencies,
 * precision and boundaries in this process.  Leaves S = B and fresh ghosts (as
 * rt_set_opacity_source does).  plan_out (7 ints, may be NULL) receives the plan
 * as rt_get_sweep_plan reports it.  Errors: RT_ERR_STATE before
 * rt_set_opacity_source. */
rt_status rt_autotune(rt_grid g, int *plan_out);

/* One formal solution that allocates nothing on the device.
 *
 * The paper has no counterpart: this entry point is for callers that cannot
 * call cudaMalloc, for example a host framework that has already reserved the
 * device memory for its own pool, or a time-critical loop that must not take
 * the device-wide synchronisation an allocation can imply.  It computes what
 * rt_create_grid + rt_set_opacity_source + rt_formal_solve(S) would (J = Lambda[S]
 * with first-iteration periodic ghosts, the default sweep plan, no FP64 bin
 * split), taking all working memory (sweep copies, ghosts, partial sums,
 * tables, control block) from one static device array of
 * RT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  The caller passes device pointers: chi, S, B
 * [nf][nz][ny][nx] (read; not validated) and J_out [nf][nz][ny][nx] (written),
 * and a cudaStream_t (NULL = the legacy default stream); the call synchronises
 * that stream before it returns.
 *   - Problems whose working memory exceeds the array return RT_ERR_ARG before
 *     any device work; so do fixed-intensity faces.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (device current): make that first call before any
 *     stream capture.  The address is kept for the life of the process, so
 *     the entry point must not be called on a device after cudaDeviceReset.
 *   - Every call shares the array and it keeps the previous call's contents
 *     (only its control block is cleared): calls that overlap on the GPU, from
 *     several streams or threads, race and must be serialised by the caller. */
#define RT_NOALLOC_SCRATCH_BYTES (64ULL << 20)
rt_status rt_formal_solve_noalloc(const rt_grid_desc *desc, const double *chi, const double *S,
                                  const double *B, double *J_out, void *stream);

/* ---------------------------------------------------------------- serving
 * A request server (no counterpart in the paper: the library's serving layer).
 * Submitted ALI solves queue in arrival order; each of the server's worker
 * threads takes the oldest one as soon as the estimated device footprint of the
 * solves already running plus the new one fits the server's budget (a solve
 * larger than the budget runs when nothing else does), creates its grid on the
 * worker's own CUDA stream, solves, takes J, S and Q back to host memory and
 * frees the grid.  Solves on different workers overlap on the GPU; each result
 * is the same as that of the same solve run alone (deterministic kernels and a
 * plan that depends on the problem only; in the shared mode, alone with the
 * plan the server gives it: its cluster size set by rt_set_sweep_config, or
 * its own plan in the largest size class).  All calls are
 * thread-safe. */
typedef struct rt_server_s *rt_server;
typedef struct {
  long long device_bytes;   /* admission budget; <= 0: 80 % of the free device memory */
  int workers;              /* worker threads (>= 1): solves in flight at most, or, in the
                               shared mode, grids being set up or read back at once */
  int shared_cluster;       /* 0: each solve on its worker.  1..16: shared mode -- every
                               admitted Jacobi solve with linear interpolation runs in
                               lock-step with the others of its size class (cells x rays x
                               frequencies below 2^22, below 2^26, above; one scheduler
                               thread and stream each), as in rt_ali_solve_many, each grid
                               of the two smaller classes planned with this many CTAs per
                               cluster where that plan fits (the largest keep their own
                               plan); the workers set grids up and read results back
                               (Gauss-Seidel and quadratic requests still run on a worker) */
} rt_server_opts;
typedef struct {
  rt_grid_desc desc;
  int interp;               /* RT_INTERP_LINEAR / RT_INTERP_QUADRATIC (0 = linear) */
  const double *chi, *eps, *B, *freq_w;   /* host arrays as for rt_set_opacity_source;
                                             copied at submission (freq_w may be NULL: 1) */
  double tol;
  int max_iter;
  int iteration;            /* RT_ITER_JACOBI (0) / RT_ITER_GAUSS_SEIDEL (linear only) */
} rt_request;
enum { RT_REQ_QUEUED = 0, RT_REQ_RUNNING = 1, RT_REQ_DONE = 2 };
typedef struct {
  int state;                /* RT_REQ_* */
  int status;               /* the solve's rt_status once done */
  int iters;
  double resid;
  double queue_ms;          /* submission to start */
  double solve_ms;          /* start to done (grid set-up, solve, moments, copies) */
  long long footprint;      /* estimated device bytes */
} rt_request_info;

/* Estimated device memory of a grid with this description (upper bound of the
 * arrays it allocates, with the moments pass; for RT_PREC_MIXED including the
 * internal FP64 grid of its FP64 iterations, but not the FP64 grid of ill-
 * conditioned bins that some media add: up to an RT_PREC_FP64 grid of those
 * bins, see RT_PREC_MIXED).  Errors: RT_ERR_ARG. */
rt_status rt_grid_footprint(const rt_grid_desc *desc, long long *bytes);
rt_status rt_server_create(const rt_server_opts *opts, rt_server *out);
/* Shared sweep launches issued by the server's scheduler so far (shared mode). */
rt_status rt_server_shared_launches(rt_server s, long long *n);
/* Waits for the running solves; queued ones are dropped. */
rt_status rt_server_destroy(rt_server s);
/* Copies the request's inputs and queues it.  Errors: RT_ERR_ARG (NULL or bad
 * description; the medium itself is validated when the solve runs). */
rt_status rt_submit(rt_server s, const rt_request *req, long long *id_out);
/* State of a request.  Errors: RT_ERR_ARG for an unknown id. */
rt_status rt_poll(rt_server s, long long id, rt_request_info *info);
/* Blocks until the request is done or timeout_s has passed (RT_ERR_TIMEOUT). */
rt_status rt_wait(rt_server s, long long id, double timeout_s, rt_request_info *info);
/* Copies the results of a finished request to host arrays (any may be NULL):
 * J and S [nf][cells], Q [cells] (the integral form), and forgets the request.
 * Returns the solve's status (RT_ERR_STATE if it is not done). */
rt_status rt_fetch(rt_server s, long long id, double *J, double *S, double *Q);

/* Measured arithmetic rates of the current device (no counterpart in the paper:
 * the ceilings the formal solution's roofline is reported against).  Writes
 * min(n, 5) values: [0] FP32 flop/s of scalar fused multiply-adds, [1] FP32
 * flop/s of packed-pair fused multiply-adds (fma.rn.f32x2), [2] special-function
 * exponentials/s (ex2.approx), [3] special-function reciprocals/s (rcp.approx),
 * [4] FP64 flop/s of fused multiply-adds.  Each is the best of three timed
 * launches of a probe kernel (8 blocks of 256 threads per SM, 8 independent
 * chains per thread) after a warm-up launch; the whole call takes well under a
 * second.  Allocates (and frees) one small device buffer and synchronises the
 * device.  Errors: RT_ERR_ARG (NULL or n < 1), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_measure_rates(double *rates, int n);

/* Message describing the last error on this thread (never NULL). */
const char *rt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RT_SC_H */
