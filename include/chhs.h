/*
 * chhs.h -- C ABI of the GB300 (sm_103a) FAS multigrid solver for the
 * second-order convex-splitting Cahn-Hilliard-Hele-Shaw scheme of
 * Chen, Feng, Liu, Wang and Wise (arXiv:1611.02967).
 *
 * The problem (Section 2, first paragraph, and Eqs. 2.4-2.7): on the box
 * (0, n_x h) x (0, n_y h) [x (0, n_z h)] with cell-centred grid functions and
 * homogeneous Neumann boundaries (Appendix A.1), given (phi^{m-1}, phi^m),
 * find (phi^{m+1}, mu^{m+1/2}, p^{m+1/2}) with
 *   phi^{m+1} - phi^m = s div_h(M(A_h phi*) grad_h mu) + s div_h(A_h phi* grad_h p)
 *   mu = chi(phi^{m+1}, phi^m) - phi* - eps^2 Lap_h(3/4 phi^{m+1} + 1/4 phi^{m-1})
 *   Lap_h p = -gamma div_h(A_h phi* grad_h mu)
 * with phi* = 3/2 phi^m - 1/2 phi^{m-1}, chi(a,b) = (a^2+b^2)(a+b)/4 and
 * M(x) = 1 + gamma x^2.  Each step is solved by FAS nonlinear multigrid
 * V(nu1, nu2)-cycles to a residual tolerance (Section 5 preamble).
 *
 * Conventions for every call:
 *  - Arrays hold interior cells only, x fastest, then y, then z
 *    (element (i,j,k) at i + n_x (j + n_y k)); doubles.
 *  - `on_device` = 0: the pointer is host memory (pageable or pinned) and the
 *    call copies synchronously.  `on_device` = 1: the pointer is device memory
 *    of the handle's device, read or written in stream order on the handle's
 *    stream.
 *  - The caller owns every buffer it passes; the handle owns its device
 *    hierarchy (or borrows the caller's arena, chhs_create_ext).
 *  - Every call returns a chhs_status; on an error the handle stays usable and
 *    chhs_last_error() describes it.  A handle is used by one host thread at a
 *    time.
 */
#ifndef CHHS_H
#define CHHS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chhs chhs_t; /* opaque handle: one run and its multigrid hierarchy */

typedef enum {
    CHHS_OK = 0,
    CHHS_ERR_INVALID_ARG = 1,   /* bad dimension, size, parameter or pointer */
    CHHS_ERR_OOM = 2,           /* device allocation failed, or the arena is too small */
    CHHS_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    CHHS_ERR_NOT_CONVERGED = 4, /* max_v V-cycles without reaching tol; state not advanced */
    CHHS_ERR_DIVERGED = 5       /* non-finite or exploding residual; state not advanced */
} chhs_status;

/* Solver options.  The paper's FAS parameters (Section 5 preamble) are the
 * defaults: V-cycles with nu1 = nu2 = 2 smoothing sweeps, tolerance 1e-10,
 * coarsest grid 2 cells per direction. */
typedef struct {
    int nu1;       /* pre-smoothing sweeps per level (default 2) */
    int nu2;       /* post-smoothing sweeps per level (default 2) */
    int max_v;     /* V-cycles per step before CHHS_ERR_NOT_CONVERGED (default 50) */
    int coarsest;  /* coarsening stops before a direction would drop below this (default 2, at least 2) */
    double tol;    /* stopping norm: sqrt(mean over cells of r_phi^2 + r_mu^2 + (s r_p)^2) (default 1e-10) */
    int precision; /* 0: double-precision V-cycles; 1: single-precision V-cycles inside a
                      double-precision defect-correction loop (same tol, measured in double) */
    double max_factor; /* pointwise guard: a step is also held until the largest residual,
                          max over cells of max(|r_phi|, |r_mu|, |s r_p|), is at most
                          max_factor * tol (default 50; 0 turns the guard off).  The mean-square
                          norm alone can pass while the residual sits in a few cells (thin
                          interfaces): at eps/h = 0.4, gamma = 4 on 64^3 it left a pointwise
                          error in phi of 1.2e-9; the default guard brings that to 4.9e-10 and
                          adds no V-cycles on the 512^2 and 128^3 workloads. */
    int coarsest_f64;  /* mixed form: 1 solves the coarsest grid of every single-precision V-cycle
                          in double precision, 0 (default) in single precision; the double form
                          always solves it in double.  Not 0 or 1: CHHS_ERR_INVALID_ARG. */
    int f64_residual;  /* mixed form: 1 forms the defect-correction residual f - N(u) of the
                          double-precision iterate with double-precision instructions; 0 (default)
                          with double-single arithmetic (pairs of floats, ~48 bits) on the
                          single-precision pipes, which run 64 times faster on GB300.  Either
                          way the stopping norm is that of the double-precision iterate.  Not 0
                          or 1: CHHS_ERR_INVALID_ARG. */
    int max_inner;     /* most V-cycles between two stopping norms, 1..4 (default 3; otherwise
                          CHHS_ERR_INVALID_ARG).  After each norm the device predicts, from the
                          contraction per V-cycle it has measured, how many V-cycles the norm
                          still needs to reach tol (rounded to the nearest, at least 1, at most max_inner)
                          and runs that many before the next norm; in the mixed form they are
                          the correction V-cycles of one defect-correction iteration.  A step
                          still ends only on a norm at or below tol.  1: a norm after every
                          V-cycle. */
} chhs_opts;

/* Fill *opts with the defaults above.  Returns CHHS_ERR_INVALID_ARG on NULL. */
chhs_status chhs_default_opts(chhs_opts* opts);

/* Device bytes the handle's hierarchy needs (levels, coefficients, scratch):
 * the admission figure for a memory budget.  0 for invalid arguments. */
size_t chhs_workspace_bytes(int dim, const int n[3], const chhs_opts* opts);

/* Create a run of dimension dim (2 or 3) on an n[0] x n[1] (x n[2]) grid of
 * spacing h > 0 with interface width eps > 0, coupling gamma >= 0 and time
 * step dt > 0 (Section 2).  Every n[a] must be >= 2.  opts NULL means the
 * defaults.  cuda_stream (a cudaStream_t, NULL = a stream the handle creates)
 * orders all of the handle's device work.  Allocates the hierarchy with
 * cudaMalloc.  The state starts at phi^0 = phi^{-1} = 0 until chhs_set_phi.
 * The grid is coarsened by 2 while every extent stays even and at least
 * opts->coarsest; the coarsest level is solved by one thread block, so a
 * grid whose coarsest level stays large (odd extents such as 65 x 65 give a
 * single level of 4,225 cells; the limit is about 1,000 cells in double
 * precision, 2,000 in the mixed form) is rejected with CHHS_ERR_INVALID_ARG,
 * as are opts with sweep counts too large for the mixed form's tiles.
 * Errors: CHHS_ERR_INVALID_ARG (out or n NULL, dim not 2 or 3, an extent
 * < 2 or > 2^20, more than 2^28 cells, h, eps or dt <= 0, gamma < 0, a
 * non-finite h, eps, gamma or dt, invalid opts -- nu1 or nu2 < 0, nu1 + nu2
 * < 1, max_v < 1, coarsest < 2, tol not > 0, precision not 0 or 1,
 * max_factor < 0 or NaN -- and
 * the cases above; these are checked before any CUDA call), CHHS_ERR_OOM,
 * CHHS_ERR_CUDA (for instance, no usable GPU). */
chhs_status chhs_create(int dim, const int n[3], double h, double eps, double gamma, double dt,
                        const chhs_opts* opts, void* cuda_stream, chhs_t** out);

/* As chhs_create, but the hierarchy lives in the caller's device buffer
 * `arena` of `arena_bytes` (>= chhs_workspace_bytes, 256-byte aligned), which
 * must outlive the handle.  The handle allocates no device memory of its own
 * apart from its CUDA graph.  Errors as chhs_create, and, checked before any
 * CUDA call, CHHS_ERR_INVALID_ARG for a NULL or misaligned arena and
 * CHHS_ERR_OOM for one smaller than chhs_workspace_bytes. */
chhs_status chhs_create_ext(int dim, const int n[3], double h, double eps, double gamma, double dt,
                            const chhs_opts* opts, void* cuda_stream, void* arena, size_t arena_bytes,
                            chhs_t** out);

/* Set the two starting levels (Remark 2.2): phi^m = phi0 and
 * phi^{m-1} = phi_prev, or phi^{m-1} = phi0 when phi_prev is NULL.  Resets
 * mu and p (the warm starts of the next solve) to zero. */
chhs_status chhs_set_phi(chhs_t* run, const double* phi0, const double* phi_prev, int on_device);

/* Advance nsteps time steps (one FAS solve each).  vcycles_out (nullable):
 * V-cycles summed over the steps taken; resid_out (nullable): the last
 * stopping norm.  Stops at the first step that fails (NOT_CONVERGED or
 * DIVERGED), leaving phi^m, phi^{m-1} at the last accepted step. */
chhs_status chhs_step(chhs_t* run, int nsteps, int* vcycles_out, double* resid_out);

/* The asynchronous half of chhs_step: enqueue nsteps steps on the handle's
 * stream and return without waiting.  The caller may record events around
 * it, and may call it several times before one chhs_wait: the steps of all
 * those calls count together.  Call chhs_wait before any other call on the
 * handle. */
chhs_status chhs_step_async(chhs_t* run, int nsteps);

/* Wait for the steps enqueued by chhs_step_async since the last wait;
 * outputs (summed over those steps) and status as chhs_step. */
chhs_status chhs_wait(chhs_t* run, int* vcycles_out, double* resid_out);

/* Kernel launches of one time step's graph: *per_vcycle for each V-cycle and
 * *per_step for the frame around the V-cycle loop (setup, restrictions of
 * phi^m and phi*, the initial norm, the mean of p and the accepted step).
 * A step with V cycles and C stopping norms after them (chhs_norm_checks)
 * launches per_step + V * per_vcycle + C kernels (one per norm). */
chhs_status chhs_launch_counts(const chhs_t* run, int* per_vcycle, int* per_step);

/* Stopping norms evaluated after V-cycles during the steps of the last
 * completed chhs_step (or chhs_step_async and chhs_wait), summed over them:
 * with max_inner > 1 fewer than the V-cycles.  Read from the handle's host
 * copy of the device state; no device work.  NULL argument:
 * CHHS_ERR_INVALID_ARG. */
chhs_status chhs_norm_checks(const chhs_t* run, int* checks);

/* Kernel kinds reported by chhs_profile_step. */
enum {
    CHHS_K_SMOOTH = 0,      /* one colour pass of the nonlinear Gauss-Seidel smoother on a coarse
                               level, or in the 2D mixed form one tile launch (its passes fused
                               with the residual and restriction, or with the prolongation);
                               units: cells updated */
    CHHS_K_RESTRICT = 1,    /* residual + restriction to the next level; units: fine cells */
    CHHS_K_COARSE_RHS = 2,  /* FAS coarse right-hand side; units: coarse cells */
    CHHS_K_PROLONG = 3,     /* prolongation + correction; units: fine cells */
    CHHS_K_COARSEST = 4,    /* the one-block tail: the bottom levels of a V-cycle and the
                               coarsest-grid solve; units: 1 per launch */
    CHHS_K_NORM = 5,        /* stopping norm on the finest grid; units: cells */
    CHHS_K_FRAME = 6,       /* setup, coefficient restriction, mean of p, accept, and the
                               mixed form's double-precision update; units: launches */
    CHHS_K_SMOOTH_FINEST = 7, /* the smoother (or its tiles) on the finest level; units: cells
                                 updated */
    CHHS_K_COUNT = 8
};

/* Advance one time step exactly as chhs_step(run, 1) does, but launch the
 * kernels one by one (no graph) with a CUDA event pair around each, and add
 * into the caller's arrays of CHHS_K_COUNT entries: device milliseconds,
 * launches and work units per kernel kind.  For profiling only: the host
 * reads the loop decision after every stopping norm and launches the
 * V-cycles it asks for.  CHHS_ERR_INVALID_ARG while
 * steps of chhs_step_async are pending (call chhs_wait first). */
chhs_status chhs_profile_step(chhs_t* run, double* ms_out, long long* launches_out, double* units_out);

/* The double-precision smoother on the finest level, alone: npasses colour
 * passes back to back (alternating colours, after one untimed pass) between
 * two CUDA events on the handle's stream; *ms_per_pass = their average
 * duration.  The finest level's (phi, mu, p) are copied aside inside the
 * handle's workspace first and restored afterwards, so the run's state is
 * unchanged bitwise; nothing is allocated.  Blocks until done.  Errors:
 * CHHS_ERR_INVALID_ARG (null pointer, npasses < 1, steps enqueued by
 * chhs_step_async and not yet waited for), CHHS_ERR_CUDA.  For profiling; it
 * has no counterpart in the paper. */
chhs_status chhs_profile_smooth(chhs_t* run, int npasses, double* ms_per_pass);

/* The single-precision finest-level smoothing launch of a mixed-precision
 * handle, alone: in 2D one pre-smoothing tile launch (nu1 sweeps fused with
 * the residual and its restriction), in 3D one colour pass of the
 * correction-form smoother; npasses launches back to back (after one
 * untimed launch) between two CUDA events on the handle's stream, and
 * *ms_per_launch = their average duration.  The run's state is unchanged
 * (the launches' own outputs are scratch that every V-cycle rewrites; the
 * finest correction is put back); nothing is allocated.  Blocks until done.
 * Errors: CHHS_ERR_INVALID_ARG (null pointer, npasses < 1, steps pending, a
 * double-precision handle, or a grid whose finest level is in the one-block
 * tail), CHHS_ERR_CUDA.  For profiling; it has no counterpart in the paper. */
chhs_status chhs_profile_smooth32(chhs_t* run, int npasses, double* ms_per_launch);

/* Measured double-precision throughput of the current device: a kernel of
 * independent fused multiply-add chains on every SM, timed with CUDA events;
 * *tflops_out in TFLOP/s (2 flops per FMA).  The roofline denominator of the
 * double-precision smoother.  Errors: CHHS_ERR_INVALID_ARG (NULL),
 * CHHS_ERR_CUDA.  No counterpart in the paper. */
chhs_status chhs_probe_fp64(double* tflops_out);

/* Measured read bandwidth of the current device's L2: a buffer of `bytes`
 * (1 MiB up to half the L2), allocated and zeroed here, is read once to bring
 * it into the L2 and then `passes` times by every SM with loads that bypass
 * L1, timed with CUDA events; *gbs_out in GB/s.  The roofline denominator of
 * kernels whose working set stays in the L2.  Errors: CHHS_ERR_INVALID_ARG
 * (NULL, passes < 1, bytes out of range), CHHS_ERR_OOM, CHHS_ERR_CUDA.  No
 * counterpart in the paper. */
chhs_status chhs_probe_l2(size_t bytes, int passes, double* gbs_out);

/* Launch shapes of one handle (see chhs_autotune). */
typedef struct {
  int tail_cells;     /* levels with at most this many cells run in the one-block tail */
  int split_threads;  /* double-precision levels with at most this many cells per colour
                         use the three-warp split update (0: never) */
  int tile_threads;   /* threads per tile on the 2D mixed form's levels of at least 512 x 256 cells */
  int coarse_nu1;     /* pre- and post-smoothing sweeps on the levels below the finest (the finest */
  int coarse_nu2;     /* keeps opts->nu1, nu2) */
  int tile_w, tile_h; /* interior of a tile on those levels (even; default 32 x 32 on 512 threads) */
  int norm_f64_per8;  /* mixed form, double-single residual: of every 8 tiles of the residual
                         kernel, how many use double-precision instructions (0..8; default 3), so
                         that the FP64 pipe works beside the single-precision ones */
  int small_tile_w, small_tile_h; /* 2D mixed form: tile interior on the smaller levels */
  int small_tile_threads;         /* (default 16 x 8 cells on 256 threads) and its block size */
  int quad_passes;    /* 3D mixed form: 1 (default) runs the colour passes of levels whose x extent
                         is a multiple of 4 with one thread per four cells of a row (16-byte loads),
                         0 with one thread per cell; the results are the same bit for bit.  Not 0
                         or 1: CHHS_ERR_INVALID_ARG.  A batch's runs always take one cell per thread
                         (chhs_batch_autotune reports 0; chhs_batch_set_tuning ignores it). */
  double ms_per_step; /* the chosen setting's time per step in the trials; -1 when no trial of
                         the setting in force was timed (every candidate failed, or the fastest
                         could not be rebuilt and the original setting was kept) */
} chhs_tuning;

/* Autotuner of the handle's launch shapes and coarse sweep counts: tries
 * candidate settings (where the one-block tail starts; in double precision,
 * up to which level size the split update is used; in the 2D mixed form, the
 * tile block size and tile shape on levels of at least 512 x 256 cells, 32 x
 * 16, 32 x 32 or 64 x 16 cells, and on the smaller levels the same shape or
 * 16 x 8 cells on 256 threads; the
 * sweeps on the levels below the finest: the options' nu1, nu2 or, when both
 * exceed 1, one each), times
 * trial_steps steps of the handle's own problem from its current state with
 * each, keeps the fastest and rebuilds the step graph with it.  The state is
 * restored after every trial and at the end, so the run continues exactly
 * where it was.  Candidates that fail (shared memory too small, a trial that
 * does not converge) are skipped.  Allocates a temporary copy of the state
 * (4 N doubles).  Blocks until done; out (nullable) receives the chosen
 * setting.  Errors: CHHS_ERR_INVALID_ARG (null run, trial_steps < 1, steps
 * enqueued by chhs_step_async and not yet waited for), CHHS_ERR_OOM,
 * CHHS_ERR_CUDA.  The paper has no counterpart (launch shapes are a property
 * of this implementation). */
chhs_status chhs_autotune(chhs_t* run, int trial_steps, chhs_tuning* out);

/* Apply a tuning (for instance one chhs_autotune chose for another run of
 * the same shape) and rebuild the step graph; ms_per_step is ignored.  The
 * state is kept.  Errors: CHHS_ERR_INVALID_ARG (NULL, steps pending, a run
 * of a batch, tail_cells < 1, split_threads < 0, tile_threads not a multiple
 * of 32 in 32..1024, coarse sweep counts < 0 or both 0, tile sides odd or
 * below 2, tiles over 4096 cells (the same for small_tile_*), norm_f64_per8
 * outside 0..8, or a setting
 * the grid cannot take -- the
 * previous tuning is then kept), CHHS_ERR_CUDA. */
chhs_status chhs_set_tuning(chhs_t* run, const chhs_tuning* tuning);

/* Discrete mass (phi^m, 1) = h^d sum phi^m (Section 4, mass conservation). */
chhs_status chhs_mass(chhs_t* run, double* mass_out);

/* E_h(phi^m) (Eq. 2.8) and, if F_out is not NULL, F_h(phi^m, phi^{m-1}) (Eq. 2.9). */
chhs_status chhs_energy(chhs_t* run, double* E_out, double* F_out);

/* Dissipation terms of the last accepted step (Eq. 2.23 and the proof of
 * Theorem 2.1): grad_mu_sq = ||grad_h mu^{m-1/2}||_2^2 and
 * u_sq = ||u^{m-1/2}||_2^2 with the velocity of Eq. 2.3,
 * u = -grad_h p - gamma A_h phi* grad_h mu, on the face grid (zero normal
 * velocity on boundary faces), and div_u_max = max over cells of
 * |div_h u| (Eq. 2.7 makes it zero up to the solver's residual).  Each output
 * is nullable.  Meaningful after at least one chhs_step. */
chhs_status chhs_dissipation(chhs_t* run, double* grad_mu_sq, double* u_sq, double* div_u_max);

/* The velocity of the last accepted step on the face grid (Eq. 2.3,
 * u = -grad_h p - gamma A_h phi* grad_h mu, with the face average A_h of
 * Appendix A.1): ux[c] is the x-component on the face between cell c and its
 * +x neighbour, uy and uz likewise for +y and +z, each an array of N values
 * in the layout of phi; faces on the domain boundary hold 0 (no flux).  uz is
 * ignored in 2D (may be NULL) and required in 3D.  Device pointers if
 * on_device, else host memory owned by the caller.  Blocks until the copy is
 * done.  Meaningful after at least one chhs_step.  Errors:
 * CHHS_ERR_INVALID_ARG (null run, ux, uy, or uz in 3D; steps enqueued by
 * chhs_step_async and not yet waited for), CHHS_ERR_CUDA. */
chhs_status chhs_velocity(chhs_t* run, double* ux, double* uy, double* uz, int on_device);

/* Copy out phi^m (the latest accepted step). */
chhs_status chhs_get_phi(chhs_t* run, double* out, int on_device);

/* Copy out the full state: phi^m, phi^{m-1}, mu^{m-1/2}, p^{m-1/2} (each
 * nullable; p has zero mean).  With chhs_set_state this is a checkpoint. */
chhs_status chhs_get_state(chhs_t* run, double* phi, double* phi_prev, double* mu, double* p,
                           int on_device);

/* Restore a state written by chhs_get_state; mu and p may be NULL (then zero). */
chhs_status chhs_set_state(chhs_t* run, const double* phi, const double* phi_prev, const double* mu,
                           const double* p, int on_device);

/* Largest grid (in cells) chhs_energy_noalloc accepts. */
#define CHHS_NOALLOC_MAX_CELLS (1 << 22)

/* Mass and energies of device-resident fields without allocating memory.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc, such as a host framework whose memory pool owns the device, or
 * a latency-bound loop that cannot take the device-wide synchronisation an
 * allocation may cause.  It needs no handle.
 *
 * phi_dev, psi_dev: device pointers to dim-dimensional grids of n[0] x n[1]
 * (x n[2]) doubles, x fastest (psi_dev NULL means psi = phi).  Outputs
 * (nullable host pointers): mass_out, E_out and F_out, the same three
 * quantities that chhs_mass and chhs_energy report for a handle's phi^m and
 * phi^{m-1}, here for phi and psi.  Work is ordered on cuda_stream (NULL =
 * the legacy default stream), and the call waits for that stream to finish
 * before it returns (the sums are read back to the host).
 *
 * Scratch: a fixed device array of about 0.8 MB inside the library, held by
 * every GPU that loads it until the process exits; grids above
 * CHHS_NOALLOC_MAX_CELLS cells return CHHS_ERR_INVALID_ARG, as do a
 * dimension other than 2 or 3, a size below 1, h <= 0 or eps <= 0.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (on different
 * streams, or from several host threads) race and must be serialised by the
 * caller.  Returns CHHS_ERR_CUDA if a CUDA call fails; a launch failure is
 * read with cudaGetLastError, which also reports (and clears) an error that
 * an earlier, unrelated launch left on the calling thread. */
chhs_status chhs_energy_noalloc(int dim, const int n[3], double h, double eps, const double* phi_dev,
                                const double* psi_dev, void* cuda_stream, double* mass_out,
                                double* E_out, double* F_out);

/* ------------------------------------------------------------------ serving
 * A request loop for many independent runs on one GPU (continuous batching).
 * A worker thread admits submitted runs first come, first served, whenever an
 * active slot is free and the run's hierarchy (chhs_workspace_bytes) fits in
 * a device memory pool allocated once at creation; each active run has its
 * own stream and advances steps_per_slice steps at a time, so runs overlap on
 * the device, and between slices finished runs are retired (their memory
 * returns to the pool) and waiting runs admitted.  Each run computes exactly
 * what chhs_create + chhs_set_phi + chhs_step would compute for it alone. */
typedef struct chhs_server chhs_server_t;

typedef struct {
    int dim;               /* 2 or 3 */
    int n[3];              /* grid size (n[2] ignored in 2D) */
    double h, eps, gamma, dt;
    int nsteps;            /* time steps to take */
    int precision;         /* as chhs_opts.precision; other options are the defaults */
    const double* phi0;    /* host, copied at submit: phi^0 */
    const double* phi_prev;/* host, copied at submit, or NULL: phi^{-1} = phi^0 */
} chhs_request;

/* Start a server with a device pool of pool_bytes, at most max_active runs
 * on the GPU at once and steps_per_slice steps per launch slice. */
chhs_status chhs_server_create(size_t pool_bytes, int max_active, int steps_per_slice, chhs_server_t** out);

/* Queue a run; *id_out identifies it.  INVALID_ARG for a bad request.  A run
 * whose hierarchy exceeds the whole pool finishes with CHHS_ERR_OOM. */
chhs_status chhs_server_submit(chhs_server_t* sv, const chhs_request* req, long long* id_out);

/* Block until run id is done or timeout_s seconds pass (then
 * CHHS_ERR_NOT_CONVERGED is returned and the run keeps going).  timeout_s
 * above 1e6 (infinity included) waits without a limit; a negative or NaN
 * timeout_s, an unknown id or a NULL server give CHHS_ERR_INVALID_ARG. */
chhs_status chhs_server_wait(chhs_server_t* sv, long long id, double timeout_s);

/* Result of run id: *done = 0 while it runs; when done, its status, V-cycles
 * summed over its steps, phi at its last step (host, n cells; nullable; NaN
 * in every cell for a run refused before it held a state, e.g. one whose
 * hierarchy exceeds the whole pool) and times3 = {submit, admit, done} in
 * seconds of a monotonic clock (nullable). */
chhs_status chhs_server_result(chhs_server_t* sv, long long id, int* done, int* status, int* vcycles,
                               double* phi_out, double* times3);

/* Forget a finished run's result (CHHS_ERR_INVALID_ARG for a run not yet
 * done or an unknown id).  A thread waiting on the run in chhs_server_wait
 * returns CHHS_OK. */
chhs_status chhs_server_release(chhs_server_t* sv, long long id);

/* Runs waiting, on the GPU and finished, and pool bytes in use (each nullable). */
chhs_status chhs_server_stats(chhs_server_t* sv, int* queued, int* active, int* done, size_t* pool_in_use);

/* Stop the worker (runs still active are abandoned) and free everything. */
void chhs_server_destroy(chhs_server_t* sv);

/* ------------------------------------------------------------------ batches
 * Many independent runs of uneven size stepped together: one CUDA graph per
 * time step of all the runs, in which every launch covers one kernel of one
 * multigrid level for all runs that have that level (the V-cycle's level l is
 * one launch over every run's level l; all runs' coarse tails are one launch
 * of one block per run; all runs' stopping norms are one launch), with the
 * V-cycle loop on the device running while any run is still iterating.  A
 * run that has converged drops out of the launches, so each run takes
 * exactly the V-cycles, and computes exactly the bits, that it does alone
 * (chhs_create with the same options).  Batches use the mixed-precision form
 * (opts->precision must be 1; NULL opts = the defaults with precision 1).
 * The paper has no counterpart: batching is a property of this
 * implementation. */
typedef struct chhs_batch chhs_batch_t;

/* One run of a batch: the chhs_create arguments (Section 2). */
typedef struct {
    int dim;      /* 2 or 3, the same for every run of a batch */
    int n[3];     /* grid size (n[2] ignored in 2D) */
    double h, eps, gamma, dt;
} chhs_run_desc;

/* Device bytes chhs_batch_create allocates for these runs (0 for invalid
 * arguments: nruns < 1, a run that chhs_create would refuse, runs of
 * different dimension, options other than the mixed-precision form). */
size_t chhs_batch_workspace_bytes(int nruns, const chhs_run_desc* runs, const chhs_opts* opts);

/* Create a batch of nruns runs (arrays: runs[nruns]) on cuda_stream (NULL =
 * a stream the batch creates).  Allocates every run's hierarchy in one
 * cudaMalloc and the launch tables in another, and captures the batch's
 * step graph.  Each run starts at phi^0 = phi^{-1} = 0.  Errors:
 * CHHS_ERR_INVALID_ARG (as chhs_batch_workspace_bytes, or a run whose
 * coarse tail needs more shared memory than a block has), CHHS_ERR_OOM,
 * CHHS_ERR_CUDA. */
chhs_status chhs_batch_create(int nruns, const chhs_run_desc* runs, const chhs_opts* opts, void* cuda_stream,
                              chhs_batch_t** out);

/* Number of runs of the batch (0 for NULL). */
int chhs_batch_size(const chhs_batch_t* batch);

/* The handle of run r (0 <= r < nruns; NULL otherwise), owned by the batch.
 * Use it with chhs_set_phi, chhs_set_state, chhs_get_phi, chhs_get_state,
 * chhs_mass, chhs_energy, chhs_dissipation and chhs_velocity (in stream
 * order on the batch's stream); chhs_step, chhs_step_async and
 * chhs_autotune refuse it (CHHS_ERR_INVALID_ARG), and chhs_destroy ignores
 * it: the batch frees it. */
chhs_t* chhs_batch_run(chhs_batch_t* batch, int r);

/* Advance every run nsteps time steps; blocks until done.  Per run (arrays
 * of nruns, each nullable): status_out (a chhs_status: CHHS_OK, or
 * CHHS_ERR_NOT_CONVERGED / CHHS_ERR_DIVERGED for a run that stopped at a
 * failed step, its phi^m and phi^{m-1} then at the last accepted step, as
 * chhs_step leaves them), vcycles_out (V-cycles summed over the steps) and
 * resid_out (the last stopping norm).  Returns CHHS_OK if every run
 * advanced, else the first failing run's status (chhs_batch_last_error
 * names it); the other runs advance either way. */
chhs_status chhs_batch_step(chhs_batch_t* batch, int nsteps, int* status_out, int* vcycles_out, double* resid_out);

/* Apply launch settings to every run of the batch and rebuild its step
 * graph; the runs' states are kept.  Of chhs_tuning the batch takes
 * tail_cells, coarse_nu1, coarse_nu2 and norm_f64_per8 (the same for all its
 * runs) and, in 2D, tile_w, tile_h and tile_threads for the per-run tile
 * launches of its large levels (default 32 x 32 cells on 512 threads; the
 * batched launch of the small levels keeps 32 x 16 on 512); the other fields
 * are ignored.  Errors:
 * CHHS_ERR_INVALID_ARG (NULL, tail_cells < 1, coarse sweep counts < 0 or both
 * 0, norm_f64_per8 outside 0..8, a tile as chhs_set_tuning refuses, or a
 * setting some run cannot take -- the previous setting is then kept),
 * CHHS_ERR_CUDA.  The paper has no counterpart. */
chhs_status chhs_batch_set_tuning(chhs_batch_t* batch, const chhs_tuning* tuning);

/* Autotuner of the batch: times trial_steps steps of all its runs from
 * their current states with each candidate setting (where the one-block
 * tail starts: levels of at most 256 / 1024 / 4096 cells in 2D, 64 / 512 /
 * 4096 in 3D; the sweeps below the finest level: the options' nu1, nu2 or,
 * when both exceed 1, one each; in 2D the large levels' tile shape, 32 x 16,
 * 32 x 32 or 64 x 16 cells), keeps the fastest and rebuilds the batch's
 * graph with it.  Every run's state is restored after each trial and at the
 * end.  Candidates that fail are skipped.  Allocates a temporary copy of
 * all states (4 doubles per cell).  out (nullable) receives the setting
 * (ms_per_step -1 if the fastest could not be rebuilt and the original was
 * kept).  Errors: CHHS_ERR_INVALID_ARG (NULL batch, trial_steps < 1),
 * CHHS_ERR_OOM, CHHS_ERR_CUDA.  The paper has no counterpart. */
chhs_status chhs_batch_autotune(chhs_batch_t* batch, int trial_steps, chhs_tuning* out);

/* Launches of the batch's step graph: per V-cycle and per step outside the
 * V-cycle loop, whatever the number of runs (plus one batched norm launch
 * per iteration of the loop).  With opts.max_inner > 1 each run takes the
 * V-cycles between norms that its own norms predict, as it would alone: the
 * graph runs a 2nd (3rd) batched V-cycle in an iteration when some run asks
 * for one, gated off for the others. */
chhs_status chhs_batch_launch_counts(const chhs_batch_t* batch, int* per_vcycle, int* per_step);

/* One time step of every run launched kernel by kernel (no graph) with a
 * CUDA event pair around each batched launch; adds into the caller's arrays
 * of CHHS_K_COUNT entries the device milliseconds and launches per kernel
 * kind (as chhs_profile_step).  For profiling: the host reads the "any run
 * iterating" flags after every norm.  Errors: CHHS_ERR_INVALID_ARG (NULL
 * argument), CHHS_ERR_CUDA. */
chhs_status chhs_batch_profile_step(chhs_batch_t* batch, double* ms_out, long long* launches_out);

/* Text of the batch's last error ("" if none). */
const char* chhs_batch_last_error(const chhs_batch_t* batch);

/* Free the batch, its runs and its device memory.  NULL is a no-op. */
void chhs_batch_destroy(chhs_batch_t* batch);

/* Number of multigrid levels of the handle (finest included). */
int chhs_num_levels(const chhs_t* run);

/* Release the handle and its device memory (not a caller's arena). NULL is a no-op. */
void chhs_destroy(chhs_t* run);

/* Text of the last error of this handle ("" if none); valid until the next call. */
const char* chhs_last_error(const chhs_t* run);

#ifdef __cplusplus
}
#endif

#endif /* CHHS_H */
