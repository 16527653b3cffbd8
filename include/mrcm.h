/*
 * mrcm.h -- C ABI of a GB300 (sm_103a) implementation of the Multiscale Robin
 * Coupled Method with Oversampling and Smoothing (MRCM-OS, arXiv 2404.13811)
 * for single-phase Darcy flow  u = -K grad p,  div u = f  (Sec. 2, Eqs. (1a)-(1d)).
 *
 * Call order (enforced; an out-of-order call returns MRCM_ERR_STATE):
 *   mrcm_create / mrcm_create_batch
 *   mrcm_build_basis       Algorithm 1, Steps 1-4 (and 6 when alpha_smooth != alpha_basis);
 *                          calling it again restarts the pipeline from the inputs
 *   mrcm_solve_interface   Algorithm 1, Step 5
 *   mrcm_smooth            Algorithm 1, Step 7 (any number of calls; additive in n_steps)
 *   mrcm_fluxes            read the current solution (any time after mrcm_solve_interface)
 *   mrcm_destroy
 *
 * Conventions
 *   Cells are addressed x fastest: cell (ix, iy, iz) has flat index
 *   ix + n[0] * (iy + n[1] * iz).  Arrays of cell data are dense in that order.
 *   Sides are numbered x-, x+, y-, y+, z-, z+ (side id = 2 * axis + s).
 *   Velocities are returned per cell and per side as the OUTWARD normal
 *   velocity of that cell (array [ncells][2 * dim]); across the subdomain
 *   skeleton they come from each cell's own subdomain and are double-valued,
 *   as in the method (Sec. 2.1).
 *   Every call runs asynchronously on the CUDA stream given at creation,
 *   except where a call states that it synchronises.
 *   Handles are not thread safe.  No exception or abort crosses this ABI:
 *   every entry point returns 0 (MRCM_OK) or a negative MRCM_ERR_* code and
 *   mrcm_last_error() describes the last failure.
 *   Device memory for factors, bases, interface system and state is owned by
 *   the handle (allocated in mrcm_create*, freed in mrcm_destroy).  Inputs are
 *   copied at creation; output buffers belong to the caller.
 */
#ifndef MRCM_H
#define MRCM_H

#ifdef __cplusplus
extern "C" {
#endif

#define MRCM_OK 0
#define MRCM_ERR_BAD_INPUT (-1)      /* invalid sizes, K <= 0 or not finite, partition mismatch */
#define MRCM_ERR_STATE (-2)          /* call out of order */
#define MRCM_ERR_CUDA (-3)           /* a CUDA runtime call failed */
#define MRCM_ERR_NOT_SPD (-4)        /* non-positive pivot in a local factorisation */
#define MRCM_ERR_NO_CONVERGENCE (-5) /* iterative refinement did not reach ir_tol in max_ir steps */
#define MRCM_ERR_SINGULAR (-6)       /* zero pivot in the interface factorisation */
#define MRCM_ERR_UNSUPPORTED (-7)    /* a size or option this build does not handle */
#define MRCM_ERR_NOMEM (-8)          /* device allocation failed */
#define MRCM_ERR_TIMEOUT (-9)        /* a kernel's bounded wait (for a staged copy) ran out; the kernel
                                        returned without its result (the context stays usable) */
#define MRCM_ERR_CHECK (-10)         /* bounds-check build only (libmrcm_check.so, compiled with
                                        -DMRCM_CHECK=1): a kernel's check of a shared-memory layout,
                                        a bulk copy, a pivot record or a write index failed; the
                                        guarded access was skipped; mrcm_last_error names the site,
                                        the block and the value */

#define MRCM_NEUMANN 0   /* u.n = value on the side (Eq. (1d)) */
#define MRCM_DIRICHLET 1 /* p = value on the side (Eq. (1c)) */

#define MRCM_P0 0 /* piecewise-constant interface spaces per coarse edge/face (Sec. 2.1) */
#define MRCM_P1 1 /* piecewise-linear: {1, t} on edges (2D), {1, s, t} on faces (3D) */

#define MRCM_FP64 0  /* local factorisations and solves in FP64 */
#define MRCM_MIXED 1 /* FP32 local factor/solves + FP64 residuals (iterative refinement) */

/* Where the particular problem of Algorithm 1 Step 4 is posed (mrcm_params.particular). */
#define MRCM_PARTICULAR_OMEGA 0 /* on Omega_i with its own factor (Eqs. (111dbar)-(122dbar); the paper's method) */
#define MRCM_PARTICULAR_HAT 1   /* variant, not in the paper: on hat-Omega_i with the basis factor */

/* Cartesian grid: cells per axis and cell size per axis (dim = 2 or 3). */
typedef struct {
    int dim;
    int n[3];
    double h[3];
} mrcm_grid;

/* Boundary data per side (x-, x+, y-, y+, z-, z+): kind MRCM_NEUMANN with the
 * outward normal velocity z, or MRCM_DIRICHLET with the pressure g; constant
 * per side (Eqs. (1c)-(1d)). */
typedef struct {
    int kind[6];
    double value[6];
} mrcm_bc;

/* Non-overlapping partition into blocks of sub[a] cells (must divide n[a]);
 * each block Omega_i is oversampled by `overlap` cells per side, clipped at
 * the domain boundary (hat-Omega_i, Sec. 2.1).  Smoothing requires
 * 0 < 2 * overlap < sub[a]. */
typedef struct {
    int sub[3];
    int overlap;
} mrcm_partition;

/* Method parameters.
 *   space        MRCM_P0 / MRCM_P1: the polynomial space used for the Robin
 *                data lambda^k on d hat-Omega_i and for M_H = V_H (Prop. 1
 *                needs the same number of functions per edge in all three).
 *   alpha_basis  Robin parameter for the basis and particular problems:
 *                beta = alpha H / K_H, K_H the harmonic mean of the two
 *                cells at the face, H the subdomain width normal to the face
 *                (Sec. 2.1, after Eq. (genRobin)).
 *   alpha_smooth the same for the smoothing solves (Sec. 3 uses 1).
 *   precision    MRCM_FP64 or MRCM_MIXED.
 *   ir_tol       relative residual (inf-norm; Jacobi-scaled for the local
 *                solves, row-equilibrated for the interface solve) that
 *                refinement must reach (mixed local solves and
 *                the interface solve).  3D local solves refine on to their
 *                residual floor: they stop at 1e-3 ir_tol, or below ir_tol
 *                once the residual no longer halves per step.
 *   max_ir       maximum refinement steps.
 *   particular   MRCM_PARTICULAR_OMEGA (0): Step 4 as in the paper, the
 *                particular problem (sources f, g, z, zero Robin data on
 *                Gamma_i) on Omega_i with an Omega_i factor of its own.
 *                MRCM_PARTICULAR_HAT (1): a variant that is not in the paper:
 *                the same sources with zero Robin data on the sides of
 *                hat-Omega_i inside Omega, solved with the kept basis factor
 *                as one more right-hand side of the basis solves, and
 *                restricted to Omega_i (pressure, Gamma_i fluxes and face
 *                pressures) like the basis functions.  No Omega_i operator is
 *                assembled or factored.  It shifts the affine local space and
 *                so changes the result (for overlap 0 the two coincide).
 *                2D and 3D (the adjoint, like the method's, 2D).
 *                Other values: MRCM_ERR_BAD_INPUT. */
typedef struct {
    int space;
    double alpha_basis;
    double alpha_smooth;
    int precision;
    double ir_tol;
    int max_ir;
    int particular;
} mrcm_params;

typedef struct mrcm_handle mrcm_handle;

/* Creates a handle for one problem.
 *   K, f         cell permeability (> 0, finite) and source density f of
 *                Eq. (1b) (the cell equation uses f * cell volume), [ncells].
 *   device_ptrs  0: K and f are host pointers; 1: device pointers.
 *   cuda_stream  cudaStream_t on which all work of this handle runs (0 = legacy default).
 * Copies K and f, plans the decomposition, colours and interface ordering,
 * and allocates all device memory of the handle.  Synchronises the stream.
 * On failure *out (when out is not NULL) still receives a handle that holds
 * only the error text for mrcm_last_error; release it with mrcm_destroy.
 * Argument checks (grid, partition, boundary kinds, params, host K and f)
 * run on the host before any device work. */
int mrcm_create(const mrcm_grid* grid, const double* K, const double* f, const mrcm_bc* bc,
                const mrcm_partition* part, const mrcm_params* params, int device_ptrs,
                void* cuda_stream, mrcm_handle** out);

/* Creates one handle for `count` independent problems (an ensemble).  Arrays
 * grids, bcs, parts have `count` entries; K[m], f[m] point at member m's
 * cells.  All members share `params`.  Every later call processes all
 * members together: one launch per kernel over all subdomains of all
 * members.  Failure behaviour as mrcm_create. */
int mrcm_create_batch(int count, const mrcm_grid* grids, const double* const* K,
                      const double* const* f, const mrcm_bc* bcs, const mrcm_partition* parts,
                      const mrcm_params* params, int device_ptrs, void* cuda_stream,
                      mrcm_handle** out);

/* Algorithm 1, Steps 1-4 (Sec. 2.1-2.2, Sec. 3): per subdomain, assemble and
 * factor the hat-Omega_i operator, solve the N_i informed-space problems of
 * Eq. (oversampling_problem), keep the restriction of each solution to
 * Omega_i (Remark, Sec. 2.2) and its flux / face-pressure traces on Gamma_i,
 * factor the Omega_i operator and solve the particular problem of Eqs.
 * (111dbar)-(122dbar) (with mrcm_params.particular = MRCM_PARTICULAR_HAT the
 * particular problem is instead one more right-hand side of the hat-Omega_i
 * solves, restricted like them, and no Omega_i operator is factored).  When
 * alpha_smooth != alpha_basis it also factors the smoothing operator
 * (Step 6). */
int mrcm_build_basis(mrcm_handle* h);   /* any stage; restarts the pipeline */

/* Algorithm 1, Step 5: assembles the interface rows of Eqs.
 * (int_ujump)-(int_pjump) tested with all of M_H x V_H, solves them for the
 * coefficients X (FP32 factorisation + FP64 iterative refinement to ir_tol;
 * when the refinement stops contracting, restarted FP64 GMRES preconditioned
 * by the same FP32 factorisation continues from its iterate, and mrcm_run
 * then runs the problem eagerly instead of replaying a captured step),
 * and assembles u = ubar + sum_j X_j Phi_j, p = pbar + sum_j X_j Psi_j
 * (Eqs. (addu), (addp), (uhatphat)).  Pure-Neumann members are solved in the
 * gauge X^0_0 = 0 and reported with zero-mean pressure.  Synchronises the
 * stream (it reads the refinement residual). */
int mrcm_solve_interface(mrcm_handle* h);

/* Algorithm 1, Step 7 (Sec. 3, Eqs. (sm_1)-(sm_2)): n_steps smoothing steps.
 * Colours c = sum_a (i_a mod 2) 2^a are visited in increasing order; each
 * subdomain of a colour takes Robin data lambda = -beta u.n + pi on
 * d hat-Omega_i \ d Omega from the current solution (beta with
 * alpha_smooth), solves on hat-Omega_i with the factor kept from Step 1 or 6,
 * and overwrites (u, p) on Omega_i.  smooth(a); smooth(b) == smooth(a + b). */
int mrcm_smooth(mrcm_handle* h, int n_steps);

/* One whole step -- mrcm_build_basis + mrcm_solve_interface + mrcm_smooth(n_steps)
 * -- for all members.  use_graph = 0: the eager calls.  use_graph = 1: the
 * first call runs eagerly (that fixes the number of interface refinement
 * steps), captures the whole step (every kernel of every phase, all members)
 * into a CUDA graph on the handle's stream and from then on replays it with
 * one graph launch; after each replay the interface residual and the local
 * status are read back (the call synchronises) and MRCM_ERR_NO_CONVERGENCE
 * is returned if the replayed refinement (the eager solve's number of steps)
 * leaves an interface residual above 1e3 ir_tol.
 * The graph is recaptured when n_steps changes.  Inputs are the ones given
 * at creation (the batching form of the method: uneven subdomains and whole
 * ensembles in one submission). */
int mrcm_run(mrcm_handle* h, int n_steps, int use_graph);

/* Writes member `member`'s current solution: u_cellfaces [ncells][2 * dim]
 * outward normal velocities, p_cells [ncells] (either may be NULL).
 * device_ptrs 0: host buffers (the call synchronises); 1: device buffers. */
int mrcm_fluxes(mrcm_handle* h, int member, double* u_cellfaces, double* p_cells,
                int device_ptrs);

/* mrcm_fluxes for callers that cannot allocate device memory when they read
 * results: mrcm_fluxes allocates a device staging buffer for host outputs and
 * reduces the pure-Neumann pressure gauge into scratch owned by the handle,
 * which fails or is not allowed where the device memory is already held by
 * another framework's caching allocator or inside a loop that must not
 * allocate.  This entry point (the paper has no counterpart; it is part of
 * this library's output interface) writes member `member`'s solution into
 * caller DEVICE buffers u_cellfaces [ncells][2 * dim] and p_cells [ncells]
 * (either may be NULL), with the same values as mrcm_fluxes, and allocates
 * nothing: its multi-block gauge reduction uses a file-scope static device
 * array of 1024 partial sums (8 KB, held by every device that loads the
 * library until the process exits), one per block of 4096 cells, so a member
 * may have at most 4194304 cells (MRCM_ERR_UNSUPPORTED otherwise).  The
 * device on which the handle was created must be the current device
 * (MRCM_ERR_BAD_INPUT otherwise).  The first call on a device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture, and not from two host threads at once.  Every
 * call shares the array: calls that overlap on the GPU (other streams, other
 * handles) race on it.  Runs on the handle's stream and does not synchronise. */
int mrcm_fluxes_static(mrcm_handle* h, int member, double* u_cellfaces, double* p_cells);

/* Replaces the permeability of every member (concatenated in member order,
 * [total cells]): values are K (is_log = 0; > 0 and finite) or log K
 * (is_log = 1; finite).  device_ptrs 0: host pointer; 1: device pointer.
 * Recomputes the face coefficients of Sec. 2.2 and returns the handle to
 * the created stage: mrcm_build_basis must run next (a captured step of
 * mrcm_run is dropped and captured again).  MRCM_ERR_BAD_INPUT when a value
 * is out of range (checked on the host for host input, on the device for
 * device input; the handle's K is then not usable).  Synchronises. */
int mrcm_set_permeability(mrcm_handle* h, const double* values, int is_log, int device_ptrs);

/* Differentiation form: reverse mode of the whole computation that produced
 * the current solution -- basis problems (Eq. (oversampling_problem)),
 * particular problems (Eqs. (111dbar)-(122dbar)), interface system (Eqs.
 * (int_ujump)-(int_pjump)), superposition (Eqs. (addu), (addp)) and every
 * smoothing step applied since the last interface solve (Eqs.
 * (sm_1)-(sm_2)) -- with respect to log K of every cell.
 *   gp    [total cells] dL/dp and gu [total cells][2 * dim] dL/du of a
 *         scalar L of the returned solution (member order, the layout of
 *         mrcm_fluxes); either may be NULL (zero).
 *   g_logK [total cells] output dL/dlog K.
 *   device_ptrs 0: host arrays (the call synchronises); 1: device arrays.
 * The kept factors serve the transposed local solves (the operators are
 * symmetric); the local forward solutions are recomputed, not stored; the
 * smoothing steps are replayed once to record the state before each colour
 * pass (n_steps x 2^dim states of (p, u), allocated by the handle on first
 * use); the interface system is solved transposed with its FP32 slab factors
 * and FP64 refinement.  Leaves the current solution unchanged.
 * MRCM_ERR_UNSUPPORTED for a member with no Dirichlet side (its pressure is
 * fixed only up to a constant) and for 3D problems.  Needs a solution
 * (MRCM_ERR_STATE). */
int mrcm_adjoint(mrcm_handle* h, const double* gp, const double* gu, double* g_logK, int device_ptrs);

/* The same reverse pass with the seeds in (velocity, pressure) order and host
 * arrays: dL_du [total cells][2 * dim], dL_dp [total cells] (either may be
 * NULL), dL_dlogK [total cells] output; all caller-owned host memory (the
 * call synchronises).  Returns and errors as mrcm_adjoint. */
int mrcm_backward(mrcm_handle* h, const double* dL_du, const double* dL_dp, double* dL_dlogK);

/* Counters of the last calls: ints[0] = number of subdomains (all members),
 * ints[1] = interface unknowns, ints[2] = interface refinement steps of the
 * last solve, ints[3] = largest local refinement count of the last
 * build/smooth call, ints[4] = local solves performed so far, ints[5] = the
 * slab inverses of the interface reduction (0 blocked Gauss-Jordan, 1 LU, 2
 * register-resident Gauss-Jordan: chosen per handle by the autotuner below),
 * ints[6] = 1 when the last interface solve needed the GMRES fallback,
 * ints[7] = where the slab-inverse choice came from (0 not made or not a
 * choice: slabs larger than 768 unknowns always use the LU; 1 the tuning
 * cache; 2 measured on this handle's first interface solve); dbl[0] = last
 * interface relative residual, dbl[1] / dbl[2] / dbl[3] = the measured device
 * ms of variants 0 / 1 / 2 (factorisation + refinement to ir_tol; 0 when not
 * measured).  Either pointer may be NULL; at most nints / ndbl entries are
 * written.
 *
 * Autotuner.  The slab inverses of the interface reduction are computed by
 * one of: Gauss-Jordan elimination with the slab held in registers across a
 * cluster of CTAs (one pivot column per step, slabs of at most 768
 * unknowns); blocked Gauss-Jordan elimination in shared memory (slabs of at
 * most 256 unknowns); an LU factorisation followed by the inverse columns
 * (any size).  The first mrcm_solve_interface of a handle (and the first
 * after mrcm_set_permeability) times every admissible variant -- device time
 * of the factorisation and of the refinement steps it needs -- and keeps the
 * fastest one that reaches ir_tol (the LU when none does); a later
 * refinement that stalls with a Gauss-Jordan variant switches the handle to
 * the LU.  With the environment variable MRCM_TUNE_CACHE naming a JSON file,
 * the choice is read from it by shape class (dimension, slab size, slab and
 * level counts, members, precision, space, ir_tol) when present and written to
 * it after a measurement.
 *
 * Per-call metrics.  With the environment variable MRCM_METRICS naming a file
 * (or "stderr"), every outermost call among mrcm_build_basis,
 * mrcm_solve_interface, mrcm_smooth, mrcm_run and mrcm_adjoint appends one
 * JSON line to it: the call, its return code, its host wall time in ms (the
 * calls synchronise, so this includes their device work), the counters above
 * and the slab-inverse choice with its source and measured times.  Calls made
 * inside mrcm_run write no line of their own. */
int mrcm_stats(const mrcm_handle* h, int* ints, int nints, double* dbl, int ndbl);

/* Device-time profiling of the calls above.  enable = 1 starts recording a
 * pair of CUDA events around every kernel group on the handle's stream (and
 * clears what was recorded); enable = 0 stops.  Phases:
 *   0 local basis / particular / smoothing-factor kernels (mrcm_build_basis)
 *   1 interface assembly, equilibration and slab factorisation
 *   2 interface refinement sweeps (residual, forward, backward, update)
 *   3 assembly of the MRCM-O solution
 *   4 smoothing colour phases (mrcm_smooth)
 *   5 replays of a captured step (mrcm_run with use_graph = 1)
 *   6 the slab LU inverses alone (a part of phase 1)
 * mrcm_timings synchronises the stream and writes, for each of the first n
 * phases (n <= 7), the summed device time in ms (ms[i]) and the number of
 * kernel launches of this library in that phase (launches[i]); either
 * pointer may be NULL (phase 5 counts graph launches; phase 6 launches are
 * also counted in phase 1).  Launches are counted whether or not profiling
 * is enabled. */
int mrcm_profile(mrcm_handle* h, int enable);
int mrcm_timings(mrcm_handle* h, double* ms, long long* launches, int n);

/* Measurement support (the paper has no counterpart): the sustained FMA
 * throughput of the current device in FP32 and in FP64, in TFLOP/s (2 flops
 * per FMA), from independent FMA chains on every SM timed with CUDA events
 * on cuda_stream (the median of three runs; about a second of device time in
 * all).  Used as the denominators of the FP32 / FP64 rooflines.  Allocates a
 * small device buffer while it runs; changes no device setting.  Either
 * pointer may be NULL (that measurement is skipped).  Synchronises. */
int mrcm_measure_fma_peaks(double* fp32_tflops, double* fp64_tflops, void* cuda_stream);

int mrcm_destroy(mrcm_handle* h);

/* Text of the last error of this handle ("" if none); valid until the next call. */
const char* mrcm_last_error(const mrcm_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_H */
