/*
 * vdp.h -- C ABI of libvdp, a GB300 (sm_103a) solver for the variable-coefficient pressure
 * Poisson equation of a low-Mach variable-density flow,
 *
 *        div( (1/rho) grad p ) = f ,                                   (Sec. 3.4 of [1])
 *
 * on a uniform, triply periodic, staggered grid (Sec. 3.1 and Sec. 3.2 case 1 of [1]), or on the
 * inflow-outflow duct of Sec. 3.2 case 2 (periodic y, z; see vdp_create_bc).  Also: the steps
 * either side of the solve in a projection substep (App. A), a multigrid V-cycle, and a
 * constant-coefficient inverse.
 *
 * [1] H. Pouransari, M. Mortazavi, A. Mani, "Parallel variable-density particle-laden turbulence
 *     simulation", CTR Annual Research Briefs (arXiv:1601.05448).
 *
 * Discretisation (the paper gives only the continuous equation and "staggered, second order"):
 *   cell (i,j,k), index c = i + nx*(j + ny*k) (x fastest), spacing h_d = L_d/n_d, periodic wrap
 *   (in the duct the faces at the two x ends carry no coefficient);
 *   1/rho on a face = 1 / (arithmetic mean of the two adjacent cell-centre densities) -- the
 *   averaging App. B of [1] uses to move rho off the cell centres;
 *   (A p)_c = sum_d b_d[c+e_d](p[c+e_d]-p[c]) - b_d[c](p[c]-p[c-e_d]),
 *   b_d[c] = 2/(rho[c-e_d]+rho[c]) / h_d^2 on the low d-face of cell c.
 * Compatibility (App. A of [1], the constant chi'): on the periodic box the left side integrates
 * to zero, so the solver replaces f by f - <f> (cell mean) and reports <f>.  The pressure is
 * returned with zero cell mean.  Convergence: relative L2 residual
 * ||(f - <f>) - A p||_2 / ||f - <f>||_2 <= tol, evaluated in FP64 from p itself.
 *
 * Memory conventions: every field is a contiguous array of nx*ny*nz doubles in the layout above.
 * Pointers passed to vdp_set_density / vdp_solve may be device pointers (e.g. torch CUDA
 * tensors' data_ptr()) or host pointers (pageable or pinned); host data is staged through
 * library-owned device buffers on the context's stream; device pointers must be 16-byte
 * aligned (VDP_EINVAL otherwise).  The caller keeps ownership of all
 * arrays it passes; the library never frees them and keeps no caller pointer after a call
 * returns.  All work is ordered on the context's stream (vdp_opts.stream; NULL = the legacy
 * default stream) and every call below returns only after its work has finished.
 *
 * Threading: a context may be used by one host thread at a time; distinct contexts are
 * independent.  Errors: functions return a vdp_status; vdp_strerror() names it.  No call
 * aborts the process.
 */
#ifndef VDP_H
#define VDP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VDP_OK = 0,
  VDP_EINVAL = 1,      /* bad argument, or call out of order (solve before set_density) */
  VDP_ENOMEM = 2,      /* device allocation failed, or a batch/HBM budget is exhausted */
  VDP_EDENSITY = 3,    /* rho has an entry <= 0, NaN or Inf */
  VDP_ENOTCONV = 4,    /* max_iter reached; p holds the best iterate (zero mean) */
  VDP_EBREAKDOWN = 5,  /* Krylov breakdown (non-positive curvature or non-finite value) */
  VDP_ETIMEOUT = 6,    /* a bounded device-side wait gave up; the context stays usable */
  VDP_ECUDA = 7        /* a CUDA runtime call failed (the message is in vdp_last_cuda_error) */
} vdp_status;

typedef enum {
  VDP_FP64 = 0,        /* FP64 everywhere */
  VDP_MIXED = 1,       /* FP32 inner Krylov with FP32 face coefficients, FP64 refinement */
  VDP_MIXED_BF16 = 2   /* as VDP_MIXED with BF16-stored face coefficients (ablation) */
} vdp_precision;

/* Boundary condition in x (vdp_create_bc).  y and z are always periodic. */
typedef enum {
  VDP_BC_PERIODIC = 0,  /* the triply periodic box (Sec. 3.2, configuration 1) */
  VDP_BC_DUCT = 1       /* the inflow-outflow duct (Sec. 3.2, configuration 2): no pressure flux
                           through the two x ends (homogeneous Neumann; the paper does not state
                           the pressure condition, this is the reading taken).  The faces at
                           x = 0 and x = Lx carry no coefficient, and the spectral passes transform
                           the even extension of each x row (2 nx points), so 2 nx must be a
                           supported length (nx in 16, 24, 32, 48, 64, 96, 128, 256) for the
                           spectral preconditioner and the fixed-point method */
} vdp_bc;

typedef enum {
  VDP_PRECOND_JACOBI = 0, /* diagonal (Jacobi) scaling, folded into the operator */
  VDP_PRECOND_CHEB = 1,   /* Jacobi + fixed polynomial: cheb_degree terms of the Chebyshev
                             iteration for the unit-diagonal operator on [0.1, 2] (degree - 1
                             stencil sweeps per Krylov iteration; symmetric positive definite,
                             so plain preconditioned CG applies); direct stencil sweep only */
  VDP_PRECOND_SPECTRAL = 2, /* the constant-coefficient inverse of the paper's Poisson iteration
                             (Sec. 3.4): z = (-L_h)^-1 r in unscaled variables, L_h the 7-point
                             Laplacian with 1/h^2 faces, applied by FP32 FFTs (five passes per
                             Krylov iteration).  The preconditioned condition number is at most
                             max(rho)/min(rho) for any grid size.  Each of nx, ny, nz must be one
                             of 32, 48, 64, 96, 128, 192, 256, 512; direct stencil sweep only;
                             batch members only in batches of ordinary launches (persistent =
                             0).  Extra memory: about 16 bytes per cell */
  VDP_PRECOND_MG = 3      /* a geometric multigrid V-cycle (no counterpart in the paper; the
                             standard mesh-independent alternative to its FFT solve): cell-
                             centred, periodic, FP32; levels halve every size while all are even
                             and the level has more than 64 cells; coarse face coefficient = 1/2
                             x the sum of the four fine faces under it; linear interpolation and
                             its transpose; one weighted Jacobi sweep (0.8) before and after the
                             coarse correction; the coarsest level (at most 512 cells, else the
                             grid is not supported) by a dense pseudo-inverse.  z = W M W rt in
                             the solve's scaled variables (W = D^1/2).  Iteration counts hardly
                             grow with the grid or the density ratio.  Needs at least one
                             coarsening (more than 64 cells, even sizes down to the coarsest);
                             direct stencil sweep only; batch members only in batches of
                             ordinary launches (persistent = 0).  In the duct the transfers do
                             not reach across the x ends  Extra memory: about 24
                             bytes per cell */
} vdp_precond;

typedef enum {
  VDP_METHOD_CG = 0,          /* preconditioned conjugate gradients (precond), FP64 refinement */
  VDP_METHOD_FIXED_POINT = 1  /* the paper's own iteration (Sec. 3.4, Eq. (Pois)): with p = p_g
                                 + dp it drops the term rho grad(1/rho) . grad(dp) and solves the
                                 constant-coefficient equation L_h dp = rho (f - A p_g) with the
                                 spectral inverse (FP32 FFTs), then p_g += damping * dp, until
                                 the FP64 residual meets tol.  Each iteration costs one FP64
                                 residual and one spectral inverse.  Converges when the density
                                 varies moderately (the paper: the rate depends on the density
                                 variation); a residual growing past 1e4 x ||f - <f>|| ends the
                                 solve with VDP_ENOTCONV.  Grid sizes as VDP_PRECOND_SPECTRAL;
                                 the density weight is taken at vdp_set_density, so select the
                                 method before setting the density (VDP_EINVAL otherwise);
                                 precond is ignored; iters counts fixed-point updates */
} vdp_method;

typedef struct {
  int precision;       /* vdp_precision (default VDP_FP64) */
  int max_iter;        /* cap on the total number of inner Krylov iterations (default 20000) */
  double inner_tol;    /* mixed precision: relative residual reduction per inner solve
                          (default 1e-4); FP64 derives its inner target from tol */
  int precond;         /* vdp_precond (default VDP_PRECOND_JACOBI) */
  int cheb_degree;     /* polynomial terms for VDP_PRECOND_CHEB, 1..16 (default 4) */
  int use_guess;       /* 1: p on entry to vdp_solve is the initial guess; 0: start from p = 0 */
  void *stream;        /* cudaStream_t for all work of this context (default NULL) */
  int stencil;         /* stencil sweep: 0 = direct register march (default), 1 = TMA-staged
                          shared-memory pipeline */
  int tile_y;          /* rows per row tile of a work unit (0 = automatic) */
  int units;           /* work units (thread blocks) per sweep (0 = automatic) */
  int stages;          /* shared-memory pipeline stages of the stencil sweep, 4..8 (0 = auto) */
  int threads;         /* threads per stencil work unit, 128..512, multiple of 32 (0 = auto) */
  int steps_per_sync;  /* 0 (default): each solve is one graph launch whose device-side loop
                          stops when the solve is done; > 0: replay graphs of that many rounds
                          with a host check of the state after each (same results) */
  int method;          /* vdp_method (default VDP_METHOD_CG) */
  double damping;      /* VDP_METHOD_FIXED_POINT: scale of each update, 0 < damping <= 2
                          (default 1, the paper's update) */
  int spec_slab;       /* spectral passes: z planes per slab, X+/Y+ and Y-/X- then alternate
                          slab by slab so a slab's spectrum is handed over in L2; 0 (default) =
                          the whole grid at once (faster on the grids measured) */
} vdp_opts;

typedef struct {
  int status;          /* vdp_status of the last solve */
  int iters;           /* total inner Krylov iterations */
  int outer_iters;     /* FP64 residual evaluations (refinement steps + final check) */
  double rel_res;      /* final FP64 relative residual ||(f-<f>) - A p|| / ||f-<f>|| */
  double rhs_mean;     /* <f> removed from the right-hand side (chi' of App. A) */
  double ms;           /* device time of the last solve in milliseconds */
  int sweeps;          /* device sweeps (kernel work phases) executed */
  int launches;        /* kernels launched by the solve (including idle steps after convergence) */
} vdp_stats;

typedef struct vdp_ctx vdp_ctx;

/* Fill *o with the defaults listed in vdp_opts. */
void vdp_default_options(vdp_opts *o);

/*
 * Create a solver for an nx x ny x nz periodic box of side L (h_d = L / n_d).
 * nx must be a multiple of 8 and at least 8 (16-byte aligned rows in every storage precision);
 * ny, nz >= 1.  Allocates all device memory the solve needs.  *out = NULL on failure.
 */
int vdp_create(int nx, int ny, int nz, double L, vdp_ctx **out);

/*
 * As vdp_create with box lengths Lx, Ly, Lz (h_d = L_d / n_d) and the boundary condition in x
 * (vdp_bc).  VDP_EINVAL for lengths that are not finite and positive or an unknown bc_x.  In the
 * duct every solve method and preconditioner works; the projection steps are for the periodic
 * box only (VDP_EINVAL there).
 */
int vdp_create_bc(int nx, int ny, int nz, double Lx, double Ly, double Lz, int bc_x,
                  vdp_ctx **out);

/* Replace the options (takes effect at the next set_density / solve). */
int vdp_set_options(vdp_ctx *ctx, const vdp_opts *opts);
int vdp_get_options(const vdp_ctx *ctx, vdp_opts *opts);

/*
 * rho: cell-centred density, nx*ny*nz doubles.  Builds the face coefficients b_d, the Jacobi
 * scaling and the inner-precision copies.  Returns VDP_EDENSITY (and keeps the previous
 * density, if any) when an entry is <= 0 or not finite.
 */
int vdp_set_density(vdp_ctx *ctx, const double *rho);

/*
 * Solve A p = rhs - <rhs> to relative residual tol (tol > 0).  rhs: nx*ny*nz doubles (not
 * modified).  p: nx*ny*nz doubles, output (and initial guess when use_guess = 1).  On return p
 * has zero mean.  A zero (or constant) rhs gives p = 0.  VDP_ENOTCONV / VDP_EBREAKDOWN leave the
 * last iterate (zero mean) in p.  Requires a prior successful vdp_set_density.
 */
int vdp_solve(vdp_ctx *ctx, const double *rhs, double *p, double tol);

/* Statistics of the last vdp_solve. */
int vdp_get_stats(const vdp_ctx *ctx, vdp_stats *stats);

/* Release the context and all its device memory.  NULL-safe. */
void vdp_destroy(vdp_ctx *ctx);

/* Name of a vdp_status. */
const char *vdp_strerror(int status);

/* Text of the last CUDA error seen by the library in this process ("" if none). */
const char *vdp_last_cuda_error(void);

/* ABI version of this library (incremented on incompatible changes). */
int vdp_version(void);

/* ------------------------------------------------------------------------------------------ */
/* Single operator application, for tests and for callers that embed the operator elsewhere.    */
/* ------------------------------------------------------------------------------------------ */

/*
 * out = A p with the context's FP64 face coefficients (after vdp_set_density).  p and out are
 * nx*ny*nz doubles (device or host); out must not alias p.
 */
int vdp_apply(vdp_ctx *ctx, const double *p, double *out);

/*
 * out = L_h^-1 g: the constant-coefficient periodic Poisson solve of the paper's iteration
 * (Sec. 3.4) with the context's grid (L_h: 7-point Laplacian, faces 1/h_d^2; the zero Fourier
 * mode of g is dropped, so out has zero mean).  Computed with the FP32 FFT passes of the
 * spectral preconditioner (relative error about 1e-6); g and out are nx*ny*nz doubles, device
 * pointers, 16-byte aligned, out must not alias g.  Needs no density.  VDP_EINVAL for grid
 * sizes the spectral passes do not support (see VDP_PRECOND_SPECTRAL).
 */
int vdp_inverse_laplacian(vdp_ctx *ctx, const double *g, double *out);

/*
 * Levels of the multigrid V-cycle for an nx x ny x nz grid (level 0 = the grid), or 0 when the
 * grid is not supported by VDP_PRECOND_MG.
 */
int vdp_mg_levels(int nx, int ny, int nz);

/*
 * out = M g: one V-cycle of VDP_PRECOND_MG (an approximation of (-A)^-1 in unscaled variables,
 * with the context's density; FP32 inside).  g and out are nx*ny*nz doubles, device pointers,
 * 16-byte aligned, out must not alias g.  VDP_EINVAL without a density or for a grid the V-cycle
 * does not support.  Allocates the levels on first use.
 */
int vdp_mg_apply(vdp_ctx *ctx, const double *g, double *out);

/* ------------------------------------------------------------------------------------------ */
/* The steps either side of the solve in one projection substep (App. A, Eq. (mom)).           */
/* ------------------------------------------------------------------------------------------ */

/*
 * Face momenta: mx, my, mz are nx*ny*nz doubles each; mx[i] is the x-momentum (rho u_x) on the
 * LOW x-face of cell i (the face shared by cells i - e_x and i, periodic), likewise my, mz.  The
 * density is the context's (vdp_set_density with rho_new); the face density is the App. B mean of
 * the two adjacent cell densities, the one the Poisson operator uses.  c = C_pre[k] * dt > 0 is
 * the substep's pressure coefficient.  All arrays are DEVICE pointers (8-byte aligned; p also
 * 16-byte aligned for vdp_project) on the context's device; the calls run on the context's stream
 * and return after it has finished.  VDP_EINVAL: no density set, c not finite and positive, a
 * host or misaligned pointer, an output that aliases an input, or a duct context (the face
 * momenta of the two x ends would need their own storage: periodic box only).
 */

/*
 * f = RHS^Pois = ( div((rho u)~ / rho_face) - rhs_div ) / c: the right side of the
 * variable-coefficient Poisson equation of App. A before its mean is removed (the solve removes
 * it: chi' = -<f>, reported as vdp_stats.rhs_mean).  rhs_div (RHS^div of App. A, cell centres)
 * may be NULL for zero.  f must not alias an input.
 */
int vdp_projection_rhs(vdp_ctx *ctx, const double *mx, const double *my, const double *mz,
                       const double *rhs_div, double c, double *f);

/*
 * Eq. (mom): (rho u_d)_new = (rho u_d)~ - c (p[i] - p[i - e_d]) / h_d on every low face, in place
 * on mx, my, mz.  p is cell-centred.  No density is needed.
 */
int vdp_projection_correct(vdp_ctx *ctx, const double *p, double c, double *mx, double *my,
                           double *mz);

/*
 * One whole projection: vdp_projection_rhs into a context-owned buffer (allocated on first use,
 * nx*ny*nz doubles), vdp_solve of div((1/rho) grad p) = RHS^Pois + chi' to relative residual tol
 * with the context's options (p is the initial guess when opts.use_guess), then
 * vdp_projection_correct in place.  Afterwards div(u_new) = rhs_div - <rhs_div> on every cell to
 * the solve's tolerance (App. A).  Returns the solve's status; when it is not VDP_OK the momenta
 * are left unchanged.  vdp_get_stats describes the solve.
 */
int vdp_project(vdp_ctx *ctx, double *mx, double *my, double *mz, const double *rhs_div,
                double c, double tol, double *p);

/*
 * vdp_project with its kernels timed: ms[0] = the right-side kernel, ms[1] = the solve
 * (vdp_stats.ms), ms[2] = the correction kernel, in milliseconds (CUDA events that bracket each
 * kernel alone; the kernels are captured into small graphs for that, which costs host time).
 * ms is host memory for 3 floats (VDP_EINVAL if NULL); results are those of vdp_project.
 */
int vdp_project_timed(vdp_ctx *ctx, double *mx, double *my, double *mz, const double *rhs_div,
                      double c, double tol, double *p, float *ms);

/* ------------------------------------------------------------------------------------------ */
/* Per-kernel timing (instrumentation; the paper has no counterpart).                          */
/* ------------------------------------------------------------------------------------------ */

/* Sweep kinds timed by vdp_solve_timed, by the phase of the method the launch advances. */
enum {
  VDP_SWEEP_RES64 = 0,   /* FP64 residual r = f - A p (refinement step, Eq. Pois operator)    */
  VDP_SWEEP_STENCIL = 1, /* search direction + stencil apply + <d, q> (one per Krylov iter.)  */
  VDP_SWEEP_CHEB = 2,    /* one Chebyshev preconditioner sweep (precond = VDP_PRECOND_CHEB)   */
  VDP_SWEEP_UPDATE = 3,  /* x, r updates + <r, r> (one per Krylov iteration)                  */
  VDP_SWEEP_OTHER = 4,   /* rhs mean removal, refinement correction p -= ..., final gauge     */
  VDP_SWEEP_SPEC_X = 5,  /* spectral preconditioner: forward and inverse real FFTs along x     */
  VDP_SWEEP_SPEC_Y = 6,  /* ... forward and inverse FFTs along y                               */
  VDP_SWEEP_SPEC_Z = 7,  /* ... FFT along z, division by the eigenvalues, inverse FFT along z   */
  VDP_SWEEP_MG = 8,      /* one whole multigrid V-cycle (all its launches, timed together)     */
  VDP_SWEEP_KINDS = 9
};

typedef struct {
  int launches[VDP_SWEEP_KINDS];  /* kernel launches of each kind in the solve               */
  double ms[VDP_SWEEP_KINDS];     /* their summed durations (CUDA events around each launch) */
  double ms_min[VDP_SWEEP_KINDS]; /* shortest single launch (0 when there was none)          */
} vdp_sweep_times;

/*
 * vdp_solve with every kernel launch timed on its own.  Instead of replaying a CUDA graph the
 * host reads the solve's state before each launch and launches only the kernel the current
 * phase needs, with a CUDA event recorded on the context's stream before and after it.  The
 * kernels, their launch configuration and the order of all arithmetic are those of vdp_solve,
 * so p, the statistics (except ms, which here includes the host round trips) and the iteration
 * counts are bitwise the same; only the gaps between launches grow.  rhs and p: device
 * pointers (VDP_EINVAL otherwise); times: output, required.  Meant for measurement, not speed.
 */
int vdp_solve_timed(vdp_ctx *ctx, const double *rhs, double *p, double tol, vdp_sweep_times *times);

/* ------------------------------------------------------------------------------------------ */
/* Batches: many independent solves advanced together (continuous batching).                   */
/* ------------------------------------------------------------------------------------------ */

/*
 * A batch advances the solves of several contexts (any grid sizes, density fields and
 * tolerances; one precision, the default direct stencil sweep) in the same device launches.
 * Each member keeps its own context, so its iterations and its result are exactly those of
 * vdp_solve on that context alone.  persistent = 1 runs each vdp_batch_run as one cooperative
 * persistent kernel looping over all members with grid-wide barriers (bounded waits);
 * persistent = 0 as the equivalent sequence of ordinary launches; either is captured into a
 * CUDA graph that is re-captured only when membership changes.  Work is ordered on `stream`
 * (NULL = legacy default stream).  A batch does not own its contexts.
 */
typedef struct vdp_batch vdp_batch;
int vdp_batch_create(int precision, int persistent, void *stream, vdp_batch **out);
void vdp_batch_destroy(vdp_batch *batch);   /* NULL-safe */

/*
 * Queue a solve of ctx (after vdp_set_density; options precision equal to the batch's):
 * A p = rhs - <rhs> to relative residual tol, as vdp_solve.  rhs and p: device pointers, 16-byte
 * aligned, valid until the member is done.  VDP_EINVAL if ctx is already a member.
 */
int vdp_batch_add(vdp_batch *batch, vdp_ctx *ctx, const double *rhs, double *p, double tol);

/*
 * Advance every unfinished member by up to max_pairs sweep pairs (about one Krylov iteration
 * each) and wait for it; *active = members still unfinished.  Finished members' statistics are
 * available through vdp_get_stats on their contexts.  VDP_ETIMEOUT if a grid barrier wait expired.
 */
int vdp_batch_run(vdp_batch *batch, int max_pairs, int *active);

/* 1 if ctx's queued solve has finished, 0 if not, -VDP_EINVAL if ctx is not a member. */
int vdp_batch_done(vdp_batch *batch, vdp_ctx *ctx);

/* Remove ctx from the batch (finished or not); the context itself is untouched. */
int vdp_batch_remove(vdp_batch *batch, vdp_ctx *ctx);

/* Number of members (finished ones included until removed). */
int vdp_batch_size(const vdp_batch *batch);

/*
 * Bound on each grid-barrier wait of the persistent kernel, in seconds (0 < seconds <= 60;
 * default 2).  A wait that expires (a lost arrival) ends the run with VDP_ETIMEOUT instead of
 * hanging; the members stay usable and the next vdp_batch_run continues them.
 */
int vdp_batch_set_wait_limit(vdp_batch *batch, double seconds);

/*
 * Failure injection for testing that path (no counterpart in the paper): the next run of a
 * persistent batch waits at its first grid barrier for one block more than it launches, so the
 * wait expires after the limit and the run returns VDP_ETIMEOUT.  Nothing faults or hangs.
 * VDP_EINVAL for a batch of ordinary launches.
 */
int vdp_batch_inject_lost_arrival(vdp_batch *batch);

/*
 * Number of slabs the spectral passes of ctx's solve run in (vdp_opts.spec_slab): 1 when the
 * whole grid is transformed at once, more when X+/Y+ and Y-/X- alternate slab by slab; 0 when
 * the solve does not use the spectral passes, or ctx is NULL.
 */
int vdp_spectral_slabs(const vdp_ctx *ctx);

/* ------------------------------------------------------------------------------------------ */
/* Measurement helper.                                                                         */
/* ------------------------------------------------------------------------------------------ */

/*
 * The FP64 FMA throughput of the current GPU, in TFLOP/s (one FMA = 2 flop), measured on
 * `stream` (cudaStream_t, NULL = legacy default) by a kernel of independent FMA chains over
 * 8 blocks of 256 threads per SM; the best of three timed launches after a warm-up.  No
 * counterpart in the paper: the FP64 stencil and residual sweeps are bound by the FP64 pipe,
 * and their roofline divides by this figure.  VDP_EINVAL for a NULL output, VDP_ECUDA on a CUDA
 * error.  Synchronises the stream.
 */
int vdp_probe_fp64(void *stream, double *tflops);

/* ------------------------------------------------------------------------------------------ */
/* A solve that allocates no device memory.                                                    */
/* ------------------------------------------------------------------------------------------ */

/*
 * The paper has no counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc: hosts whose device memory belongs to a pool or budget manager that reserves the
 * GPU up front and forbids side allocations (a cudaMalloc there fails, or takes memory promised
 * to another user), and latency-critical loops that cannot take the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree.
 *
 * vdp_solve_noalloc does what vdp_create + vdp_set_density + vdp_solve + vdp_destroy do with
 * default options (and gives the same pressure), for grids of at most VDP_NOALLOC_MAX_CELLS
 * cells.  Every intermediate (face coefficients, Jacobi scaling, Krylov vectors, partial sums,
 * solver state) lives in one fixed array of VDP_NOALLOC_SCRATCH_BYTES bytes of device memory
 * that the CUDA runtime reserves when the library is loaded, on every GPU that loads it, and
 * keeps until the process exits.  The call makes no cudaMalloc, cudaFree or other allocating
 * call.
 *
 *   nx, ny, nz, L   grid and box as in vdp_create (nx a multiple of 8); nx*ny*nz above
 *                   VDP_NOALLOC_MAX_CELLS is rejected with VDP_EINVAL
 *   rho, rhs        device pointers of the current device, nx*ny*nz doubles (rhs 16-byte
 *                   aligned); not modified
 *   p               device pointer of the current device, nx*ny*nz doubles, 16-byte aligned;
 *                   output (zero mean)
 *   tol             relative residual target as in vdp_solve
 *   precision       vdp_precision
 *   stream          cudaStream_t for all work (NULL = legacy default stream); the call
 *                   synchronises this stream and returns after the work has finished
 *   stats           optional (may be NULL); ms is not measured (0)
 * Returns a vdp_status as vdp_solve / vdp_set_density do.  VDP_EINVAL for host pointers,
 * pointers of another device, and buffers whose allocation ends before nx*ny*nz doubles -- the
 * allocation as the driver sees it: an array carved out of a larger allocation by a caching
 * allocator (a PyTorch tensor, a memory pool) passes this check whatever its own length, so such
 * callers must pass arrays of nx*ny*nz doubles (the Python binding checks their sizes).
 *
 * Set-up: the first call on a device (and the first after that device's context was destroyed
 * and created again, e.g. by cudaDeviceReset) looks up the device address of the array in the
 * current context with cudaGetSymbolAddress; make that first call before any stream capture
 * begins.  All calls in the process share the one array and it keeps the contents of the last
 * call (the solve clears what must start at zero): calls whose GPU work overlaps -- from two host
 * threads, or on two streams -- race and corrupt each other, so serialise them.
 */
#define VDP_NOALLOC_MAX_CELLS 65536
#define VDP_NOALLOC_SCRATCH_BYTES 7276544
int vdp_solve_noalloc(int nx, int ny, int nz, double L, const double *rho, const double *rhs,
                      double *p, double tol, int precision, void *stream, vdp_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* VDP_H */
