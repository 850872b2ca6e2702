/*
 * imex.h - C-ABI of the GB300 immersed Newmark IMEX library (libimex).
 *
 * The library time-steps the scalar wave equation
 *     rho u'' - div(rho c^2 grad u) = f_t(t) f_x(x)   on a box minus holes,
 * discretised by the spectral cell method, with the immersed Newmark IMEX
 * scheme of Faßbender et al., "Implicit-Explicit Time Integration for the
 * Immersed Wave Equation" (arXiv 2310.14712):
 *   - explicit DOFs I_d (supported only by uncut cells): central differences on
 *     the GLL-lumped diagonal mass (Eqs. CDMstep, CDMacc);
 *   - implicit DOFs I_c (touching a cut cell): trapezoidal Newmark
 *     (beta = 1/4, gamma = 1/2) with S = M^cc + beta dt^2 K^cc factorised once
 *     (Fig. TrapCDMIMEX).
 * Setup runs on the host (C++); every time step runs in CUDA kernels for
 * sm_103a on the caller's stream.  All arithmetic is IEEE FP64.
 *
 * Conventions
 *   - Every function returns 0 (IMEX_OK) or a negative IMEX_ERR_* code; no C++
 *     exception crosses the ABI.  imex_last_error() describes the last failure
 *     of the calling thread.
 *   - Pointers passed in are owned by the caller and only read during the call.
 *     The context owns all device memory it allocates (through the optional
 *     allocator hooks, else cudaMalloc) and releases it in imex_destroy().
 *   - Fields use the canonical layout: the (n_x p + 1) x (n_y p + 1)
 *     [x (n_z p + 1)] lattice of GLL nodes of the Cartesian cell grid,
 *     x fastest, FP64, inactive nodes (only in empty cells) = 0.
 *   - imex_step() is asynchronous on the given stream; device-side failures
 *     surface at the next synchronising call.
 */
#ifndef IMEX_H
#define IMEX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IMEX_OK 0
#define IMEX_ERR_ARG (-1)      /* invalid argument or size */
#define IMEX_ERR_GEOM (-2)     /* degenerate geometry */
#define IMEX_ERR_ALLOC (-3)    /* allocation failed */
#define IMEX_ERR_CUDA (-4)     /* CUDA runtime error */
#define IMEX_ERR_NOT_SPD (-5)  /* S or M^cc not positive definite */
#define IMEX_ERR_TIMEOUT (-6)  /* reserved: a bounded device wait gave up (no kernel of this
                                  library waits on a flag; none returns it) */
#define IMEX_ERR_DIVERGED (-7) /* non-finite field values */

/* Source time functions f_t (Sec. Spatial discretization: f(t) = f_t(t) f_x). */
#define IMEX_WAVELET_RICKER 0      /* (1 - 2 pi^2 f0^2 s^2) exp(-pi^2 f0^2 s^2), s = t - 1/f0 */
#define IMEX_WAVELET_GAUSS_DERIV 1 /* Eq. ft of the 2D example, t0 = 1/f0, sigma_t = 1/(2 pi f0) */
#define IMEX_WAVELET_SINE_BURST 2  /* two-cycle sine burst of the 3D example */

/* Field selectors for imex_fields / imex_set_fields (canonical full-grid layout). */
#define IMEX_FIELD_U 0          /* u_n on all active nodes */
#define IMEX_FIELD_U_PREV_D 1   /* u^d_{n-1} on I_d (CDM history), 0 elsewhere */
#define IMEX_FIELD_V_C 2        /* velocity on I_c, 0 elsewhere */
#define IMEX_FIELD_A_C 3        /* acceleration on I_c, 0 elsewhere */
#define IMEX_FIELD_FX 4         /* assembled spatial load f_x (read only) */
#define IMEX_FIELD_MASK_D 5     /* 1.0 on I_d, 0 elsewhere (read only) */
#define IMEX_FIELD_MASK_C 6     /* 1.0 on I_c, 0 elsewhere (read only) */

typedef struct imex_ctx imex_ctx; /* opaque; owned by the library */

/* Geometry and material (Sec. Spatial discretization).  Read during setup only. */
typedef struct {
  int dim;               /* 2 or 3 */
  double lo[3], hi[3];   /* embedding box Omega */
  int ncells[3];         /* Cartesian cells per axis (>= 1) */
  int nholes;            /* holes removed from Omega */
  const double *holes;   /* nholes x (centre[dim], semi_axes[dim]); axis-aligned ellipsoids */
  int tree_depth;        /* spacetree depth for cut cells, root = level 0 */
  double rho;            /* density (> 0) */
  double c0;             /* wave speed (> 0) */
  const double *cell_c;  /* optional per-cell wave speed (prod ncells, x fastest) or NULL */
} imex_mesh;

/* Source: Gaussian bell(s) f_x (Eq. fx) times a wavelet f_t.  nsrc bells are summed. */
typedef struct {
  int nsrc;
  const double *pos;     /* nsrc x dim */
  double f0;             /* wavelet frequency */
  double sigma;          /* bell width */
  double amp;            /* bell amplitude (the paper uses 10) */
  int wavelet;           /* IMEX_WAVELET_* */
} imex_source;

/* Optional device allocator (e.g. a PyTorch caching allocator).  NULL -> cudaMalloc. */
typedef struct {
  void *(*alloc)(size_t bytes, void *user); /* returns a device pointer or NULL */
  void (*release)(void *ptr, void *user);
  void *user;
} imex_alloc;

typedef struct {
  int64_t n_nodes;       /* canonical lattice size */
  int64_t n_d, n_c;      /* |I_d|, |I_c| */
  int64_t n_cut, n_uncut, n_empty;
  int64_t n_iface;       /* cells contributing to K^c u (cut + uncut touching I_c) */
  int64_t nnz_L;         /* nonzeros of the Cholesky factor of S */
  int64_t n_components;  /* connected components of I_c */
  int64_t n_tree;        /* nested-dissection tree nodes */
  int64_t max_block;     /* largest supernode */
  int64_t step;          /* steps taken so far, n */
  int64_t device_bytes;  /* device memory held by the context */
  double dt, dt_crit_uncut;
  double setup_seconds;
  double residual_S, residual_M; /* relative residuals of a host replay of the device solve */
  int64_t solve_levels;    /* tree levels walked per pass of the implicit solve (one launch each) */
  int64_t solve_ctas;      /* CTAs of the widest solve launch */
  int64_t solve_smem_bytes;/* shared memory requested per walk CTA: at least solve_smem_needed,
                              raised by the setup autotuner when a larger request (fewer CTAs of
                              the explicit launch beside a walk CTA) measured faster */
  int64_t launches_per_step; /* kernel launches of one imex_step step */
  int64_t rhs_pairs;       /* (c-row, interface cell) pairs of K^c u: one P^d dot product each */
  int64_t ncols;           /* independent source columns (imex_setup_batch) */
  int64_t explicit_tile_cells;   /* cells per side of an explicit-apply tile, or strip width of the
                                    sweep (autotuned) */
  double explicit_tile_us_large; /* setup timing with the larger tile: one whole step (factorised
                                    contexts with implicit DOFs) or one explicit launch (others);
                                    0: not timed */
  double explicit_tile_us_small; /* the same, smaller tile */
  int64_t scheme;                /* IMEX_SCHEME_* of the context */
  double dt_crit_cut_min;        /* smallest cut-cell critical step for the scheme's mass
                                    (central-difference schemes; 0 otherwise) */
  int64_t factorized;            /* 1: factorised implicit solve available; 0: imex_setup_pcg */
  int64_t explicit_variant;      /* explicit apply in use: 0 larger tiles, 1 smaller tiles,
                                    2 persistent strip sweep, 3 the sweep in shorter chunks with
                                    more CTAs per SM, 4..7 the split launch (explicit_split_us)
                                    (2D; autotuned at setup, IMEX_EXPLICIT_TILE=large|small|sweep|
                                    sweep_short|large_split1|large_split2|small_split2|
                                    small_split4 pins it) */
  double explicit_sweep_us;      /* setup timing of variant 2 (as the tile timings) */
  double explicit_sweep_short_us;/* setup timing of variant 3 */
  int64_t large_supernodes;      /* walked supernodes of more than 256 diagonal or ancestor rows,
                                    solved by row chunks over many CTAs */
  int64_t max_rows;              /* largest ancestor row set of a supernode */
  int64_t solve_smem_needed;     /* shared memory a walk CTA needs (factor blocks staged when
                                    they fit) */
  double explicit_split_us[4];   /* setup timings of variants 4..7: the split launch (the tiles
                                    owning nodes the implicit solve reads and the prediction, then
                                    the solve, while the other tiles run on a second stream with
                                    1 or 2 CTAs per SM (larger tiles) or 2 or 4 (smaller tiles);
                                    2D factorised contexts, direct solve; 0: not timed) */
  int64_t solve_col_block;       /* independent columns per walk / dense-top CTA: the factor
                                    blocks are staged once per block of columns (autotuned for
                                    ncols > 1, IMEX_COL_BLOCK=n pins it) */
  double solve_col_block_us[7];  /* setup timing of one whole step with 1, 2, 4, ..., 64 columns
                                    per CTA (0: not timed) */
} imex_stats;

/*
 * imex_setup - discretise, partition and factorise; upload to the current device.
 *   p      : polynomial order of the GLL Lagrange basis (1..8; 2D p <= 8, 3D p <= 4)
 *   alpha  : fictitious-domain indicator alpha_f in (0, 1] (scales rho, so M, K, f)
 *   dt     : time step; <= 0 selects 0.9 x the critical step of one uncut cell
 *            (2 / sqrt(lambda_max(K_e, M_e)), Table criticaltimestepsizes)
 *   alloc  : optional allocator hooks (NULL -> cudaMalloc)
 *   out    : receives the context
 * The initial state is u_0 = 0, v_0 = 0 with the derived CDM history
 * u^d_{-1} and initial acceleration a^c_0 (Fig. TrapCDMIMEX "Calculation of
 * initial acceleration"); imex_set_initial() replaces it.
 * Errors: IMEX_ERR_ARG, IMEX_ERR_GEOM, IMEX_ERR_NOT_SPD, IMEX_ERR_ALLOC, IMEX_ERR_CUDA.
 */
int imex_setup(const imex_mesh *mesh, int p, double alpha, double dt, const imex_source *src,
               const imex_alloc *alloc, imex_ctx **out);

/*
 * imex_setup_batch - imex_setup() for ncols independent simulations that share
 * the geometry, order, alpha, dt and source time function and differ only in
 * the source position: column k is loaded by the bell at src->pos[k] alone
 * (src->nsrc == ncols; with ncols == 1 the nsrc bells are summed, as in
 * imex_setup).  One factorisation serves every column; each launch of a step
 * covers all columns.  Every field exchanged through imex_fields,
 * imex_set_fields and imex_set_initial then holds ncols canonical grids, one
 * after the other (len = ncols * n_nodes).
 *   ncols : 1 .. 256
 * Errors: as imex_setup; IMEX_ERR_ARG if ncols is out of range or
 * ncols > 1 and src->nsrc != ncols.
 * No counterpart in the paper (it runs one source): independent right-hand
 * sides are the batched form of the same method.
 */
int imex_setup_batch(const imex_mesh *mesh, int p, double alpha, double dt, const imex_source *src,
                     int ncols, const imex_alloc *alloc, imex_ctx **out);

/*
 * Time integration schemes on the same discretisation: the method and the
 * paper's comparison schemes (Sec. "Lumping of Cut Cells", Table
 * criticaltimestepsizes, the runtime comparisons).
 *   IMEX_SCHEME_IMEX        : Newmark IMEX (Fig. TrapCDMIMEX)
 *   IMEX_SCHEME_CDM         : central differences on every DOF (Eqs. CDMstep,
 *                             CDMacc) with the consistent SCM mass: diagonal on
 *                             I_d, the consistent cut-cell blocks on I_c, so a
 *                             step is the diagonal update of I_d and a solve
 *                             with M^cc for a^c_n
 *   IMEX_SCHEME_CDM_HRZ     : the same with every cut-cell mass HRZ-lumped
 *                             (Eqs. HRZ: the diagonal scaled to the element
 *                             mass, off-diagonal entries dropped)
 *   IMEX_SCHEME_TRAPEZOIDAL : trapezoidal Newmark (beta = 1/4, gamma = 1/2) on
 *                             every DOF (I_d empty, S = M + beta dt^2 K)
 */
#define IMEX_SCHEME_IMEX 0
#define IMEX_SCHEME_CDM 1
#define IMEX_SCHEME_CDM_HRZ 2
#define IMEX_SCHEME_TRAPEZOIDAL 3

/*
 * imex_setup_scheme - imex_setup_batch() with a time integration scheme.
 *   scheme : IMEX_SCHEME_*
 *   dt     : <= 0 selects 0.9 x the scheme's cell-wise critical step: that of
 *            one uncut cell (IMEX, trapezoidal), or the smaller of that and the
 *            smallest cut-cell value 2 / sqrt(lambda_max(K_e, M_e)) for the
 *            scheme's cut-cell mass (central differences; the assembled
 *            lambda_max is bounded by the largest cell-wise one)
 * State: the central-difference schemes keep (u_n, u_{n-1}) on every active DOF:
 * IMEX_FIELD_U_PREV_D then holds u_{n-1} on I_c too, IMEX_FIELD_A_C the
 * acceleration a^c_{n-1} of the last step (a^c_0 before the first) and
 * IMEX_FIELD_V_C the initial velocity.  The trapezoidal scheme has every
 * active DOF in I_c.
 * Errors: as imex_setup_batch; IMEX_ERR_ARG for an unknown scheme;
 * IMEX_ERR_NOT_SPD if a cut-cell mass is not positive definite.  The
 * iterative solvers (imex_set_solver) and imex_adjoint take the IMEX scheme
 * only (the iterative solvers also the trapezoidal one).
 */
int imex_setup_scheme(const imex_mesh *mesh, int p, double alpha, double dt, const imex_source *src,
                      int ncols, int scheme, const imex_alloc *alloc, imex_ctx **out);

/*
 * imex_setup_pcg - a single-column context without a factorisation: no
 * nested dissection, no Cholesky factor, no solve schedule.  Every implicit
 * solve of S (Fig. TrapCDMIMEX "Acceleration calculation") is preconditioned
 * CG (imex_set_solver: IMEX_SOLVER_PCG_JACOBI, the default, with maxit 5000,
 * or IMEX_SOLVER_PCG_FSAI after imex_pcg_train); the right-hand sides come
 * from one warp-per-row kernel over the same (row, interface cell) pairs; the
 * initial acceleration solves M^cc a^c_0 = f_t(0) f^c - K^c u_0 by
 * Jacobi-preconditioned CG to 1e-12.  For partitions whose factor does not
 * fit the device solve (3D voids, where dissection separators exceed 256
 * rows).  With no direct solve to fall back on, a solve that misses the
 * tolerance still applies its last iterate and counts as a fallback in
 * imex_pcg_status.  The implicit DOFs are in grid order.
 *   scheme : IMEX_SCHEME_IMEX or IMEX_SCHEME_TRAPEZOIDAL
 * Not available on such a context: IMEX_SOLVER_DIRECT, imex_adjoint,
 * imex_step_noalloc (IMEX_ERR_ARG).
 * Errors: as imex_setup.
 */
int imex_setup_pcg(const imex_mesh *mesh, int p, double alpha, double dt, const imex_source *src, int scheme,
                   const imex_alloc *alloc, imex_ctx **out);

/*
 * imex_step - advance n >= 0 Newmark IMEX steps (Fig. TrapCDMIMEX), each:
 *   diagonal CDM step on I_d, prediction on I_c, acceleration calculation
 *   S a^c_{n+1} = f_t(t_{n+1}) f_x^c - K^c u_pred, correction on I_c.
 * stream: a cudaStream_t (NULL = legacy default stream).  Asynchronous.
 * Errors: IMEX_ERR_ARG, IMEX_ERR_CUDA (launch failures).
 */
int imex_step(imex_ctx *ctx, int64_t n, void *stream);

#define IMEX_PROFILE_PHASES 3
/*
 * imex_step_profile - imex_step() with CUDA events recorded on `stream`,
 * synchronising after each step.  phase_ms[3] receives the summed device
 * times (ms) of: [0] explicit apply + CDM update + prediction, [1] implicit
 * chain (right-hand sides, solve, correction), [2] whole steps.  For
 * measurement; results equal imex_step()'s.
 */
int imex_step_profile(imex_ctx *ctx, int64_t n, void *stream, double *phase_ms);

/*
 * imex_step_io - advance n steps like imex_step(), with host I/O every step:
 *   ft_samples : NULL (use the built-in wavelet) or n+1 host values
 *                f_t(t_{n0}), ..., f_t(t_{n0+n}) replacing it (e.g. a recorded
 *                or inverted source signature); step k reads samples k, k+1
 *   rec_nodes  : nrec canonical node indices (receivers), 0 <= nrec <= 4096
 *   traces     : n x ncols x nrec host array; entry (k, col, i) receives
 *                u_{n0+k+1} of column col at receiver i
 * Every step copies its two samples in and its receiver values out; the
 * copies run on two copy streams of the context, ordered by events against
 * the steps on `stream` (ring buffers of 8 slots), so that the step kernels
 * do not wait for them.  Pinned host arrays make the copies asynchronous;
 * pageable ones work too.  Synchronous (returns when the traces are on the
 * host); the host arrays must stay valid until then.
 * Errors: IMEX_ERR_ARG (bad sizes or node indices), IMEX_ERR_CUDA.
 */
int imex_step_io(imex_ctx *ctx, int64_t n, const double *ft_samples, const int64_t *rec_nodes,
                 int nrec, double *traces, void *stream);

/*
 * imex_step_noalloc - the same n steps as imex_step(), for callers that must
 * not allocate device memory while they run: it makes no allocation of any
 * kind.  The scratch of the factorised implicit solve (the descendant update
 * vectors, the solution vector and the right-hand sides, each column after
 * column; with supernodes of more than 256 rows also the backward products)
 * is not taken from the context but from one fixed 2 MiB array
 * (262,144 doubles) compiled into the library, which every GPU that loads
 * the library keeps until the process exits.  Typical callers run under a
 * device-memory budget fixed at start-up or inside code regions where
 * allocation calls are not permitted.
 *   - Capacity: with U = the context's update-vector length and n_c its
 *     implicit DOFs, each rounded up to even, a problem fits when
 *     (U + 2 n_c) x ncols <= 262,144 ((U + 3 n_c) x ncols when the factor has
 *     supernodes of more than 256 rows); larger problems are rejected with
 *     IMEX_ERR_ARG before anything is launched.
 *   - Contexts only: factorised (not imex_setup_pcg) and with the direct
 *     solver (imex_set_solver: IMEX_SOLVER_DIRECT, the default); the PCG
 *     solvers keep their vectors in context memory, so a context set to
 *     PCG is rejected with IMEX_ERR_ARG (use imex_step).  Every scheme
 *     (imex_setup_scheme) and every column count is accepted.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the array and it keeps the last call's contents.
 *     Nothing in it needs to start at zero: each entry is written before it
 *     is read within a step.  Calls that overlap on the GPU (other streams,
 *     other contexts, at the same time) race on the array.
 * Results are bit-identical to imex_step() on the same context state.
 * No counterpart in the paper: this is an interface choice of the library.
 */
int imex_step_noalloc(imex_ctx *ctx, int64_t n, void *stream);

/*
 * Iterative solve of the implicit partition (no counterpart in the paper,
 * which factorises S once; Sec. "Time integration").  With a PCG solver each
 * step solves S a^c_{n+1} = rhs by preconditioned conjugate gradients
 * (Saad, Algorithm 9.1) started from a^c_n and stopped at
 * ||rhs - S a|| <= tol ||rhs||; a step whose PCG does not reach tol within
 * maxit iterations falls back to the factorised direct solve (same step,
 * same stream, no host round trip).  Single-column contexts only.
 *   IMEX_SOLVER_DIRECT     : the factorised solve (default)
 *   IMEX_SOLVER_PCG_FSAI   : M^{-1} = G G^T, G lower triangular on the pattern
 *                            of S, learned by imex_pcg_train (initially
 *                            diag(S)^{-1/2})
 *   IMEX_SOLVER_PCG_JACOBI : M^{-1} = diag(S)^{-1}
 */
#define IMEX_SOLVER_DIRECT 0
#define IMEX_SOLVER_PCG_FSAI 1
#define IMEX_SOLVER_PCG_JACOBI 2

/* imex_set_solver - select the solver; tol > 0, 1 <= maxit <= 100000.
 * Errors: IMEX_ERR_ARG (bad values, or a PCG solver on a multi-column context). */
int imex_set_solver(imex_ctx *ctx, int solver, double tol, int maxit);

/*
 * imex_pcg_train - learn G: `epochs` steps of Adam (Kingma and Ba, Algorithm 1;
 * learning rate lr, in units of G_ij sqrt(S_ii), diagonal kept >= 1e-3) on
 * Kaporin's functional K(G) = tr(G^T S G) - 2 sum_i log G_ii over the lower
 * pattern of S, continuing from the current G.  loss_hist: NULL or `epochs`
 * host doubles receiving K before each step.  Synchronous.
 */
int imex_pcg_train(imex_ctx *ctx, int epochs, double lr, double *loss_hist);

/*
 * imex_pcg_status - last PCG solve: iterations, relative residual, and the
 * totals since setup (iterations, steps that fell back to the direct solve).
 * Synchronous.  Any pointer may be NULL.
 */
/*
 * imex_pcg_train_guess - learn the starting guess of the PCG solves from the
 * method's own solutions (no counterpart in the paper; the north-star's
 * learned part).  Advances the context by nsteps >= 4 steps with its current
 * solver, keeping a^c after every step (a temporary device buffer of
 * (nsteps + 1) n_c doubles), then runs `epochs` Adam steps (Kingma and Ba,
 * Algorithm 1; learning rate lr, from w = (1, 0, 0)) on
 *   E(w) = sum_s ||w0 a_s + w1 a_{s-1} + w2 a_{s-2} - a_{s+1}||^2 / ||a_{s+1}||^2
 * with the library's gradient kernels.  Afterwards every PCG solve starts
 * from x0 = w0 a^c_n + w1 a^c_{n-1} + w2 a^c_{n-2} (instead of a^c_n) once two
 * PCG solves since the last direct solve or state change have filled the
 * history.  loss_hist (epochs doubles) and w_out (3) may be NULL.
 * Single-column contexts.  Errors: IMEX_ERR_ARG, IMEX_ERR_ALLOC, IMEX_ERR_CUDA.
 */
int imex_pcg_train_guess(imex_ctx *ctx, int nsteps, int epochs, double lr, double *loss_hist, double *w_out);

/*
 * imex_pcg_set_guess - enable (with the weights w[3], or the trained ones when
 * w is NULL) or disable (enable = 0: start from a^c_n) the learned starting
 * guess of the PCG solves.  Errors: IMEX_ERR_ARG, IMEX_ERR_CUDA.
 */
int imex_pcg_set_guess(imex_ctx *ctx, int enable, const double *w);

/*
 * imex_pcg_fsai_closed_form - set G of the FSAI preconditioner to the
 * minimiser of Kaporin's functional on its pattern, computed directly on the
 * host (column j: S_QQ y = e_j on the rows Q of the column,
 * G_Qj = y / sqrt(y_j); Kolotilina and Yeremin's factorised sparse
 * approximate inverse), for comparison with the trained G; later training
 * continues from it.  Errors: IMEX_ERR_ARG, IMEX_ERR_NOT_SPD, IMEX_ERR_CUDA.
 */
int imex_pcg_fsai_closed_form(imex_ctx *ctx);

int imex_pcg_status(imex_ctx *ctx, int64_t *iters_last, double *res_last, int64_t *iters_total,
                    int64_t *fallbacks);

/*
 * imex_fsai_kaporin - the training kernels on caller data (device pointers):
 * K(G) and its gradient for S (n x n CSR: s_ptr, s_col, s_val) and G (lower
 * triangular CSR with sorted columns and a nonzero diagonal: g_ptr, g_col,
 * g_val).  grad: nnz(G) device doubles; loss: host double.  Synchronous on
 * `stream`.  For checking the kernels against a CPU definition.
 */
int imex_fsai_kaporin(int n, const int *s_ptr, const int *s_col, const double *s_val, const int *g_ptr,
                      const int *g_col, const double *g_val, double *grad, double *loss, void *stream);

/*
 * imex_adjoint - misfit J = 1/2 sum_{n=1..N} sum_cols sum_r (u_n[rec_r] - d)^2
 * of the next N = nsteps steps and its gradient dJ/dc_e with respect to the
 * wave speed of every cell, by the discrete adjoint of the IMEX step (no
 * counterpart in the paper, which names full-waveform inversion as the use).
 *   rec_nodes : nrec canonical node indices (host)
 *   data      : N x ncols x nrec observed traces (host), entry (n-1, col, r)
 *               compared with u_n of column col at receiver r
 *   checkpoint_every : forward states kept every that many steps; each
 *               segment is recomputed once in the reverse sweep
 *   grad      : ncells (product of mesh->ncells) host doubles, overwritten
 *               (0 for empty cells); misfit: host double
 * Runs forward from the current state and leaves the context N steps later.
 * The dependence of the starting state on c is not differentiated (it has
 * none when it is the setup's state u_0 = v_0 = 0).  Uses the factorised
 * solve; temporary device memory (about (N / checkpoint_every + checkpoint_every)
 * ncols n_nodes doubles) is allocated for the call.  Synchronous.
 */
int imex_adjoint(imex_ctx *ctx, int64_t nsteps, const int64_t *rec_nodes, int nrec, const double *data,
                 int checkpoint_every, double *grad, double *misfit);

/*
 * imex_fields - copy one field (IMEX_FIELD_*) in canonical layout into dst.
 *   len          : number of doubles in dst; must equal ncols * imex_stats.n_nodes
 *                  (column after column)
 *   dst_on_device: nonzero if dst is device memory (copy stays on the device)
 * Synchronises the context's last stream.  Errors: IMEX_ERR_ARG, IMEX_ERR_CUDA.
 */
int imex_fields(imex_ctx *ctx, int which, double *dst, int64_t len, int dst_on_device);

/*
 * imex_set_fields - overwrite one state field (U, U_PREV_D, V_C or A_C) from src
 * (canonical layout, len = ncols * n_nodes); entries outside the field's partition are
 * ignored.  With imex_set_step() this restores a checkpoint exactly.
 */
int imex_set_fields(imex_ctx *ctx, int which, const double *src, int64_t len, int src_on_device);

/* imex_set_step - set the step counter n (t_n = n dt). */
int imex_set_step(imex_ctx *ctx, int64_t n);

/*
 * imex_set_initial - restart from u_0, v_0 (canonical layout, len = ncols * n_nodes) at
 * n = 0: stores u_0, v^c_0, and computes on the device the CDM history
 * u^d_{-1} = u^d_0 - dt v^d_0 + dt^2/2 a^d_0 (Taylor start) and a^c_0 from
 * M^cc a^c_0 = f_t(0) f_x^c - K^c u_0.  v0 may be NULL (zero).
 */
int imex_set_initial(imex_ctx *ctx, const double *u0, const double *v0, int64_t len, int on_device);

/* imex_info - sizes, counts and the time step. */
int imex_info(imex_ctx *ctx, imex_stats *out);

/*
 * imex_check_finite - health check of the state after the steps issued so far
 * (synchronises the context's stream): *max_abs_u receives max |u_n| over the
 * active DOFs of every column.  Returns IMEX_ERR_DIVERGED if u_n, u_{n-1} or
 * the c-partition velocity or acceleration holds a non-finite value (an
 * unstable step, e.g. a central-difference scheme above its critical step),
 * else IMEX_OK.  max_abs_u may be NULL.
 */
int imex_check_finite(imex_ctx *ctx, double *max_abs_u);

/*
 * imex_probe_fp64 - throughput of the current device's FP64 pipe, the
 * denominator of the roofline of the FP64-bound step kernels (no counterpart
 * in the paper; a measurement helper).  One launch of 4 x SMs CTAs x 256
 * threads, each thread running eight independent chains of `iters`
 * instructions of one kind: 0 fused multiply-add, 1 add, 2 multiply (runtime
 * operands, values kept in normal range), timed with CUDA events after a
 * warm-up launch on the legacy default stream (synchronises the device).
 *   lane_ops_per_s : receives thread-level instructions per second (an FMA
 *                    counts as one; 2 flops)
 *   seconds        : receives the timed launch's duration (may be NULL)
 * Errors: IMEX_ERR_ARG (kind, iters < 1, NULL output), IMEX_ERR_ALLOC,
 * IMEX_ERR_CUDA.
 */
int imex_probe_fp64(int kind, int iters, double *lane_ops_per_s, double *seconds);

/* imex_last_error - message of the calling thread's last failure ("" if none). */
const char *imex_last_error(void);

/* imex_destroy - free device and host state; NULL is ignored. */
void imex_destroy(imex_ctx *ctx);

/*
 * Host-side building blocks (no GPU needed), for tests of the setup path:
 * imex_gll_points - GLL points and weights of order p (p+1 values each).
 * imex_gauss_points - n-point Gauss-Legendre rule.
 */
int imex_gll_points(int p, double *x, double *w);
int imex_gauss_points(int n, double *x, double *w);

/*
 * imex_host_setup_export - run the host setup only (no GPU) and export the
 * partition and implicit system for checking: node_class (n_nodes bytes:
 * 0 inactive, 1 I_d, 2 I_c; may be NULL), fx (n_nodes doubles; may be NULL).
 * stats receives the counts.  Same arguments as imex_setup.
 */
int imex_host_setup_export(const imex_mesh *mesh, int p, double alpha, double dt,
                           const imex_source *src, uint8_t *node_class, double *fx,
                           imex_stats *stats);

/*
 * imex_host_implicit_system - run the host setup only (no GPU) and export the
 * implicit system as the library factorises it (Fig. TrapCDMIMEX,
 * "Calculation and factorization of system matrix"):
 * S = M^cc + beta dt^2 K^cc (beta = 1/4) and M^cc on the pattern of S (zeros
 * where M^cc has no entry), CSR over the c-indices (the library's
 * nested-dissection order), full symmetric pattern, columns ascending.
 * Two calls: with s_col == NULL only *n_c and *nnz are written; then, with
 * *n_c and *nnz as returned, c_node (n_c: the grid node of each c-index),
 * s_ptr (n_c + 1), s_col (nnz), s_val and m_val (nnz) are filled.  All
 * arrays are host memory owned by the caller.  Same problem arguments as
 * imex_setup.  Errors: IMEX_ERR_ARG (NULL sizes, sizes that differ from the
 * system's on the second call), IMEX_ERR_GEOM, IMEX_ERR_ALLOC.
 */
int imex_host_implicit_system(const imex_mesh *mesh, int p, double alpha, double dt,
                              const imex_source *src, int64_t *n_c, int64_t *nnz, int64_t *c_node,
                              int64_t *s_ptr, int32_t *s_col, double *s_val, double *m_val);

/*
 * imex_host_element_matrices - run the host discretisation only (no GPU, no
 * factorisation) and return the element matrices of `ncell` cells (flat cell
 * ids, x fastest) as the library assembles them (Sec. Spatial
 * discretization): cut cells K_e, M_e by the spacetree quadrature with the
 * fictitious domain scaled by alpha; uncut cells the reference stiffness
 * scaled by c_e^2 / c0^2 and the GLL-lumped (diagonal) mass; empty cells
 * zero.  K and M receive ncell x P^d x P^d doubles (cell after cell,
 * column-major; both symmetric); cell_type (may be NULL) receives 0 uncut,
 * 1 cut, 2 empty.  Errors: IMEX_ERR_ARG (bad sizes, cell id out of range),
 * IMEX_ERR_GEOM.
 */
int imex_host_element_matrices(const imex_mesh *mesh, int p, double alpha, const imex_source *src,
                               int ncell, const int64_t *cells, double *K, double *M,
                               int8_t *cell_type);

#ifdef __cplusplus
}
#endif
#endif /* IMEX_H */
