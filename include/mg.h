/*
 * mg.h -- C ABI of the GB300 (sm_103a) multigrid pressure Poisson solver.
 *
 * The solver computes the pressure p of the projection step of an
 * incompressible VOF multiphase flow solver (paper §2: Eq. (1) div u = 0 and
 * Eq. (2) with the pressure force -grad p / rho), i.e. the variable-coefficient
 * Poisson problem
 *
 *        -div( (1/rho) grad p ) = b        on a uniform cell-centred grid,
 *
 * with homogeneous Neumann walls, density rho mixed from phase volume
 * fractions by Eq. (5), and a geometric multigrid V-cycle as the solver (the
 * multigrid pressure solver of §4.3.2).  Discretisation, fixed here because the
 * paper states it nowhere:
 *
 *   cells    (i,j,k), spacing h, linear index (k*ny + j)*nx + i (x fastest);
 *            a cell array has nx*ny*nz elements, shape (nz, ny, nx).
 *   faces    bx: shape (nz, ny, nx+1), entry i is the face between cells i-1
 *            and i; by: (nz, ny+1, nx); bz: (nz+1, ny, nx).  The first and last
 *            face along each axis are walls: their values are ignored on input
 *            (zero flux) and written as 0 on output.
 *   beta     face coefficient = 1 / harmonic mean of the two cell densities
 *            (= (1/rho_L + 1/rho_R) / 2).
 *   operator (A p)_c = (1/h^2) sum_{interior faces f of c} beta_f (p_c - p_nb(f)).
 *            A is symmetric positive semidefinite; its null space is the constants.
 *   solution the zero-mean p with A p = b - mean(b).
 *   V-cycle  red-black Gauss-Seidel (red = (i+j+k) even; pre sweeps red then
 *            black, post sweeps black then red), residual, 8:1 restriction
 *            (mean of the 8 children), prolongation (cell-centred trilinear, or
 *            constant), face coarsening (a coarse face = mean of the 4 fine
 *            faces tiling it, operator spacing doubled), and an exact dense
 *            solve e = A_c^+ (r - mean r) on the coarsest level.  Levels halve
 *            every dimension while all are even and the largest exceeds
 *            opts.coarsest.
 *   FP64     plain FP64 V-cycles on p until |b~ - A p| / |b~| <= rtol.
 *   MIXED    FP64 defect correction: r = b~ - A p in FP64, one FP32 V-cycle
 *            on r, p += correction in FP64, zero mean; same stopping rule.
 *   MIXED_DF as MIXED, but the outer residual and update carry p, b~ and the
 *            finest-level coefficients as pairs of FP32 numbers (hi + lo, about
 *            48 significant bits) and use FP32 arithmetic with error-free
 *            transformations; FP64 is used only to enter and leave the loop.
 *            Needs an even nx and |b~| < 1e30.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers (CUDA global memory of the device the
 *     handle was created on), owned by the caller, contiguous, in the layouts
 *     above; the library keeps no reference to them after the call returns.
 *     Unless a parameter says otherwise they are double (FP64).  The solution
 *     arrays of mg_solve (p) and mg_adjoint (lam) must be 16-byte aligned (any
 *     cudaMalloc or torch allocation is); MG_ERR_ARG otherwise.
 *   - Work is queued on the CUDA stream given to mg_create.  Entry points that
 *     need a scalar result on the host (mg_solve, mg_adjoint, the norm outputs)
 *     synchronise that stream; the others return once the work is queued.
 *   - All device memory the handle needs is allocated in mg_create; no other
 *     entry point allocates device memory.
 *   - Return value: MG_OK (0) or a negative MG_ERR_* code; no exception or
 *     signal crosses the ABI.  mg_last_error() gives a message for the last
 *     failure on that handle.  After MG_ERR_CUDA the handle should be destroyed.
 *   - A handle is not thread safe: calls on one handle must not overlap.
 */
#ifndef MG_POISSON_H
#define MG_POISSON_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MG_OK = 0,
    MG_ERR_ARG = -1,           /* bad argument: null pointer, size, option */
    MG_ERR_DENSITY = -2,       /* a density or face coefficient is not finite and > 0 */
    MG_ERR_NOT_CONVERGED = -3, /* max_cycles reached before rtol */
    MG_ERR_DIVERGED = -4,      /* residual became non-finite or grew without bound */
    MG_ERR_CUDA = -5,          /* a CUDA runtime call failed */
    MG_ERR_OOM = -6,           /* device memory allocation failed (mg_create only) */
    MG_ERR_STATE = -7          /* call order: e.g. solve before coefficients were set */
};

enum { MG_FP64 = 0, MG_MIXED = 1, MG_MIXED_DF = 2 };
enum { MG_METHOD_VCYCLE = 0, MG_METHOD_FCG = 1 }; /* mg_opts.method */
enum { MG_PROLONG_TRILINEAR = 0, MG_PROLONG_CONSTANT = 1 };
enum { MG_F64 = 0, MG_F32 = 1 }; /* element type of component-level arrays */

#define MG_MAX_LEVELS 24
#define MG_MAX_COARSE 1024 /* largest coarsest-level cell count (dense solve) */
#define MG_HIST_LEN 256

typedef struct mg_handle mg_handle;

typedef struct {
    int nx, ny, nz;   /* cells per dimension, each >= 1, nx*ny*nz >= 2 */
    double h;         /* grid spacing, > 0 */
    int precision;    /* MG_FP64, MG_MIXED or MG_MIXED_DF */
    int pre, post;    /* RBGS sweeps before / after the coarse correction (>= 0) */
    int coarsest;     /* stop coarsening once the largest dimension is <= this (>= 2) */
    int prolong;      /* MG_PROLONG_TRILINEAR or MG_PROLONG_CONSTANT */
    double rtol;      /* relative residual tolerance, |b~ - A p|_2 / |b~|_2 */
    int max_cycles;   /* V-cycles, >= 0 (the mixed modes stop before an outer iteration
                         that would exceed it) */
    int warm_start;   /* 1: mg_solve starts from the p passed in; 0: from p = 0 */
    int inner_cycles; /* mixed modes: FP32 V-cycles per outer iteration (1..8), the first from
                         zero, the next ones continuing from the previous correction; the
                         FP64 (or double-float) residual and update run once per outer
                         iteration.  0 (V-cycle iteration only): adaptive, 6 V-cycles in the
                         first outer iteration, then as many (1..6) as the contraction per
                         V-cycle observed in the last outer iteration predicts the tolerance
                         still needs, so that few FP64 residuals are evaluated without adding
                         V-cycles.  With
                         MG_METHOD_FCG: the flexible-CG iterations per outer iteration (1..8).
                         Must be 1 for MG_FP64. */
    int method;       /* MG_METHOD_VCYCLE: V-cycle iteration (defect correction in the mixed
                         modes).  MG_METHOD_FCG: conjugate gradients preconditioned by one
                         V-cycle, flexible (Polak-Ribiere) form: in MG_FP64 the whole solve, with
                         FP64 vectors; in the mixed modes the inner solver of each outer
                         iteration, in FP32 on the finest level (needs nx % 8 == 0).  The
                         stopping test uses the CG-updated residual in MG_FP64 and the outer
                         residual in the mixed modes; max_cycles counts V-cycles. */
    int fused_sweeps; /* mixed modes, finest level with an operator from a density and nx a
                         multiple of 128: 1 smooths with fused red-black sweeps (one pass over
                         the grid per sweep instead of two, planes staged in shared memory by
                         bulk copies; bitwise the same results); 0 (default) with two half sweeps
                         per sweep, which is faster on GB300 (the fused sweep is bound by its
                         instruction issue, not by memory).  Other levels and layouts always
                         use half sweeps. */
} mg_opts;

typedef struct {
    int status;                     /* same as the return value */
    int cycles;                     /* V-cycles run */
    int outer;                      /* outer iterations (= cycles for MG_FP64 and for
                                       inner_cycles 1) */
    double relres;                  /* final relative residual */
    double relres_hist[MG_HIST_LEN];/* relres after k outer iterations, k = 0..min(outer, HIST-1) */
    double ms;                      /* device time of the call (CUDA events) */
} mg_stats;

/* Defaults: 2/2 sweeps, coarsest 4, trilinear, rtol 1e-10, 200 cycles, FP64, cold start,
   one V-cycle per outer iteration, V-cycle iteration (MG_METHOD_VCYCLE), half sweeps. */
void mg_default_opts(mg_opts *opts);

/* Create a solver for one grid.  `stream` is a cudaStream_t (NULL = legacy
 * default stream) on the current device.  Allocates every device buffer the
 * handle will use (hierarchy, scratch, coarse inverse) and a small mapped
 * pinned host buffer (cudaHostAllocMapped) into which kernels store the
 * scalars the host waits for, so that those waits never queue behind copies
 * other streams run on the copy engines: nothing is allocated later.  It also records the levels below the finest of one V-cycle as a
 * CUDA graph (on a private stream; nothing runs), which every cycle replays;
 * where recording is refused the cycles launch those kernels one by one.  On failure *out is NULL and the code says why (MG_ERR_ARG: opts;
 * MG_ERR_OOM; MG_ERR_CUDA). */
int mg_create(const mg_opts *opts, void *stream, mg_handle **out);

/* Free the handle and all its device memory (synchronises its stream). NULL is a no-op. */
int mg_destroy(mg_handle *h);

/* Text of the last error on this handle ("" if none); valid until the next call. */
const char *mg_last_error(const mg_handle *h);

/* Number of multigrid levels, and the (nx, ny, nz) of level l (0 = finest). */
int mg_num_levels(const mg_handle *h);
int mg_level_dims(const mg_handle *h, int level, int *dims3);

/* Eq. (5): rho = sum_{q<nfrac} rho_q f_q + rho_{nfrac} (1 - sum_{q<nfrac} f_q), evaluated as
 * rho_{nfrac} + sum_{q<nfrac} (rho_q - rho_{nfrac}) f_q (equal up to FP64 rounding).
 * frac_dev: host array of nfrac (1..4) device pointers to cell arrays;
 * rho_phase: host array of nfrac+1 phase densities; rho_dev: output cell array. */
int mg_density_from_fractions(mg_handle *h, int nfrac, const double *const *frac_dev,
                              const double *rho_phase, double *rho_dev);

/* Set the operator from a cell density field (device, cell array): face
 * coefficients 1/harmonic-mean(rho), every coarse level, and the coarse
 * inverse.  Checks that rho is finite and > 0 everywhere (MG_ERR_DENSITY
 * otherwise; the previous operator is then no longer valid).  Synchronises. */
int mg_set_density(mg_handle *h, const double *rho_dev);

/* Set the operator from face coefficients beta (device, face layouts above;
 * wall entries ignored).  Interior entries must be finite and > 0
 * (MG_ERR_DENSITY).  Synchronises. */
int mg_set_face_coeffs(mg_handle *h, const double *bx, const double *by, const double *bz);

/* Copy the FP64 face coefficients of level l into caller arrays in the face
 * layouts of that level's dimensions (walls written as 0). */
int mg_get_level_faces(mg_handle *h, int level, double *bx, double *by, double *bz);

/* CSF face quantity for a surface-tension RHS term: on interior faces
 * csf_f = (kappa_L + kappa_R)/2 * (f_R - f_L) / h, walls 0.  f, kappa: cells. */
int mg_csf_faces(mg_handle *h, const double *f, const double *kappa, double *csfx, double *csfy,
                 double *csfz);

/* RHS assembly b = b0 + D u + sigma * D(beta * csf), D the cell divergence
 * (D u)_c = sum_faces (+u on the high face, -u on the low face) / h over
 * interior faces.  Each term is optional: b0 (cell array) may be NULL; u* are
 * face arrays or all NULL; csf* are face arrays or all NULL.  beta = the
 * handle's current fine face coefficients (needed only when csf is given).
 * b: output cell array; it may be the same array as b0. */
int mg_rhs(mg_handle *h, const double *b0, const double *ux, const double *uy, const double *uz,
           const double *csfx, const double *csfy, const double *csfz, double sigma, double *b);

/* Solve A p = b - mean(b) with mean(p) = 0 to opts.rtol.  b: cell array (not
 * modified); p: cell array, output (and the initial guess if warm_start).
 * stats may be NULL.  Returns MG_OK, MG_ERR_NOT_CONVERGED (p holds the last
 * iterate, zero mean) or MG_ERR_DIVERGED.  Synchronises. */
int mg_solve(mg_handle *h, const double *b, double *p, mg_stats *stats);

/* Adjoint of mg_solve for a loss L with dL/dp = w.  Solves A lam = w - mean(w)
 * (zero-mean lam = dL/db) with the same method and tolerance, then forms
 *   dL/dbeta_f = -(lam_L - lam_R)(p_L - p_R)/h^2 + sigma csf_f (lam_L - lam_R)/h
 * on every interior face (FP32 outputs gbx/gby/gbz in the face layouts, walls
 * 0) and dL/dsigma = sum_f beta_f csf_f (lam_L - lam_R)/h, where the forward
 * RHS was b = D u + sigma D(beta csf).  p is the forward solution.  The csf
 * arrays may be NULL (no surface term: the sigma terms vanish and *dLdsigma
 * is set to 0).  gbx/gby/gbz and dLdsigma may be NULL to skip them.  The
 * operator must be the one p was solved with.  Synchronises. */
int mg_adjoint(mg_handle *h, const double *w, const double *p, double *lam, float *gbx,
               float *gby, float *gbz, const double *csfx, const double *csfy, const double *csfz,
               double sigma, double *dLdsigma, mg_stats *stats);

/* Velocity correction of the projection step (paper §2: the face velocities of
 * Eq. (2) made divergence-free, Eq. (1)).  On every interior face
 *   o_f = u_f + beta_f ( (p_R - p_L)/h + sigma csf_f ),
 * and o_f = u_f on the walls; beta the handle's current fine face
 * coefficients, p the solution of A p = D u + sigma D(beta csf) (mg_rhs +
 * mg_solve on the same u, csf and sigma), so that D o = 0 up to the solve's
 * residual.  ux, uy, uz: input face arrays; ox, oy, oz: output face arrays,
 * either all three equal to ux, uy, uz (in place) or none of them overlapping
 * them (MG_ERR_ARG for a mix).  csf*: face arrays, or all NULL (no surface
 * term; sigma is then ignored).  FP64 arithmetic.  MG_ERR_STATE if no
 * coefficients are set.  Returns once queued. */
int mg_project(mg_handle *h, const double *p, const double *csfx, const double *csfy,
               const double *csfz, double sigma, const double *ux, const double *uy,
               const double *uz, double *ox, double *oy, double *oz);

/* Density adjoint: carries the face-coefficient gradients of mg_adjoint back
 * through beta_f = (1/rho_L + 1/rho_R)/2 and Eq. (5):
 *   dL/drho_c = -1/(2 rho_c^2) * sum_{interior faces f of c} dL/dbeta_f,
 *   dL/df_q   = dL/drho_c * (rho_q - rho_{nfrac})           (q < nfrac).
 * rho: cell array (the density the operator was set from, finite and > 0);
 * gbx, gby, gbz: FLOAT face arrays (as mg_adjoint writes them; wall entries
 * ignored); drho: output cell array (double).  nfrac = 0 skips the fraction
 * gradients; otherwise 1..4, rho_phase a host array of nfrac+1 phase
 * densities (as for mg_density_from_fractions) and dfrac_dev a host array of
 * nfrac device pointers to output cell arrays.  The face gradients are FP32,
 * so the sum and the factor are formed in FP32 (FP64 for densities outside
 * [2^-20, 2^21)) and the results carry FP32 precision.  Uses only the handle's
 * dimensions and stream (no operator needed).  Returns once queued.
 * The fraction path covers the density dependence only: a surface term whose
 * csf was built from a fraction (mg_csf_faces) contributes no further term. */
int mg_density_grads(mg_handle *h, const double *rho, const float *gbx, const float *gby,
                     const float *gbz, double *drho, int nfrac, const double *rho_phase,
                     double *const *dfrac_dev);

/* ---- component steps of the V-cycle on level `level` --------------------------
 * For callers that assemble their own cycles, and for step-by-step checking.
 * dtype MG_F64 uses the FP64 coefficients, MG_F32 the FP32 copies (MIXED and
 * MIXED_DF handles); arrays are then double or float cell arrays of that level.
 * Physical scaling: level l has spacing h * 2^l. */

/* y = A_l x */
int mg_apply(mg_handle *h, int level, int dtype, const void *x, void *y);

/* `sweeps` full red-black Gauss-Seidel sweeps on x in place for A_l x = b;
 * order 0 = red then black (pre-smoothing), 1 = black then red (post).
 * The smoothing components (this one and the two fused ones below) run in the
 * handle's V-cycle precision: MG_F64 on MG_FP64 handles, MG_F32 on MG_MIXED. */
int mg_smooth(mg_handle *h, int level, int dtype, void *x, const void *b, int sweeps, int order);

/* The V-cycle's downward step, fused as the cycle runs it: x <- `sweeps` pre-smoothing
 * sweeps (red then black) starting from x (from zero when x_is_zero; x's contents are
 * then ignored), and bc (level+1) = mean of the 8 children of b - A_l x. */
int mg_presmooth_restrict(mg_handle *h, int level, int dtype, void *x, const void *b, int sweeps,
                          int x_is_zero, void *bc);

/* The V-cycle's upward step, fused as the cycle runs it: x <- `sweeps`
 * post-smoothing sweeps (black then red) of x + P ec (ec on level+1). */
int mg_prolong_postsmooth(mg_handle *h, int level, int dtype, const void *ec, void *x, const void *b,
                          int sweeps);

/* r = b - A_l x, and (if norm2 != NULL) |r|_2 on the host (synchronises). */
int mg_residual(mg_handle *h, int level, int dtype, const void *x, const void *b, void *r,
                double *norm2);

/* bc (level+1) = mean of the 8 children of (b - A_l x). */
int mg_residual_restrict(mg_handle *h, int level, int dtype, const void *x, const void *b,
                         void *bc);

/* x (level) += P ec (ec on level+1), with the handle's prolongation kind. */
int mg_prolong_correct(mg_handle *h, int level, int dtype, const void *ec, void *x);

/* e = A_c^+ (r - mean r) on the coarsest level (FP64 arithmetic for both dtypes). */
int mg_coarse_solve(mg_handle *h, int dtype, const void *r, void *e);

/* ---- instrumentation ------------------------------------------------------------
 * With profiling on, the library records a CUDA event pair around every launch
 * of a level-0 kernel class below, and around each of the coarser groups below
 * (on the handle's stream), and accumulates the elapsed device time per class.
 * It measures the kernels inside real solves; it adds two event records per
 * timed interval and nothing else. */
enum {
    MG_PROF_SMOOTH = 0,         /* finest-level fused sweep passes (with the restriction or
                                   prolongation some of them carry) */
    MG_PROF_RESID_RESTRICT = 1, /* finest-level standalone residual + restriction (pre = 0) */
    MG_PROF_PROLONG = 2,        /* finest-level standalone prolongation + correction (post = 0) */
    MG_PROF_COARSE = 3,         /* dense coarse solve when the finest level is the coarsest */
    MG_PROF_FINE_RESIDUAL = 4,  /* FP64 residual / norm pass of the outer loop */
    MG_PROF_UPDATE = 5,         /* MIXED solution update */
    MG_PROF_ADJOINT_GRAD = 6,   /* fused adjoint gradient kernel */
    MG_PROF_PROJECT = 7,        /* velocity correction (mg_project) */
    MG_PROF_DENSITY_GRAD = 8,   /* density adjoint (mg_density_grads) */
    MG_PROF_COARSE_LEVELS = 9,  /* the V-cycle below the finest level: one interval per V-cycle
                                   (the replayed graph of its launches, or the launches) */
    MG_PROF_SETUP = 10,         /* operator set-up: one interval per mg_set_density /
                                   mg_set_face_coeffs (faces, coarsening, packs, coarse inverse) */
    MG_PROF_RHS = 11,           /* right-hand side (mg_rhs) */
    MG_PROF_DENSITY = 12,       /* density from the fractions (mg_density_from_fractions) */
    MG_PROF_NCLASS = 13
};

/* Turn timing on (1) or off (0); either way the accumulated totals are reset. */
int mg_profile(mg_handle *h, int enable);

/* Intervals timed (launches, or V-cycles / calls for the grouped classes) and their
 * total device milliseconds for one class. */
int mg_profile_read(mg_handle *h, int cls, long long *launches, double *ms);

/* Number of CUDA kernels this library has launched in this process (all handles). */
long long mg_kernel_launches(void);

/* Test hook: arm one-shot faults on this handle, for tests of the failure paths (0 disarms).
 *   MG_INJECT_FUSED_WAIT  the next fused sweep (opts.fused_sweeps, grid with nz >= 3): its first
 *                         block issues no copies for one plane while still announcing their
 *                         bytes, so that block's bounded wait runs out (about a second) with no
 *                         copy in flight to that stage; it sets bit 4 of the device error word,
 *                         later blocks return at once, and the solve returns MG_ERR_CUDA and
 *                         clears the error word (the handle stays usable).
 *   MG_INJECT_DIVERGE     the next outer residual norm the solve reads back (after its first
 *                         V-cycle or outer iteration) is replaced by infinity on the host: the
 *                         solve returns MG_ERR_DIVERGED.
 * Each fault fires once.  MG_ERR_ARG for unknown bits. */
enum { MG_INJECT_FUSED_WAIT = 1, MG_INJECT_DIVERGE = 2 };
int mg_debug_inject(mg_handle *h, int faults);

/* FP64 fused multiply-add rate of the current device, for the roofline of the FP64
 * kernels (no handle needed).  Launches `blocks` blocks of 256 threads, each thread running 8
 * independent chains of `iters` dependent FP64 FMAs; one short untimed launch, then one timed
 * launch with CUDA events on `stream` (a cudaStream_t, NULL = legacy default stream).
 * sink: device array of at least `blocks` doubles (overwritten with per-block sums, so that
 * no chain is dead code).  *tflops = 2 * FMAs / time (an FMA counts as two flops; an FP64
 * add or multiply issues at the FMA rate, so one FP64 instruction per second counts half of
 * this figure); *ms (may be NULL) = the timed launch's duration.  Synchronises `stream`.
 * MG_ERR_ARG for a null sink/tflops or non-positive sizes; MG_ERR_CUDA if a launch fails. */
int mg_fp64_fma_rate(void *stream, double *sink, int blocks, int iters, double *tflops, double *ms);

/* ---- domain decomposition in z slabs -------------------------------------------------------
 * The decomposition of the paper's MPI runs (§4.1; the multigrid level switches named as a
 * scaling cost in §4.3.2) for the FP64 V-cycle, with every rank's slab held as its own buffers
 * on the current GPU.  Level l of the hierarchy (the levels of mg_create) is cut into `ranks`
 * slabs of planes[l] = nz_l / ranks planes along z while it is not the coarsest level and every
 * slab keeps an even number (>= 2) of planes (so that each restriction pair stays inside one
 * slab), for at most max_decomposed levels (0: as many as allowed).  A slab holds its own
 * planes plus one ghost plane of x below and above; after every red or black half sweep and
 * after the prolongation the neighbours' boundary planes are copied into the ghost planes
 * (the halo exchange).  From switch_level on the hierarchy is held whole by one rank: the
 * last decomposed level's restriction writes every slab's coarse planes into one array (the
 * gather), a whole-grid handle runs the rest of the V-cycle, and each slab's prolongation
 * reads its coarse planes and their neighbours from there.  The norm and the mean of p are
 * sums of per-slab partial sums.  One V-cycle gives bitwise the whole-grid FP64 V-cycle.
 * The mixed-precision solve (precision MG_MIXED) cuts its levels the same way, down to the
 * deepest switch level its kernels allow (every cut level's nx a multiple of 16, the last cut
 * level's slabs a multiple of 4 planes): FP32 slabs of the colour-split layout with a ghost plane
 * per colour below and above, an exchange of the colour just updated after every half sweep and
 * after the prolongation, the last cut level's restriction written into the whole-grid handle's
 * FP32 level, the rest of each inner V-cycle on that handle, and the FP64 outer loop (residual,
 * norms, update) slab by slab with p's ghost planes exchanged before each residual; every cell
 * sees the whole-grid mixed solve's arithmetic, the outer loop's FP32-accumulated sums
 * differing in grouping only.
 * Arrays passed in and out are whole-grid device arrays (cell layout above). */
#define MG_DD_MAX_RANKS 64
typedef struct mg_dd mg_dd;
typedef struct {
    int ranks;                      /* slabs */
    int levels;                     /* levels of the hierarchy (as mg_num_levels) */
    int switch_level;               /* first level held whole; levels below are cut (>= 1) */
    int nx[MG_MAX_LEVELS], ny[MG_MAX_LEVELS], nz[MG_MAX_LEVELS];  /* whole-grid dims per level */
    int planes[MG_MAX_LEVELS];      /* planes per slab on the cut levels, 0 from switch_level */
} mg_dd_plan;

/* The plan alone (host only, no GPU): MG_ERR_ARG if level 0 cannot be cut (nz not a multiple
 * of 2 * ranks, a single level, bad sizes).  Rank r owns planes [r planes[l], (r+1) planes[l])
 * of level l; its neighbours are r - 1 and r + 1. */
int mg_dd_make_plan(int nx, int ny, int nz, int coarsest, int ranks, int max_decomposed, mg_dd_plan *plan);

/* Create a decomposed solver.  opts: method MG_METHOD_VCYCLE, warm_start 0, and either
 * precision MG_FP64 with inner_cycles 1, or precision MG_MIXED (inner_cycles as for mg_create)
 * with pre >= 1, post >= 1, trilinear prolongation, nx a multiple of 16 and nz a multiple of
 * 4 * ranks; other fields as for mg_create.  MG_ERR_ARG otherwise.
 * Allocates every slab's buffers and the whole-grid handle of the switch level on the current
 * device. */
int mg_dd_create(const mg_opts *opts, int ranks, int max_decomposed, void *stream, mg_dd **out);
int mg_dd_destroy(mg_dd *dd);
const char *mg_dd_last_error(const mg_dd *dd);
int mg_dd_get_plan(const mg_dd *dd, mg_dd_plan *plan);
/* Halo exchanges of one V-cycle and the bytes they copy between slabs (mixed: FP32 planes of
 * one colour; the outer loop's exchange of p's FP64 planes, once per outer iteration, apart). */
int mg_dd_traffic(const mg_dd *dd, long long *exchanges, long long *halo_bytes);
/* Operator from a whole-grid density (as mg_set_density); each slab takes its faces, the
 * coarse slabs are coarsened slab by slab.  Synchronises. */
int mg_dd_set_density(mg_dd *dd, const double *rho);
/* One FP64 V-cycle for A x = b (b as given, no mean removed), x in place; FP64 solvers only
 * (MG_ERR_ARG for a mixed one).  Synchronises. */
int mg_dd_vcycle(mg_dd *dd, const double *b, double *x);
/* As mg_solve in the solver's precision (MG_FP64 or MG_MIXED): zero-mean p with
 * A p = b - mean(b) to opts.rtol, from p = 0. */
int mg_dd_solve(mg_dd *dd, const double *b, double *p, mg_stats *stats);

/* ---- allocation-free entry point ----------------------------------------------------
 * The paper has no counterpart to this call.  It exists for callers that cannot
 * allocate device memory when they need a solve: programs whose device memory
 * belongs to another allocator (a framework's caching pool, where an extra
 * cudaMalloc can fail or fragment the pool), loops held to a fixed memory
 * budget, and code that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree may cause.
 *
 * e = A^+ (r - mean r): the exact zero-mean solution of the cell-centred
 * Neumann operator above on a small grid, for face coefficients bx, by, bz in
 * the face layouts (wall entries ignored; interior entries finite and > 0,
 * else MG_ERR_DENSITY).  r, e: cell arrays.  All pointers are device
 * pointers; `stream` is a cudaStream_t (NULL = legacy default stream).  The
 * call builds the dense pseudo-inverse from scratch and applies it; it needs
 * no handle and calls no cudaMalloc, cudaFree or other allocating routine.
 * Working memory is one fixed array in this library's device image (about
 * 2.1 MB, held on every GPU that loads the library until the process exits),
 * so nx*ny*nz must be at most MG_NOALLOC_MAX_CELLS (MG_ERR_ARG otherwise).
 * The first call on each device looks up that array's device address (with
 * that device current); make it before any stream capture.  Every call uses
 * the same array, which keeps the previous call's contents: calls that can
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The call reads its error word back to the host
 * and synchronises `stream` before returning. */
#define MG_NOALLOC_MAX_CELLS 512
int mg_dense_solve_noalloc(int nx, int ny, int nz, double h, const double *bx, const double *by,
                           const double *bz, const double *r, double *e, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MG_POISSON_H */
