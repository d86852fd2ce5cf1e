/*
 * grav.h — C ABI of libgrav.so: a matrix-free rectangular-prism gravity
 * operator and its depth-weighted data-space inversion on one NVIDIA B300
 * (sm_103a).
 *
 * The operator (the paper's Section 2.1, Eq. 1-6):
 *     d_i = sum_k G_ik m_k,   G_ik = gamma * sum_{p,q,r in {1,2}} (-1)^(p+q+r) Psi(x_p, y_q, z_r)
 *     Psi(x,y,z) = z atan(x y / (z R)) - x ln(R + y) - y ln(R + x),  R = |(x,y,z)|     (Eq. 2-3)
 * with (x_p, y_q, z_r) the prism vertices relative to station i.  G is never
 * stored: every product recomputes it.
 *
 * The inversion (Section 2.2, Eq. 7-11, with W_d = lambda I and
 * W_m = W^-2 = diag((zc_k + z0)^2)):
 *     m = m_ref + W^-2 G^T (G W^-2 G^T + lambda I)^-1 (d - G m_ref),
 *     lambda = lambda_scale * trace(G W^-2 G^T) / N,
 * solved by conjugate gradients on the N x N system (Section 3.1: the
 * inversion is iterative CG with no factorisation).
 *
 * Conventions
 *   - Units: metres, kg/m^3, data in mGal (1 mGal = 1e-5 m/s^2);
 *     gamma = 6.67430e-11 m^3 kg^-1 s^-2.
 *   - z is DEPTH, positive down.  The mesh top is ze[0].  Every station must
 *     lie strictly above the mesh top (station z < ze[0]); the result for a
 *     station at or below the top is unspecified (finite or NaN values, never
 *     a memory fault).
 *   - Cell k = (i, j, l) has linear index k = i + nx*(j + ny*l).
 *   - g_z is reported positive down: a positive contrast below a station
 *     gives a positive anomaly.
 *   - Ownership: the caller owns every input and output buffer.  The library
 *     owns only its scratch, which lives inside a grav_ctx or a grav_plan.
 *   - Streams: every call enqueues its work on the given stream and returns
 *     without waiting for it, unless stated otherwise.  Calls sharing one
 *     grav_ctx or one grav_plan must be ordered (same stream, or explicitly
 *     synchronised): their scratch is shared.
 *   - Errors: every function returns GRAV_OK (0) or a negative GRAV_E* code
 *     and leaves a message for grav_last_error().  Invalid arguments are
 *     rejected before anything is enqueued.  Kernels never trap; a bounded
 *     device-side wait that gives up sets a device status word that the next
 *     synchronising call reports as GRAV_EDEVICE.
 */
#ifndef GRAV_H_
#define GRAV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t), passed through opaquely; NULL = legacy default stream. */
typedef struct CUstream_st *grav_stream_t;

/* ---- status codes --------------------------------------------------------- */
#define GRAV_OK              0
#define GRAV_EINVAL         -1   /* bad argument, descriptor or size */
#define GRAV_ENOMEM         -2   /* device allocation failed / over the HBM budget */
#define GRAV_ENOTCONVERGED  -3   /* CG hit max_iter; the last iterate is still written */
#define GRAV_ETIMEDOUT      -4   /* a bounded host wait expired */
#define GRAV_EDEVICE        -5   /* CUDA error or device status word set */
#define GRAV_ECANCELED      -6   /* job cancelled */
#define GRAV_ENOTFOUND      -7   /* unknown job id */
#define GRAV_EBUSY          -8   /* the serving queue is full */

/* ---- precision modes ------------------------------------------------------ */
/* GRAV_FP64: Eq. 1-3 evaluated in FP64 once per (station, mesh node) and
 *   differenced across shared nodes (summation by parts of Eq. 1 + Eq. 5).
 *   Needs nx+1 <= 8528 (a row of node weights is staged in shared memory);
 *   GRAV_EINVAL otherwise.
 * GRAV_MIXED: every cell contributes through an FP32 point-mass far-field term
 *   gamma rho V dz / R^3 (times the box's quadrupole factor when the cells are
 *   not cubes) with compensated (two-sum) accumulation; cells whose centre
 *   lies within near_cells cell widths (width = the largest cell edge) of a
 *   station are corrected to the exact FP64 prism value (Eq. 1) for that
 *   station.  CG dots and step lengths stay in FP64.  The input vector (m for
 *   the forward, r for the adjoint) is divided by its largest magnitude before
 *   the FP32 arithmetic and the FP64 result multiplied back, so a product
 *   scales exactly with a power-of-two scaling of its input at any magnitude.
 *   Requires a uniform mesh (constant dx, dy, dz; a x b x c cells with any
 *   a, b, c); GRAV_EINVAL otherwise.
 */
#define GRAV_FP64    0
#define GRAV_MIXED   1
/* GRAV_MIXED_CORNER: the literal reading "FP32 corner terms with compensated
 *   summation, FP64 only for near-field prisms": Eq. 2-3 in FP32 at every mesh
 *   node (node-shared) plus the same FP64 near-window correction as
 *   GRAV_MIXED.  Forward product only (grav_forward / grav_plan_forward); it
 *   exists to measure that scheme's error, which FP32 cancellation of the
 *   corner differences makes far larger than GRAV_MIXED's (2.8e-5 against
 *   7.3e-7 of max|d| on an 80 x 80 x 40 mesh of 50 m cells, 6,561 stations). */
#define GRAV_MIXED_CORNER 2

/* ---- descriptors ---------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;            /* cells per axis, each >= 1 */
    const double *xe;          /* HOST array, nx+1 strictly increasing x edges (m) */
    const double *ye;          /* HOST array, ny+1 strictly increasing y edges (m) */
    const double *ze;          /* HOST array, nz+1 strictly increasing depths (m); ze[0] = mesh top */
} grav_mesh;

typedef struct {
    int64_t n;                 /* number of stations: >= 1 for plans and jobs; the one-shot calls also take
                                  n = 0 (x, y, z unused): forward writes nothing, adjoint writes zeros, diag
                                  writes nothing (trace 0), the inversion writes m_ref (or zeros) */
    const double *x, *y, *z;   /* DEVICE arrays of n doubles; z = -(height above z = 0) */
} grav_survey;

typedef struct {
    int precision;             /* GRAV_FP64, GRAV_MIXED or GRAV_MIXED_CORNER (forward only) */
    double z0;                 /* depth-weight offset (m): W^-2 = (zc + z0)^2, zc = cell-centre depth below ze[0] */
    double lambda_scale;       /* lambda = lambda_scale * trace(G W^-2 G^T) / N  (default 1e-2) */
    double lambda;             /* > 0: use this lambda instead of the trace rule */
    double tol;                /* CG stops when ||dd - A y|| <= tol ||dd|| (recurrence residual) */
    int max_iter;              /* CG iteration cap */
    int check_every;           /* host convergence check period in iterations (0 = automatic) */
    double near_cells;         /* GRAV_MIXED near-field radius in cell widths (default 8) */
    double timeout_s;          /* bound on every host wait of a call (default 3600 s) */
    int precond;               /* CG preconditioner: 0 none, 1 Jacobi, diag(G W^-2 G^T + lambda I)^-1, 2 randomized
                                  Nystrom (Frangella, Tropp and Udell 2023) of G W^-2 G^T from nys_rank products
                                  with the operator on a mesh coarsened nys_coarsen times per axis (uniform
                                  meshes; single CG solve; N*(nys_rank + reorth)*8 extra bytes, and during
                                  the set-up 8*N*nys_rank bytes more plus one block of the explicit coarse
                                  operator of at most 4 GB) (default 0) */
    int cache_g;               /* GRAV_FP64 only: 1 = build G explicitly once when it fits the context budget
                                  (formed in FP64, kept as double-float pairs: N*M*8 bytes, a 48-bit
                                  significand) and stream it for every product, computed in double-float
                                  arithmetic (an FP64 GEMV is bound by this GPU's FP64 pipe, below HBM
                                  speed); 0 = always recompute (default 0) */
    int outer_max;             /* > 0: the paper's outer model-update loop (Section 2.2): at most outer_max
                                  updates y += alpha dy, dy from <= inner_max CG iterations on A dy = dd - A y,
                                  alpha by backtracking on the objective of Eq. 7; 0 = one CG solve (default) */
    int inner_max;             /* CG iterations per outer update (default 20) */
    int reorth;                /* single CG solve without preconditioner (precond = 0, outer_max = 0): keep up
                                  to this many normalised residuals (N*reorth*8 bytes of HBM, at most 4096)
                                  and reorthogonalise every new residual against them (twice), which
                                  restores the convergence CG loses to rounding on this system (a restart
                                  from the true residual starts a fresh basis; at most 16 restarts);
                                  0 = plain CG (default 1000) */
    int check_stations;        /* mixed modes, > 0: state the error of the result against the FP64 operator
                                  at this many evenly spaced stations (inversions: of G m_out; serving
                                  forward jobs: of d), in grav_solve_info.fp64_rel_err; 0 = off (default) */
    int nys_rank;              /* precond = 2: sketch size ell (products with the coarse operator), 1..8192;
                                  0 = automatic: GRAV_MIXED N / 45 clamped to [100, 4000], GRAV_FP64
                                  min(3000, N / 2) (default 0) */
    int nys_coarsen;           /* precond = 2: coarsening factor per axis of the sketch operator, 1..8;
                                  0 = automatic: GRAV_MIXED min(3, min(nx, ny, nz) / 8), at least 1;
                                  GRAV_FP64 1 (default 0) */
    int refine;                /* GRAV_FP64 inversions (grav_datainv_solve*, uniform meshes): > 0 solves the FP64
                                  system by mixed-precision iterative refinement, at most `refine` correction
                                  steps: each runs a GRAV_MIXED CG solve (near_cells, precond, nys_*, reorth,
                                  max_iter apply to it; tolerance tol / 2 (not below 2e-7) for the first step, 1e-2 of the current
                                  residual after that) on the current residual, adds its solution to y and
                                  recomputes the residual dd - (G W^-2 G^T + lambda I) y with the FP64
                                  operator; it stops when that FP64 residual is <= tol ||dd||.  lambda comes
                                  from the trace as in FP64 mode (diag_fp64 picks its arithmetic), and
                                  m = m_ref + W^-2 G^T y from the FP64 adjoint of the final y (the one its
                                  residual used).  No counterpart in the paper.  0 = FP64 CG (default) */
    int near_fp64;             /* GRAV_MIXED: 1 = form the near-field table from the corner function in FP64;
                                  0 (default) = in double-float (pairs of FP32 numbers on the FP32 pipe,
                                  ~2^-45 of R (|ln R| + 1) per corner value against the ~2^-39 the table's
                                  FP32 entries need; the products differ from the FP64-formed table's by
                                  <= ~1e-9 of max, and the set-up is ~3x faster) */
    int diag_fp64;             /* GRAV_FP64 (matrix-free): 1 = the diagonal of G W^-2 G^T (the trace for lambda
                                  and the Jacobi preconditioner) from the corner function in FP64; 0 (default)
                                  = in double-float (FP32 pairs on the FP32 pipe): a sum of squares, so the
                                  ~2^-45 per-node error stays at <= ~3e-13 of each entry for stations over
                                  the mesh (~1e-11 for stations far off it, whose entries are all far
                                  field), 13x faster */
} grav_options;

typedef struct {
    int iters;                 /* CG iterations performed */
    int converged;             /* 1 if the recurrence residual reached tol */
    double rel_res;            /* recurrence ||r|| / ||dd|| at exit */
    double true_rel_res;       /* ||dd - (G W^-2 G^T + lambda I) y|| / ||dd||, recomputed with the same operator */
    double lambda;             /* lambda used */
    double trace;              /* trace(G W^-2 G^T) (0 if lambda was given) */
    double seconds;            /* wall time of the solve */
    int outer;                 /* outer updates performed (outer_max > 0); with refine, FP64 residual evaluations */
    double alpha_min;          /* smallest accepted step length of the outer loop (1 if never backtracked) */
    int restarts;              /* single CG solve: restarts from the recomputed true residual */
    double fp64_rel_err;       /* check_stations > 0: max |mixed - FP64| over the checked stations relative to
                                  max |g|: the larger of max |FP64| there and max |d_i| over every station
                                  (see grav_plan_check_fp64); -1 when not checked */
    double nys_shift;          /* precond = 2: the shift nu / lambda the Nystrom factorisation needed
                                  (1e-3 unless T lost definiteness); 0 otherwise */
    double nys_setup_s;        /* precond = 2: wall time of the preconditioner's set-up (sketch, Gram
                                  matrices, host factorisation and inverse); 0 otherwise */
} grav_solve_info;

typedef struct grav_ctx grav_ctx;
typedef struct grav_plan grav_plan;

/* Fills *opt with the defaults: GRAV_FP64, z0 = 50, lambda_scale = 1e-2,
 * lambda = 0, tol = 1e-6, max_iter = 1000, check_every = 0,
 * near_cells = 8, timeout_s = 3600, precond = 0, cache_g = 0, outer_max = 0,
 * inner_max = 20, reorth = 1000, check_stations = 0. */
void grav_options_default(grav_options *opt);

/* Library version string (static storage). */
const char *grav_version(void);

/* ---- context -------------------------------------------------------------- */
/* Creates a context on CUDA device `device`.  hbm_budget (bytes) caps the
 * device memory the context's plans and serving jobs may hold (0 = 90 % of
 * the device's free memory at creation).  Returns GRAV_EINVAL for a bad
 * device, GRAV_EDEVICE if the device cannot be initialised. */
int grav_ctx_create(grav_ctx **out, int device, size_t hbm_budget);

/* Destroys the context: waits (bounded by 60 s) for its serving jobs to stop,
 * frees its scratch.  Plans created from it must be destroyed first. */
int grav_ctx_destroy(grav_ctx *ctx);

/* Message of the last error on this context (thread-local per context; never NULL). */
const char *grav_last_error(grav_ctx *ctx);

/* Blocks (bounded by timeout_s) until `stream` is idle and reports any
 * device status word set by this context's kernels (GRAV_EDEVICE). */
int grav_ctx_sync(grav_ctx *ctx, grav_stream_t stream, double timeout_s);

/* ---- one-shot operator calls (Section 2.1, Eq. 5-6) ----------------------- */
/* d[i] = sum_k G_ik m[k] (mGal).  m: DEVICE, nx*ny*nz doubles (kg/m^3).
 * d: DEVICE, survey->n doubles.  opt may be NULL (defaults).  Builds a
 * transient plan (GRAV_MIXED: includes the near-field set-up), enqueues
 * the product and releases the plan in stream order. */
int grav_forward(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey,
                 const double *m, double *d, const grav_options *opt, grav_stream_t stream);

/* gtr[k] = sum_i G_ik r[i], times (zc_k + z0)^2 when depth_weighted != 0.
 * r: DEVICE, survey->n doubles; gtr: DEVICE, nx*ny*nz doubles. */
int grav_adjoint(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey,
                 const double *r, double *gtr, int depth_weighted,
                 const grav_options *opt, grav_stream_t stream);

/* diag[i] = sum_k G_ik^2 (zc_k + z0)^2, the diagonal of G W^-2 G^T, and
 * (when trace != NULL, HOST) its sum.  diag: DEVICE, survey->n doubles.
 * Synchronises the stream when trace != NULL. */
int grav_diag(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey,
              double *diag, double *trace, const grav_options *opt, grav_stream_t stream);

/* ---- data-space inversion (Section 2.2, Eq. 10-11) ------------------------ */
/* m_out = m_ref + W^-2 G^T y with (G W^-2 G^T + lambda I) y = d - G m_ref,
 * y by CG from y = 0.  d: DEVICE, n doubles (mGal).  m_ref: DEVICE, M
 * doubles or NULL (zero).  m_out: DEVICE, M doubles.  y_out: DEVICE, n
 * doubles, or NULL.  info: HOST, may be NULL.  Synchronises `stream`
 * (bounded host waits).  Returns GRAV_ENOTCONVERGED, with m_out written from
 * the last iterate, when max_iter is reached. */
int grav_datainv_solve(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey,
                       const double *d, const double *m_ref, double *m_out, double *y_out,
                       grav_solve_info *info, const grav_options *opt, grav_stream_t stream);

/* grav_datainv_solve with two additions (the paper has no counterpart; they
 * serve checkpoint / resume and convergence records):
 *   y0: DEVICE, n doubles, or NULL — CG starts from y = y0 instead of 0, e.g.
 *       the y_out of an earlier call that stopped at max_iter (resume); the
 *       tolerance stays relative to ||d - G m_ref||.
 *   res_hist: DEVICE, res_hist_len doubles, or NULL — the single CG solve
 *       writes its recurrence relative residual after iteration k into
 *       res_hist[k] (k < res_hist_len); unused entries are -1.
 * GRAV_EINVAL for host pointers or res_hist_len < 1 with res_hist given. */
int grav_datainv_solve_ex(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey,
                          const double *d, const double *m_ref, double *m_out, double *y_out,
                          grav_solve_info *info, const grav_options *opt, grav_stream_t stream,
                          const double *y0, double *res_hist, int res_hist_len);

/* ---- reusable plans ------------------------------------------------------- */
/* A plan holds one (mesh, survey, options) problem resident on the device:
 * the mesh edges, the station arrays' derived forms, the operator scratch and,
 * for GRAV_MIXED, the near-field correction of every station.  The
 * survey arrays are read when the plan is created and must not change while
 * the plan is used.  Creation enqueues set-up work on `stream`. */
int grav_plan_create(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey,
                     const grav_options *opt, grav_plan **out, grav_stream_t stream);
int grav_plan_forward(grav_plan *plan, const double *m, double *d, grav_stream_t stream);
int grav_plan_adjoint(grav_plan *plan, const double *r, double *gtr, int depth_weighted,
                      grav_stream_t stream);
/* Device bytes the plan holds. */
size_t grav_plan_bytes(const grav_plan *plan);
/* Releases the plan's memory in stream order after the work already
 * enqueued on `stream`. */
int grav_plan_destroy(grav_plan *plan, grav_stream_t stream);

/* ---- serving: continuous admission of jobs ------------------------------- */
/* A context runs a scheduler with K slots (default 4, or GRAV_SERVE_SLOTS in
 * the environment, or grav_serve_config before the first submit).  Each slot
 * is a host worker thread with its own non-blocking CUDA stream.  Submitted
 * jobs wait in a queue; a free slot takes the oldest job as soon as the job's
 * device footprint (its plan, plus the CG vectors for an inversion) fits in
 * the context's HBM budget next to the jobs already running.  When the oldest
 * job does not fit, the first later job that does may start instead
 * (backfill), at most 8 times before the oldest job is served first.  Jobs
 * therefore start while others are still on the GPU and their kernels
 * overlap on the device.
 *
 * Plans stay resident: a finished job leaves its plan (mesh tables, station
 * arrays, near-field table, the trace of G W^-2 G^T and, after a precond = 2
 * solve, its Nystrom preconditioner) in a cache of idle plans,
 * and a later job with the same mesh edges, the same survey arrays (device
 * pointers and n) holding the same values (a 64-bit fingerprint of x, y, z is
 * taken on the device when the job starts), and the same precision, z0,
 * near_cells and cache_g runs on it without building one; a Nystrom solve
 * with the same lambda, rank and coarsening also reuses the preconditioner.  Idle plans count
 * against the HBM budget and are released, least recently used first, when
 * an admission needs the memory or the cache exceeds its entry limit.  Every
 * kernel is deterministic and a reused plan holds the same tables, so a
 * job's result is bitwise the same alone, in a mix, and on a fresh or a
 * resident plan.  The serving entry points are the request-loop counterpart
 * of the paper's single inversion run (Section 3.1); the paper has no serving
 * layer. */
#define GRAV_JOB_FORWARD   0   /* output d = G input */
#define GRAV_JOB_INVERT    1   /* output m from data `input`, as grav_datainv_solve */

#define GRAV_JOB_QUEUED    0
#define GRAV_JOB_RUNNING   1
#define GRAV_JOB_DONE      2   /* finished; grav_wait returns GRAV_OK or GRAV_ENOTCONVERGED */
#define GRAV_JOB_FAILED    3
#define GRAV_JOB_CANCELED  4

typedef struct {
    int kind;                  /* GRAV_JOB_FORWARD or GRAV_JOB_INVERT */
    grav_mesh mesh;            /* HOST edges, copied at submit */
    grav_survey survey;        /* DEVICE arrays: must stay valid and unchanged until the job finishes */
    const double *input;       /* DEVICE: m (FORWARD, M doubles) or d (INVERT, n doubles) */
    const double *m_ref;       /* DEVICE, M doubles, or NULL (INVERT only) */
    double *output;            /* DEVICE: d (FORWARD, n doubles) or m (INVERT, M doubles) */
    grav_options opt;          /* copied at submit */
} grav_job;

/* Sets the number of slots (1..64); GRAV_EBUSY once the scheduler has started. */
int grav_serve_config(grav_ctx *ctx, int slots);
/* Validates and queues a job (never waits for the GPU).  GRAV_EINVAL for a bad
 * descriptor, GRAV_ENOMEM if the job alone exceeds the context budget,
 * GRAV_EBUSY if the queue is full.  *job_id receives the job's id. */
int grav_submit(grav_ctx *ctx, const grav_job *job, uint64_t *job_id);
/* Non-blocking: *state (GRAV_JOB_*) and, for inversions, the solve info so far. */
int grav_poll(grav_ctx *ctx, uint64_t job_id, int *state, grav_solve_info *info);
/* Waits at most timeout_s for the job to finish; returns the job's result
 * (GRAV_OK, GRAV_ENOTCONVERGED, GRAV_ECANCELED or the error that failed it),
 * or GRAV_ETIMEDOUT. */
int grav_wait(grav_ctx *ctx, uint64_t job_id, double timeout_s);
/* Cancels a queued job at once, or asks a running inversion to stop at its
 * next CG check (a running forward job completes). */
int grav_cancel(grav_ctx *ctx, uint64_t job_id);
/* Steady-clock times (seconds) of submission, start and end of a job (0 if not yet). */
int grav_job_times(grav_ctx *ctx, uint64_t job_id, double *t_submit, double *t_start, double *t_end);
/* Forgets a finished job's record (GRAV_EBUSY while queued or running). */
int grav_job_release(grav_ctx *ctx, uint64_t job_id);
/* Plan of a job: *plan_reused = 1 if it ran on a resident plan; *setup_s =
 * host wall time of building its plan (0 when reused); *footprint = the
 * device bytes its admission reserved.  Any pointer may be NULL. */
int grav_job_plan(grav_ctx *ctx, uint64_t job_id, int *plan_reused, double *setup_s, size_t *footprint);
/* At most max_plans idle plans stay resident (0..1024, default 16; 0 turns
 * the plan cache off).  May be called at any time; excess plans are released
 * at the next admission or job end. */
int grav_serve_plan_cache(grav_ctx *ctx, int max_plans);
/* Plans built and reused by the scheduler so far, idle plans resident now and
 * their device bytes.  Any pointer may be NULL. */
int grav_serve_stats(grav_ctx *ctx, int64_t *plans_built, int64_t *plans_reused, int *plans_resident,
                     size_t *bytes_resident);

/* ---- forward product without device allocation --------------------------- */
/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory while they run (a framework whose allocator
 * owns all device memory, a fixed pre-reserved memory budget, or code that
 * cannot afford the device synchronisation an allocation may imply): it needs
 * no grav_ctx and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Computes the same d = G m as grav_forward with GRAV_FP64, on the CURRENT
 * CUDA device and on `stream`.  mesh: HOST edge arrays as for every other
 * call.  survey arrays, m (nx*ny*nz doubles) and d (n doubles): DEVICE
 * pointers on the current device, owned by the caller.
 *
 * Scratch: one 64 MiB static device array inside libgrav (mesh edges, node
 * weights, per-chunk partial sums, a status word), held by every GPU that
 * loads the library until the process exits.  Problems whose node weights
 * ((ny+1)(nz+1)(nx+1 rounded up to even) doubles) plus one partial per
 * station do not fit are rejected with GRAV_EINVAL and a message naming the
 * sizes, as are meshes above 2^30 cells or 2^30 nodes and meshes with
 * nx+1 > 8528 (one row of node weights is staged in shared memory); all of
 * these are rejected before anything is enqueued.
 *
 * Device failure: the kernel's waits on its copies are bounded; if one runs
 * out, the product is incomplete and every entry of d is set to NaN (no host
 * synchronisation is needed to see it: check d).  GRAV_OK only means that
 * the work was enqueued.  Every call shares that array and keeps the previous call's
 * contents, so calls that overlap on the GPU (different streams, threads or
 * processes' contexts on the same device without ordering) race and give
 * wrong results: order them on one stream.  The first call on each device
 * looks the array's device address up (cudaGetSymbolAddress) and caches it;
 * make that first call before any stream capture.  Returns without waiting
 * for the GPU. */
int grav_forward_fp64_noalloc(const grav_mesh *mesh, const grav_survey *survey, const double *m, double *d,
                              grav_stream_t stream);

/* States the error of a product of this plan against the FP64 operator:
 * d (DEVICE, survey n doubles) is compared at n_check evenly spaced stations
 * (index floor(k n / n_check)) with G m evaluated in FP64 (Eq. 1-3, node
 * shared) on those stations alone.  m: DEVICE, M doubles.  *max_abs_err and
 * *rel_err (HOST; max |d - d64| at the checked stations, and that over max |g|,
 * taken as the larger of max |d64| there and max |d_i| over all n stations, so
 * that a sample missing the anomaly does not inflate it) may be NULL.
 * Synchronises `stream`.  Costs n_check / N of one FP64 forward product.
 * 1 <= n_check <= n, else GRAV_EINVAL. */
int grav_plan_check_fp64(grav_plan *plan, const double *m, const double *d, int n_check, double *max_abs_err,
                         double *rel_err, grav_stream_t stream);

/* ---- measurement ------------------------------------------------------------ */
/* Total number of CUDA kernels this library has launched in the process
 * (all contexts).  Used to attribute device work to libgrav in benchmarks. */
uint64_t grav_launch_count(void);

/* Writes a one-line JSON description of the plan's launch configuration
 * (kernels chosen, chunking, near-field box, device bytes) into buf (HOST,
 * len bytes, NUL-terminated, truncated if short).  Returns the length needed
 * including the NUL, or a negative GRAV_E* code. */
int grav_plan_describe(const grav_plan *plan, char *buf, size_t len);

/* Stage timing of one plan with CUDA events on the launching stream.
 * enable != 0 starts recording the device time of the plan's main kernels
 * (0 forward main kernel, 1 adjoint main kernel, 2 forward near-field apply,
 * 3 adjoint near-field apply); ms/counts (HOST, 4 entries each, may be NULL)
 * receive the summed milliseconds and launch counts recorded since the last
 * read (this waits for the recorded events) and reset them. */
int grav_plan_timing(grav_plan *plan, int enable, double *ms, int64_t *counts);

/* Pipe-rate microbenchmark on `device` (synchronous, ~0.2 s).  out (HOST, 19
 * doubles): [0] MUFU rsqrt/s, [1] SM MHz seen, [2] MUFU lg2/s, [3] MHz,
 * [4] FP32 FMA/s, [5] MHz, [6] FP64 FMA/s, [7] MHz, [8] FP32 FMA/s issued as
 * packed fma.rn.f32x2, [9] MHz, [10] SM count, then CUDA's FP64 functions:
 * [11] log/s, [12] MHz, [13] atan/s, [14] MHz, [15] sqrt/s, [16] MHz,
 * [17] divisions/s, [18] MHz, then this library's table-driven FP64 functions
 * used inside Eq. 2-3: [19] log/s, [20] MHz, [21] atan(a/b)/s, [22] MHz, then
 * MUFU [23] rcp/s, [24] MHz, [25] ex2/s, [26] MHz.
 * out: HOST, >= 27 doubles.  Per-clock rates per SM: rate / (MHz*1e6 * out[10]). */
int grav_bench_pipes(int device, double *out);

/* Self-check of the device-side failure path (the paper has no counterpart):
 * launches one kernel whose bounded mbarrier wait cannot complete (nothing
 * arrives), so it gives up after limit_ms (0 < limit_ms <= 1000), records the
 * timeout bit in the context's status word and returns; the call then reads
 * and clears the status word like every synchronising call.  Expected result:
 * GRAV_EDEVICE with a "bounded device wait expired" message, the context still
 * usable.  Synchronises `stream`. */
int grav_selftest_wait(grav_ctx *ctx, double limit_ms, grav_stream_t stream);

/* Self-check of the FP64 elementary functions inside Eq. 2-3 (the paper has
 * no counterpart): out[i] = f(a[i], b[i]) on ctx's device, with fn = 0 this
 * library's log(a), 1 its atan(a / b) (b > 0), 2 CUDA's log(a), 3 CUDA's
 * atan(a / b); and the double-float (FP32 pair) forms the near-field set-up
 * uses, arguments rounded to double-float and results returned as hi + lo:
 * 4 log(a), 5 atan(a / b) (b > 0), 6 Psi(x, y, z) of Eq. 2-3 with x = a[i],
 * y = b[i], z = a[n + i] > 0 (a holds 2n doubles for fn 6).  a, b (fn 1, 3,
 * 5 and 6), out: DEVICE, n doubles.  Enqueued on `stream`; GRAV_EINVAL for a
 * bad fn, n < 0 or NULL pointers. */
int grav_eval_fn64(grav_ctx *ctx, int fn, const double *a, const double *b, double *out, int64_t n,
                   grav_stream_t stream);

/* Self-check of the randomized Nystrom preconditioner's sketch operator
 * (precond = 2; not in the paper): Y = K_c X with K_c = G_c W_c^-2 G_c^T / c^3
 * the depth-weighted operator of the mesh coarsened c x c x c (cells of c
 * times the size, same origin and stations; GRAV_MIXED far term plus an FP64-
 * formed near-field table within 3 coarse cells), applied the way the sketch
 * applies it: explicit FP32 blocks of G_c W_c^-1 c^-3/2 and two FP32 GEMMs.
 * X, Y: DEVICE, column-major n x k doubles (X is rounded to FP32).  mesh must
 * be uniform; opt gives z0 (NULL: defaults).  1 <= coarsen <= 8, k >= 1, else
 * GRAV_EINVAL.  Synchronises `stream`. */
int grav_nystrom_coarse_apply(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, int coarsen,
                              const double *X, int k, double *Y, const grav_options *opt,
                              grav_stream_t stream);

/* Self-check of the dense kernels behind the Nystrom preconditioner (not in
 * the paper), on ctx's device, enqueued on `stream`:
 *   op 0: C (+)= A B, FP32, A(m, k) = A[k + lda m]  (C float, m-fastest: C[m + ldc n])
 *   op 1: C (+)= A B, FP32, A(m, k) = A[m + lda k]
 *         (ops 0-1: B(k, n) = B[k + ldb n]; M x N output, inner dimension K)
 *   op 2: C (+)= A^T A, lower triangle only (C double, C[i + N j], i >= j, i, j < N),
 *         A(k, i) = A[k + lda i], k < K; exact FP32 products, double-float sums.
 *   op 3: as op 1 with B(k, n) = B[n + ldb k] and C(m, n) = C[n + ldc m]
 *   op 4: as op 1 with B(k, n) = B[n + ldb k]
 *   op 5: as op 2 with A(k, i) = A[i + lda k]
 *   op 6: the preconditioner's FP64 factorisation: A is an N x N symmetric
 *         positive definite matrix of doubles (column-major, lower triangle
 *         read), C receives 2 N^2 doubles: L with T = L L^T in its lower
 *         triangle (the upper triangle keeps A's values) and then L^-1
 *         (column-major, zeros above the diagonal).  Synchronises the stream;
 *         GRAV_EDEVICE if a pivot is not positive.  M, K, B, lda, ldb, ldc and
 *         accumulate are not used.
 * accumulate = 1 adds to C.  All pointers DEVICE, 16-byte aligned; lda, ldb,
 * ldc, K (and M for ops 0-1, 3-4) multiples of 4; an n-major B or C (and the
 * op 5 A) needs rows of at least N rounded up to 4, whose padding may be
 * read (op 3: written); GRAV_EINVAL otherwise. */
int grav_dense_check(grav_ctx *ctx, int op, int M, int N, int K, const float *A, int64_t lda, const float *B,
                     int64_t ldb, void *C, int64_t ldc, int accumulate, grav_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GRAV_H_ */
