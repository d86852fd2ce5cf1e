// Internal host-side declarations of libgrav: context, plan, launchers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "grav.h"

namespace grav {

// Mesh-node lattice geometry handed to the FP64 kernels by value.
struct Geo {
    int nx, ny, nz;
    const double *xe, *ye, *ze;   // device edges
    int64_t N;                    // stations
    const double *fn = nullptr;   // device table of the FP64 log / atan (kFnTableSize doubles)
};

// Layout of the FP32 far-field operator (GRAV_MIXED).
struct MixedGeo {
    int nx, ny, nz, nzp;          // nzp: nz rounded up to a multiple of 4
    int ncol;                     // nx * ny
    const float *cx;              // [nx][2] cell-centre x as (hi, lo) relative to x_ref
    const float *cy;              // [ny][2]
    const float *czc;             // [nzp] cell-centre depth (FP32), padded
    int64_t N;
    float qa, qb, qg;             // quadrupole coefficients A, B, C of the a x b x c cells (0 for cubes)
    const float *ex;              // [nx+1][2] x edges as (hi, lo) relative to x_ref (GRAV_MIXED_CORNER)
    const float *ey;              // [ny+1][2]
    const float *ez;              // [nz+1] edge depths (FP32)
};

// Near-field box of GRAV_MIXED: per station, a bx x by x bz block of cells
// starting at column (i0, j0) (depth layers 0..bz-1).
struct NearGeo {
    int bx, by, bz;
    int slots;                    // bx * by * bz
    int ld;                       // table row stride in floats: slots rounded up to a multiple of 4
                                  // (16-byte rows for TMA bulk copies and float4 loads; pad entries 0)
    double radius_cells;          // near_cells
    double width;                 // cell width the radius is measured in: max(a, c)
    int nbx, nby;                 // bin grid: i0 + (bx-1) in [0, nbx)
};

struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
    bool overflow = false;
    void *take(size_t bytes) {
        size_t off = (used + 255) & ~size_t(255);
        if (!base || off + bytes > size) {
            overflow = true;
            return nullptr;
        }
        used = off + bytes;
        return base + off;
    }
};

}  // namespace grav

struct grav_ctx {
    int device = 0;
    size_t hbm_budget = 0;
    std::atomic<size_t> hbm_used{0};
    cudaMemPool_t pool = nullptr;
    int *d_status = nullptr;       // device status word
    int *h_status = nullptr;       // pinned mirror
    std::mutex err_mu;
    std::string last_error;
    int sm_count = 148;
    void *serve = nullptr;         // serving scheduler (serve.cpp)
    double *d_fn = nullptr;        // FP64 log / atan table (fp64_kernels.cu, fill_fn_table)
};

namespace grav {
// Stages whose device time a plan can record with CUDA events.
enum Stage : int { kStageFwdMain = 0, kStageAdjMain = 1, kStageFwdNear = 2, kStageAdjNear = 3, kStageCount = 4 };
struct StageTimer {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;         // pairs (start, stop)
    std::vector<int> stage_of;             // per used pair
    int used = 0;
    double ms[kStageCount] = {0, 0, 0, 0};
    int64_t count[kStageCount] = {0, 0, 0, 0};
};
}  // namespace grav

struct grav_plan {
    grav_ctx *ctx = nullptr;
    mutable grav::StageTimer timer;
    grav_options opt{};
    int nx = 0, ny = 0, nz = 0;
    int64_t N = 0, M = 0, Nn = 0;
    std::vector<double> xe, ye, ze;       // host copies
    bool cubic = false;
    bool uniform = false;                 // uniform a x b x c cells (needed by GRAV_MIXED)
    double cell_a = 0, cell_b = 0, cell_c = 0;   // uniform cell size along x, y, z (when uniform)
    grav::Arena arena;
    size_t bytes = 0;

    // common device data
    double *d_xe = nullptr, *d_ye = nullptr, *d_ze = nullptr;
    double *d_w2 = nullptr;               // [nz] (zc + z0)^2
    const double *sx = nullptr, *sy = nullptr, *sz = nullptr;   // caller's survey arrays

    // FP64 path
    int ldw = 0;                          // padded node-row length (nx+1 rounded to even)
    int f64_rows_per_chunk = 0, f64_nchunk = 0;
    int a64_groups = 0, a64_nschunk = 0, a64_schunk_len = 0;
    int f64_diag_jrows = 0, f64_diag_nchunk = 0;
    double *w = nullptr;                  // node weights [(ny+1)(nz+1)][ldw]
    double *part = nullptr;               // forward partials [nchunk][N]
    double4_16a *st4 = nullptr;               // stations (x, y, z, r)
    double *upart = nullptr;              // adjoint partials [nschunk][Nn]
    double *u = nullptr;                  // [Nn]
    int cached = 0;                       // 1: explicit G stored (cell-major [M][N], double-float pairs)
    int c_nchunk = 0;                     // cell chunks of the stored-G forward product
    float2 *Gc = nullptr;                 // G formed in FP64, kept as (hi, lo) FP32 pairs (8 bytes per entry)
    float2 *m_df = nullptr, *r_df = nullptr;   // the product's input vector split the same way ([M], [N])

    // mixed path
    grav::MixedGeo mg{};
    grav::NearGeo ng{};
    float *m_cx = nullptr, *m_cy = nullptr, *m_czc = nullptr;
    float *qT = nullptr;                  // [ncol][nzp] gamma*1e5*V*rho (FP32)
    float *qN = nullptr;                  // [M] the same values in natural cell order (near field)
    float *m_w2f = nullptr;               // [nzp] (zc + z0)^2 in FP32
    float4 *st32 = nullptr;               // stations (xh, xl, yh, yl)
    float2 *stz = nullptr;                // stations (z, r)
    unsigned long long *rmax_bits = nullptr;   // max|r| of the last mixed adjoint (bits of a double)
    unsigned long long *mmax_bits = nullptr;   // max|m| of the last mixed forward (bits of a double)
    int m_fwd_cols_per_chunk = 0, m_fwd_nchunk = 0;
    int m_adj_tz = 0, m_adj_ngz = 0, m_adj_nschunk = 0, m_adj_schunk_len = 0;
    int m_adj_bc = 0;                     // 1: broadcast adjoint layout (large meshes), 0: lanes split stations
    double *m_part = nullptr;             // [nchunk][N] forward partials (hi+lo in FP64)
    double *m_apart = nullptr;            // [nschunk][M] adjoint partials
    float *dG = nullptr;                  // [N][slots] near-field correction (mGal per kg/m^3), formed in double-float or FP64
    int *st_i0 = nullptr, *st_j0 = nullptr;   // box origin per station
    int *near_off = nullptr;              // [slots] cell offset of each window-box slot from the box origin
    double *diag_corr = nullptr;          // [N] near-field correction of diag(G W^-2 G^T)
    int *bin_start = nullptr;             // [nbins+1]
    int *bin_st = nullptr;                // [N] station indices sorted by bin
    double *near_corr = nullptr;          // [N] forward near-field correction scratch
    double *m_cellacc = nullptr;          // [M] adjoint scratch
    double *near_tpart = nullptr;         // per station tile: FP64 near adjoint sums over its cell region
    int near_adj_rows = 0;                // near adjoint: 3 layer-split, 2 warp-private, 1 station-streaming, 0 cell-tiled
    int near_fwd_tile = 0;                // near forward: 1 per station-bin tile (q staged), 0 warp per station
    float *cr_w32 = nullptr;              // GRAV_MIXED_CORNER: node weights, FP32 rows of cr_ldw
    double *cr_part = nullptr;            // [cr_nchunk][N] row-chunk partials of the corner forward
    int cr_ldw = 0, cr_rows_per_chunk = 0, cr_nchunk = 0;

    double trace_cache = 0.0;             // trace(G W^-2 G^T) of an earlier solve on this plan (0: none)
    // Resident Nystrom preconditioner (serving keeps plans): when keep_nys is
    // set, a solve leaves its preconditioner here and a later solve with the
    // same lambda, rank, coarsening and seed reuses it (nys_key: those four).
    int keep_nys = 0;
    void *nys_kept = nullptr;             // grav::NysState *, owned by the plan
    double nys_key[4] = {0, 0, 0, 0};

    // CG / diag scratch
    double *diag = nullptr;               // [N]
    double *vec = nullptr;                // CG vectors
    double *scal = nullptr;               // device scalars
};

namespace grav {

// error helpers (api.cu)
int set_error(grav_ctx *ctx, int code, const char *fmt, ...);
int cuda_error(grav_ctx *ctx, cudaError_t e, const char *what);

// plan internals (api.cu), used by the solver and the serving scheduler
int plan_create(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const grav_options &o,
                grav_plan **out, cudaStream_t s);
int plan_prepare(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const grav_options &o,
                 grav_plan **out);                      // validation + sizing, no device work
int plan_allocate(grav_plan *p, cudaStream_t s);        // deletes p on failure
size_t solve_bytes(const grav_plan *p);
void plan_destroy(grav_plan *p, cudaStream_t s);
int plan_forward_ex(grav_plan *p, const double *m, double *d, const double *add, double add_scale, cudaStream_t s);
int plan_adjoint_ex(grav_plan *p, const double *r, double *out, int depth_weighted, const double *add,
                    cudaStream_t s);
int plan_diag(grav_plan *p, double *diag, cudaStream_t s);
int read_status(grav_ctx *ctx, cudaStream_t s, double timeout_s);
// y0 (may be null): CG starts from y = y0; hist (may be null): the recurrence
// relative residual after each iteration, hist_len entries (-1 when unused).
int solve_on_plan(grav_plan *p, const double *d, const double *m_ref, double *m_out, double *y_out,
                  grav_solve_info *info, cudaStream_t s, const std::atomic<int> *cancel,
                  const double *y0 = nullptr, double *hist = nullptr, int hist_len = 0);

// Randomized Nystrom preconditioner of G W^-2 G^T + lambda I (nystrom.cu):
// Y (N x ell), the Cholesky factor L of the ell x ell Woodbury matrix,
// scratch t, the cuBLAS handle and the device block holding them.
struct NysState {
    int ell = 0;
    int64_t N = 0, ldy = 0;               // ldy: N rounded up to a multiple of 4
    double mu = 0.0, nu = 0.0;
    float *Y = nullptr;                   // Y = K_c Omega, ldy x ell, column-major (FP32 values)
    double *Linv = nullptr;               // L^-1, ell x ell column-major, lower (T = L L^T)
    double *t = nullptr, *u = nullptr, *v = nullptr;   // [ell] application scratch
    double *tp = nullptr;                 // [row chunks][ell] partial sums of Y^T r
    float *vh = nullptr, *vl = nullptr;   // [ell] v as FP32 pairs
    float *rh = nullptr, *rl = nullptr;   // [ldy] r as FP32 pairs
    char *mem = nullptr;
    size_t bytes = 0;
};
size_t nys_bytes(int64_t N, int ell);
void nys_sizes(const grav_plan *p, int *ell, int *cf);   // resolves the automatic (0) rank and coarsening
size_t nys_peak_bytes(const grav_plan *p);               // persistent + set-up HBM of nys_build
// Y = K_c X (N x k, device, column-major) with the explicit coarse operator of the sketch
int nys_coarse_apply(grav_plan *p, int cf, const double *X, int k, double *Y, cudaStream_t s);
int nys_build(grav_plan *p, double lam, int ell, int cf, uint64_t seed, NysState *st, cudaStream_t s);
void nys_apply(const NysState &st, const double *r, double *z, cudaStream_t s);
void nys_free(grav_plan *p, NysState *st, cudaStream_t s);
// device bytes a plan holds, its resident Nystrom preconditioner included
size_t plan_resident_bytes(const grav_plan *p);
// bounded host wait for an event (GRAV_ETIMEDOUT after timeout_s)
int host_wait(grav_ctx *ctx, cudaEvent_t ev, double timeout_s, const char *what);

// serving scheduler (serve.cpp)
void serve_shutdown(grav_ctx *ctx);

// kernel-launch accounting and stage timing (api.cu)
void note_launches(int n);
void stage_begin(const grav_plan *p, int stage, cudaStream_t s);
void stage_end(const grav_plan *p, int stage, cudaStream_t s);

// FP64 launchers (fp64_kernels.cu)
void fp64_setup(grav_plan *p, cudaStream_t s);
void launch_node_weights(const grav_plan *p, const double *m, cudaStream_t s);
void launch_fwd64(const grav_plan *p, cudaStream_t s);
// out[i] = fs * (scale * sum_c part[c][i] + add2[i]) + add_scale * add[i], fs = *fbits as a double
// (1 when fbits is null); add and add2 may be null
void launch_reduce_rows(const double *part, int nchunk, int64_t n, double scale, const double *add,
                        double add_scale, const double *add2, double *out, cudaStream_t s,
                        const unsigned long long *fbits = nullptr);
void launch_adj64(const grav_plan *p, const double *r, cudaStream_t s);
void launch_adj_finish(const grav_plan *p, const double *u, double scale, int depth_weighted,
                       const double *add, double *out, cudaStream_t s);
void launch_diag64(const grav_plan *p, double *diag, cudaStream_t s);
void launch_build_g64(const grav_plan *p, float2 *Gc, double *diag, cudaStream_t s);
void launch_cached_fwd(const grav_plan *p, const double *m, const double *add, double add_scale, double *d,
                       cudaStream_t s);
void launch_cached_diag(const grav_plan *p, double *diag, cudaStream_t s);
int cached_fwd_tiles(int64_t N);   // station tiles of the stored-G forward
int cached_fwd_ctas_per_sm();      // its resident CTAs per SM
void launch_cached_adj(const grav_plan *p, const double *r, int depth_weighted, const double *add, double *out,
                       cudaStream_t s);
size_t fwd64_smem_bytes(const grav_plan *p);
// Returns the number of kernels launched, or -1 (nothing launched) when the
// forward kernel's shared-memory limit cannot be set.
int launch_fwd64_raw(Geo g, int ldw, const double *m, double *w, int rows_per_chunk, int nchunk,
                     const double *sx, const double *sy, const double *sz, double *part, int *status,
                     cudaStream_t s);
int fwd64_stations_per_cta();
// Largest nx+1 whose padded node row (with the two stage buffers of one row
// each) fits k_fwd64's 200 KB dynamic shared memory.
int fwd64_max_nodes_x();

// mixed launchers (mixed_kernels.cu)
int mixed_setup(grav_plan *p, cudaStream_t s);   // 0 or a GRAV_E* code
int near_setup_warps(const grav_plan *p);         // 0: window too large for shared memory
// normalize: q in units of max|m| (mmax_bits); the forward's row reduction multiplies back
void launch_mixed_prep_q(const grav_plan *p, const double *m, cudaStream_t s, bool normalize);
void launch_mixed_fwd(const grav_plan *p, cudaStream_t s);
void launch_mixed_near_fwd(const grav_plan *p, const double *m, cudaStream_t s);
void launch_mixed_adj(const grav_plan *p, const double *r, cudaStream_t s);
void launch_mixed_adj_finish(const grav_plan *p, const double *r, int depth_weighted, const double *add,
                             double *out, cudaStream_t s);
void launch_mixed_diag(const grav_plan *p, double *diag, cudaStream_t s);
size_t mixed_scratch_bytes(const grav_plan *p);
// *bits = bit pattern of max |v_i| (a non-negative double), for n doubles on the device
void launch_absmax(const double *v, int64_t n, unsigned long long *bits, cudaStream_t s);
int mixed_fwd_tail(const grav_plan *p);   // 1: the far-field forward runs the layers left after groups of 4
int mixed_adj_last_group(const grav_plan *p);
// out_{x,y,z}[k] = s{x,y,z}[i_k], out_d[k] = d[i_k], i_k = floor(k n / n_check)
void launch_gather_check(const double *sx, const double *sy, const double *sz, const double *d, int64_t n,
                         int n_check, double *ox, double *oy, double *oz, double *od, cudaStream_t s);
int check_fp64(grav_plan *p, const double *m, const double *d, int n_check, double *max_abs, double *rel,
               cudaStream_t s);
// Host-side NVTX range around a library stage (visible in Nsight timelines and
// usable as an ncu --nvtx filter); costs nothing without a tool attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
// Device view of a plan's mesh, stations and function table.
Geo make_geo(const grav_plan *p);
// Host: fills the kFnTableSize-double table of the FP64 log / atan (long-double
// logl / atanl values split into high and low doubles).
void fill_fn_table(double *t);
int fn_table_size();
void launch_corner_fwd(const grav_plan *p, const double *m, cudaStream_t s);

// Device factorisation of the Nystrom matrix (chol_kernels.cu), FP64,
// column-major lower n x n: T = lam (M + nu I) + G; T = L L^T in place
// (*fail |= 1 on a pivot that is not positive); Li = L^-1 (zeros above the
// diagonal).  Enqueued on s.
void launch_form_T(int n, double lam, double nu, const double *M, const double *G, double *T, cudaStream_t s);
void launch_potrf_lower(double *A, int n, int *fail, cudaStream_t s);
void launch_trinv_lower(const double *L, double *Li, int n, cudaStream_t s);
// dense kernels of the Nystrom preconditioner (dense_kernels.cu).  Return -1
// (nothing launched) when the layout requirements are not met.
// C (+)= A B in FP32: A(m, k) = A[k + lda m] (a_kmajor) or A[m + lda k];
// B(k, n) = B[n + ldb k] (b_nmajor) or B[k + ldb n]; C(m, n) = C[n + ldc m]
// (c_nmajor) or C[m + ldc n].  lda, ldb, ldc, K, M (and N when b_nmajor or
// c_nmajor) multiples of 4, bases 16-byte aligned.
int launch_sgemm(bool a_kmajor, int M, int N, int K, const float *A, int64_t lda, const float *B, int64_t ldb,
                 float *C, int64_t ldc, bool accumulate, cudaStream_t s, bool b_nmajor = false,
                 bool c_nmajor = false);
// G (+)= X^T X (lower triangle, G[i + n j], i >= j) for X(k, i) = X[k + ldx i]
// (or X[i + ldx k] when k_slow), k < K, i < n; exact FP32 products,
// double-float sums.  ldx, K (n when k_slow) multiples of 4.
int launch_gram_df(int n, int K, const float *X, int64_t ldx, double *G, bool accumulate, cudaStream_t s,
                   bool k_slow = false);
// z = (r - Y Linv^T Linv Y^T r) / mu  (Y FP32 [ldy][ell], Linv FP64 lower)
int64_t nys_tpart_chunks(int64_t n);   // row chunks of the Y^T r partial sums (tp: chunks x ell doubles)
void launch_nys_apply(const float *Y, int64_t ldy, int64_t n, int ell, const double *Linv, double mu,
                      const double *r, double *z, float *rh, float *rl, double *tp, double *t, double *u, double *v,
                      float *vh, float *vl, cudaStream_t s);

// vector kernels (cg_kernels.cu)
void launch_dot(const double *a, const double *b, int64_t n, double *partials, double *out, cudaStream_t s);
constexpr int kDotBlocks = 296;

}  // namespace grav
