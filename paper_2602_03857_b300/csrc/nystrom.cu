// Randomized Nystrom preconditioner for the data-space system
//   A = K + lambda I,  K = G W^-2 G^T   (option precond = 2)
//
// Method: Frangella, Tropp and Udell, "Randomized Nystrom preconditioning",
// SIAM J. Matrix Anal. Appl. 44 (2023): a rank-ell Nystrom approximation
// K_hat = Y (Omega^T Y)^-1 Y^T from ell products Y = K Omega with a Gaussian
// test matrix Omega, and the preconditioner P = K_hat + lambda I.  Here:
//
// * K is sketched through the operator on a mesh coarsened cf x cf x cf
//   (cells cf a x cf b x cf c, same stations; 1/cf^3 of the pairs per
//   product).  A coarse cell's column of G is the sum of its cf^3 fine
//   columns, so sum_{k in C} w_k g_k g_k^T ~ (w_C / cf^3) g_C g_C^T and
//   K ~ G_c W_c^-2 G_c^T / cf^3.  Depth weighting makes K dominated by deep
//   cells, whose fields at the stations are smooth, so the coarse operator
//   carries K's leading eigenvectors.
// * Omega is Gaussian scaled by 1/sqrt(N) (no orthonormalisation: for
//   N >> ell its columns are already nearly orthonormal, and K_hat does not
//   depend on a change of basis of Omega's range); Y_nu = Y + nu Omega with
//   nu = sqrt(N) eps ||Y||_F keeps Omega^T Y_nu positive definite.
// * P^-1 by the Woodbury identity applied to K_hat = Y_nu M^-1 Y_nu^T,
//   M = Omega^T Y_nu:  (mu I + Y_nu M^-1 Y_nu^T)^-1 r
//     = (r - Y_nu T^-1 Y_nu^T r) / mu,  T = mu M + Y_nu^T Y_nu,  mu = lambda - nu,
//   with one ell x ell Cholesky factor T = L L^T (on the host).  Applying it
//   costs two GEMVs with the N x ell matrix Y_nu and two triangular solves.
//
// cuBLAS supplies the ell x ell GEMM and rank-k update and the GEMV / TRSV of the
// application (plain library dense algebra); the sketch products are this
// library's operator kernels.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "cg.h"
#include "internal.h"

namespace grav {
namespace {

// SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014): a bijective
// mix of a 64-bit counter, used as a counter-based uniform generator.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// out[i] = scale * N(0, 1) from the Box-Muller transform of two uniforms
// drawn from counters 2i and 2i+1 of the stream `seed` (deterministic).
__global__ void k_randn(double *__restrict__ out, int64_t n, uint64_t seed, double scale) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = splitmix64(seed ^ (2ull * (uint64_t)i));
        const uint64_t b = splitmix64(seed ^ (2ull * (uint64_t)i + 1ull));
        const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
        const double u2 = (double)(b >> 11) * 0x1.0p-53;           // [0, 1)
        out[i] = scale * sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    }
}

// y = a * y + b * x
__global__ void k_axpby_n(double a, double *__restrict__ y, double b, const double *__restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * y[i] + b * x[i];
}

inline unsigned grid_n(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 148LL * 32)); }

// sum_k a[k] b[k], k < n, in four interleaved partial sums
inline double dot4(const double *a, const double *b, int n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 4 <= n; k += 4) {
        s0 += a[k] * b[k];
        s1 += a[k + 1] * b[k + 1];
        s2 += a[k + 2] * b[k + 2];
        s3 += a[k + 3] * b[k + 3];
    }
    for (; k < n; ++k) s0 += a[k] * b[k];
    return (s0 + s1) + (s2 + s3);
}

// In-place Cholesky A = L L^T of a symmetric n x n row-major matrix (lower
// triangle used and overwritten with L), column by column (Cholesky-Crout:
// L_ij = (A_ij - L_i,<j . L_j,<j) / L_jj, rows of a column in parallel);
// false if a pivot is not positive.
bool cholesky_rowmajor(std::vector<double> &A, int n) {
    for (int j = 0; j < n; ++j) {
        double *Lj = &A[(size_t)j * n];
        const double d = Lj[j] - dot4(Lj, Lj, j);
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        Lj[j] = ljj;
        const double inv = 1.0 / ljj;
#pragma omp parallel for schedule(static) if (n - j > 256)
        for (int i = j + 1; i < n; ++i) {
            double *Li = &A[(size_t)i * n];
            Li[j] = (Li[j] - dot4(Li, Lj, j)) * inv;
        }
    }
    return true;
}

}  // namespace

size_t nys_bytes(int64_t N, int ell) {
    // persistent part: Y_nu (N x ell), L (ell x ell), t (ell)
    return 8ull * ((size_t)N * ell + (size_t)ell * ell + ell) + 3 * 256;
}

int nys_build(grav_plan *p, double lam, int ell, int cf, uint64_t seed, NysState *st, cudaStream_t s) {
    grav_ctx *ctx = p->ctx;
    NvtxRange nv("grav::nystrom_build");
    const int64_t N = p->N;
    if (!p->uniform) return set_error(ctx, GRAV_EINVAL, "precond = 2 (Nystrom) needs a mesh of uniform cells");
    // Automatic sizes (0).  The sketch products run on the mixed coarse
    // operator, so their cost relative to one CG iteration is ~1/cf^3 in mixed
    // mode but ~1/(600 cf^3) in FP64 mode, where a large sketch is nearly free.
    //   mixed: rank N / 60 in [100, 3000], coarsening min(4, smallest cell count / 8);
    //   FP64:  rank min(3000, N / 2), coarsening min(2, smallest cell count / 8).
    // Measured (inversion to 1e-6; without a preconditioner in brackets):
    //   210 x 210 x 75 cells x 178,797 stations, mixed: (rank, coarsening) (1000, 2)
    //   99.9 s, (2000, 3) 74.6 s, (3000, 3) 85.0 s, (3000, 4) 70.5 s [153 s];
    //   80 x 80 x 40 x 6,561, FP64: (109, 4) 119 s, (1500, 2) 30.4 s, (3000, 2) 24.4 s [99 s].
    const bool f64 = p->opt.precision == GRAV_FP64;
    const int mmin = std::min(p->nx, std::min(p->ny, p->nz));
    if (ell <= 0)
        ell = f64 ? (int)std::min<int64_t>(3000, std::max<int64_t>(1, N / 2))
                  : (int)std::min<int64_t>(3000, std::max<int64_t>(100, (N + 30) / 60));
    if (cf <= 0) cf = std::max(1, std::min(f64 ? 2 : 4, mmin / 8));
    ell = (int)std::min<int64_t>(ell, N);
    if (ell < 1 || cf < 1) return set_error(ctx, GRAV_EINVAL, "Nystrom rank and coarsening must be >= 1");
    *st = NysState{};
    st->ell = ell;
    st->N = N;
    // coarse mesh: cf x cf x cf cells of the same origin (it may reach past
    // the fine mesh by less than one coarse cell on each axis)
    const int nxc = (p->nx + cf - 1) / cf, nyc = (p->ny + cf - 1) / cf, nzc = (p->nz + cf - 1) / cf;
    std::vector<double> xc(nxc + 1), yc(nyc + 1), zc(nzc + 1);
    for (int i = 0; i <= nxc; ++i) xc[i] = p->xe[0] + (double)i * cf * p->cell_a;
    for (int j = 0; j <= nyc; ++j) yc[j] = p->ye[0] + (double)j * cf * p->cell_b;
    for (int l = 0; l <= nzc; ++l) zc[l] = p->ze[0] + (double)l * cf * p->cell_c;
    const grav_mesh cm{nxc, nyc, nzc, xc.data(), yc.data(), zc.data()};
    const grav_survey sv{N, p->sx, p->sy, p->sz};
    grav_options oc;
    grav_options_default(&oc);
    oc.precision = GRAV_MIXED;
    oc.near_cells = 3.0;
    oc.z0 = p->opt.z0;
    oc.timeout_s = p->opt.timeout_s;
    grav_plan *cp = nullptr;
    int rc = plan_create(ctx, &cm, &sv, oc, &cp, s);
    if (rc) return rc;
    const int64_t Mc = (int64_t)nxc * nyc * nzc;
    // persistent block
    st->bytes = nys_bytes(N, ell);
    // temporary block: Omega (N x ell), q (Mc), M and Y^T Y (ell x ell each), dot partials, scalar
    const size_t tmp_bytes = 8ull * ((size_t)N * ell + Mc + 2ull * ell * ell + kDotBlocks + 8) + 5 * 256;
    if (ctx->hbm_used.load() + st->bytes + tmp_bytes > ctx->hbm_budget) {
        plan_destroy(cp, s);
        return set_error(ctx, GRAV_ENOMEM, "Nystrom preconditioner (rank %d) exceeds the HBM budget", ell);
    }
    char *tmp = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&st->mem, st->bytes, ctx->pool, s);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&tmp, tmp_bytes, ctx->pool, s);
    if (e != cudaSuccess) {
        if (st->mem) cudaFreeAsync(st->mem, s);
        st->mem = nullptr;
        plan_destroy(cp, s);
        return cuda_error(ctx, e, "Nystrom allocation");
    }
    ctx->hbm_used += st->bytes + tmp_bytes;
    Arena pa;
    pa.base = st->mem; pa.size = st->bytes;
    st->Y = (double *)pa.take(8ull * N * ell);
    st->L = (double *)pa.take(8ull * ell * ell);
    st->t = (double *)pa.take(8ull * ell);
    Arena ta;
    ta.base = tmp; ta.size = tmp_bytes;
    double *Om = (double *)ta.take(8ull * N * ell);
    double *qc = (double *)ta.take(8ull * Mc);
    double *Mm = (double *)ta.take(8ull * ell * ell);
    double *YY = (double *)ta.take(8ull * ell * ell);
    double *dp = (double *)ta.take(8ull * kDotBlocks);
    double *sc = (double *)ta.take(64);
    cublasHandle_t h = nullptr;
    std::vector<double> hM((size_t)ell * ell), hYY((size_t)ell * ell);
    double *hs = nullptr;
    cudaEvent_t ev = nullptr;
    do {
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) {
            rc = set_error(ctx, GRAV_EDEVICE, "cublasCreate failed");
            break;
        }
        st->blas = h;
        cublasSetStream(h, s);
        // Omega ~ N(0, 1/N); Y = K_c Omega column by column (depth-weighted adjoint, then forward)
        k_randn<<<grid_n(N * ell), 256, 0, s>>>(Om, N * ell, seed, 1.0 / std::sqrt((double)N));
        note_launches(1);
        for (int j = 0; j < ell && !rc; ++j) {
            rc = plan_adjoint_ex(cp, Om + (size_t)j * N, qc, 1, nullptr, s);
            if (!rc) rc = plan_forward_ex(cp, qc, st->Y + (size_t)j * N, nullptr, 0.0, s);
        }
        if (rc) break;
        const double inv_c3 = 1.0 / ((double)cf * cf * cf);
        k_axpby_n<<<grid_n(N * ell), 256, 0, s>>>(inv_c3, st->Y, 0.0, Om, N * ell);
        launch_dot(st->Y, st->Y, N * ell, dp, sc, s);
        note_launches(1);
        cudaMallocHost((void **)&hs, 64);
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaMemcpyAsync(hs, sc, 8, cudaMemcpyDeviceToHost, s);
        cudaEventRecord(ev, s);
        if ((rc = host_wait(ctx, ev, p->opt.timeout_s, "Nystrom sketch"))) break;
        st->nu = std::sqrt((double)N) * 2.220446049250313e-16 * std::sqrt(std::max(hs[0], 0.0));
        st->mu = lam - st->nu;
        if (!(st->mu > 0.0) || !std::isfinite(st->mu)) {
            rc = set_error(ctx, GRAV_EDEVICE, "Nystrom shift %g not below lambda %g", st->nu, lam);
            break;
        }
        k_axpby_n<<<grid_n(N * ell), 256, 0, s>>>(1.0, st->Y, st->nu, Om, N * ell);   // Y_nu
        note_launches(1);
        const double one = 1.0, zero = 0.0;
        // M = Omega^T Y_nu (full), Y_nu^T Y_nu (lower triangle only: symmetric rank-k update)
        if (cublasDgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, ell, ell, (int)N, &one, Om, (int)N, st->Y, (int)N, &zero, Mm,
                        ell) != CUBLAS_STATUS_SUCCESS ||
            cublasDsyrk(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, ell, (int)N, &one, st->Y, (int)N, &zero, YY, ell) !=
                CUBLAS_STATUS_SUCCESS) {
            rc = set_error(ctx, GRAV_EDEVICE, "cuBLAS GEMM failed in the Nystrom set-up");
            break;
        }
        cudaMemcpyAsync(hM.data(), Mm, 8ull * ell * ell, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hYY.data(), YY, 8ull * ell * ell, cudaMemcpyDeviceToHost, s);
        cudaEventRecord(ev, s);
        if ((rc = host_wait(ctx, ev, p->opt.timeout_s, "Nystrom Gram matrices"))) break;
        // T = mu sym(M) + Y^T Y (column-major results; the rank-k update filled
        // the lower triangle, (i, j) with i >= j at i + ell j)
        std::vector<double> T((size_t)ell * ell);
        for (int i = 0; i < ell; ++i)
            for (int j = 0; j < ell; ++j) {
                const size_t ij = (size_t)i + (size_t)ell * j, ji = (size_t)j + (size_t)ell * i;
                T[(size_t)i * ell + j] = st->mu * 0.5 * (hM[ij] + hM[ji]) + (i >= j ? hYY[ij] : hYY[ji]);
            }
        if (!cholesky_rowmajor(T, ell)) {
            rc = set_error(ctx, GRAV_EDEVICE, "Nystrom matrix T is not positive definite (rank %d)", ell);
            break;
        }
        // column-major lower factor for cuBLAS: Lc(i, j) = L[i][j] for i >= j
        std::vector<double> Lc((size_t)ell * ell, 0.0);
        for (int j = 0; j < ell; ++j)
            for (int i = j; i < ell; ++i) Lc[(size_t)i + (size_t)ell * j] = T[(size_t)i * ell + j];
        cudaMemcpyAsync(st->L, Lc.data(), 8ull * ell * ell, cudaMemcpyHostToDevice, s);
        cudaEventRecord(ev, s);
        rc = host_wait(ctx, ev, p->opt.timeout_s, "Nystrom factor upload");
    } while (false);
    if (ev) cudaEventDestroy(ev);
    if (hs) cudaFreeHost(hs);
    cudaFreeAsync(tmp, s);
    ctx->hbm_used -= tmp_bytes;
    plan_destroy(cp, s);
    if (rc) nys_free(p, st, s);
    return rc;
}

void nys_apply(const NysState &st, const double *r, double *z, cudaStream_t s) {
    cublasHandle_t h = (cublasHandle_t)st.blas;
    cublasSetStream(h, s);
    const double one = 1.0, zero = 0.0, mone = -1.0, inv_mu = 1.0 / st.mu;
    const int n = (int)st.N, ell = st.ell;
    cublasDgemv(h, CUBLAS_OP_T, n, ell, &one, st.Y, n, r, 1, &zero, st.t, 1);   // t = Y^T r
    cublasDtrsv(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, ell, st.L, ell, st.t, 1);
    cublasDtrsv(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, ell, st.L, ell, st.t, 1);
    cudaMemcpyAsync(z, r, 8ull * st.N, cudaMemcpyDeviceToDevice, s);
    cublasDgemv(h, CUBLAS_OP_N, n, ell, &mone, st.Y, n, st.t, 1, &one, z, 1);    // z = r - Y t
    cublasDscal(h, n, &inv_mu, z, 1);
}

void nys_free(grav_plan *p, NysState *st, cudaStream_t s) {
    if (st->blas) cublasDestroy((cublasHandle_t)st->blas);
    if (st->mem) {
        cudaFreeAsync(st->mem, s);
        p->ctx->hbm_used -= st->bytes;
    }
    *st = NysState{};
}

}  // namespace grav
