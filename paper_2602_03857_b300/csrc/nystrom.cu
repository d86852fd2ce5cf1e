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
//   depend on a change of basis of Omega's range).
// * With K_c = B B^T and Z = B^T Omega, the Nystrom approximation
//   K Omega (Omega^T K Omega)^-1 Omega^T K is Y M^-1 Y^T with Y = B Z and
//   M = Z^T Z.  M is formed as a Gram matrix (positive semidefinite whatever
//   the rounding of Z), and K_hat = Y (M + nu I)^-1 Y^T is positive
//   semidefinite for any Y; the shift nu (1e-3 lambda, raised if the
//   factorisation needs it) only shrinks K_hat in directions whose Rayleigh
//   quotient is far below lambda, where P is lambda I either way.  (The
//   published method shifts Y by nu Omega instead; with FP32 products the
//   Gram form is what keeps T positive definite when ell is a large share
//   of N.)
// * P^-1 by the Woodbury identity applied to K_hat:
//     (lambda I + Y M_nu^-1 Y^T)^-1 r = (r - Y T^-1 Y^T r) / lambda,
//     T = lambda M_nu + Y^T Y,
//   with one ell x ell Cholesky factor T = L L^T and its inverse L^-1 (on
//   the device, FP64, blocked, chol_kernels.cu; ell^3 / 3 FMAs; ell <= 8192).  Applying it costs two GEMVs
//   with the N x ell matrix Y and two triangular products with L^-1
//   (T^-1 = L^-T L^-1).  Y holds FP32 values (the sketch products are FP32),
//   so Y is kept in FP32 and the GEMVs take exact FP32 products of Y with
//   the FP32-pair split of the FP64 vector, summed in double-float
//   arithmetic: half the bytes of an FP64 Y and no FP64-pipe work.  The
//   application is the symmetric W W^T form, W = Y L^-T, on the stored numbers.
// * The ell sketch products Y = K_c Omega share every pair term: the coarse
//   operator is formed explicitly, one block of cells at a time, as
//   B = G_c W_c^-1 / cf^(3/2) in FP32 (K_c = B B^T; far term plus the coarse
//   plan's near-field table, the entries the coarse mixed operator applies),
//   and Y = sum_b B_b (B_b^T Omega) by two FP32 GEMMs per block.  One pair
//   evaluation then serves all ell columns instead of one, and the products
//   run at the FP32 GEMM rate.  The Gram matrices M = Z^T Z and Y^T Y take
//   exact FP32 products summed in double-float arithmetic on the FP32 pipe
//   (FP64-class sums at the FP32 rate; this GPU's FP64 pipe runs at 1/64 of it).
//
// All dense products are this library's own kernels (dense_kernels.cu).
// Vectors of N stations are stored with a leading dimension ldy = N rounded
// up to a multiple of 4 (16-byte columns); the padding rows hold zeros.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "cg.h"
#include "device_common.cuh"
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

// Omega: out[j + ldo s] = scale * N(0, 1) (rounded to FP32) for s < n, j < k,
// from the Box-Muller transform of two uniforms drawn from counters 2i and
// 2i+1, i = s + n j, of the stream `seed` (deterministic); entries with
// s >= n (up to ld_rows) or j >= k (up to ldo) are 0.  Station-major, so
// that the sketch GEMM reads Omega with its reduction index (the station) slow.
__global__ void k_randn32_t(float *__restrict__ out, int64_t n, int64_t ld_rows, int k, int64_t ldo, uint64_t seed,
                            double scale) {
    const double two_pi = 6.283185307179586476925286766559;
    const int64_t total = ld_rows * ldo;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = q % ldo, s = q / ldo;
        if (s >= n || j >= k) {
            out[q] = 0.0f;
            continue;
        }
        const uint64_t i = (uint64_t)(s + n * j);
        const uint64_t a = splitmix64(seed ^ (2ull * i));
        const uint64_t b = splitmix64(seed ^ (2ull * i + 1ull));
        const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
        const double u2 = (double)(b >> 11) * 0x1.0p-53;           // [0, 1)
        out[q] = (float)(scale * sqrt(-2.0 * log(u1)) * cos(two_pi * u2));
    }
}

inline unsigned grid_n(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 148LL * 32)); }

// y[s + ldy j] = x[s + n j] rounded to FP32 (s < n; padding rows 0), j < k
__global__ void k_narrow(const double *__restrict__ x, int64_t n, int k, float *__restrict__ y, int64_t ldy) {
    const int64_t total = ldy * k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = q % ldy, j = q / ldy;
        y[q] = s < n ? (float)x[s + n * j] : 0.0f;
    }
}

// y[s + n j] = x[s + ldx j] (s < n, j < k)
__global__ void k_widen(const float *__restrict__ x, int64_t ldx, int64_t n, int k, double *__restrict__ y) {
    const int64_t total = n * k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
        y[q] = (double)x[q % n + ldx * (q / n)];
}

// Explicit block of the scaled coarse operator B = G_c W_c^-1 / cf^(3/2)
// (K_c = B B^T), cells c0 <= c < c0 + cb in natural order, station-fastest
// B[(c - c0) ldb + s] (FP32) and, when Bt is given, also cell-fastest
// Bt[(c - c0) + ldt s] (each thread's 16 consecutive cells as four float4).  The far part is the mixed operator's own FP32
// point-mass (+ quadrupole) term of the pair; fac[l] = gamma V (zc_l + z0) / cf^1.5.
constexpr int kNysCells = 16;   // cells per thread

template <bool QUAD>
__global__ void __launch_bounds__(256) k_nys_far(MixedGeo g, const float4 *__restrict__ st32,
                                                 const float2 *__restrict__ stz, int64_t N, int64_t ldb, int64_t c0,
                                                 int cb, const float *__restrict__ fac, float *__restrict__ B,
                                                 float *__restrict__ Bt, int64_t ldt) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const float4 S = st32[s];
    const float zs = stz[s].x;
    const int k0 = blockIdx.y * kNysCells, k1 = min(cb, k0 + kNysCells);
    // (i, j, l) of cell c0 + k0, then stepped along x (meshes hold at most 2^30 cells)
    const int c = (int)(c0 + k0);
    int l = c / g.ncol, i = (c - l * g.ncol) % g.nx, j = (c - l * g.ncol) / g.nx;
    float vals[kNysCells];
#pragma unroll
    for (int u = 0; u < kNysCells; ++u) vals[u] = 0.0f;
    for (int k = k0; k < k1; ++k) {
        const float2 X = make_float2(g.cx[2 * i], g.cx[2 * i + 1]);
        const float2 Y = make_float2(g.cy[2 * j], g.cy[2 * j + 1]);
        const float dx = (X.x - S.x) + (X.y - S.y);
        const float dy = (Y.x - S.z) + (Y.y - S.w);
        const float h2 = fmaf(dx, dx, dy * dy);
        const float ph = QUAD ? far_ph(X, Y, S.x, S.y, S.z, S.w, g.qa, g.qb) : 0.0f;
        const float dz = g.czc[l] - zs;
        const float R2 = fmaf(dz, dz, h2);
        const float v = far_k<QUAD>(dz, R2, g.qg, ph) * fac[l];
        B[(int64_t)k * ldb + s] = v;
        vals[k - k0] = v;
        if (++i == g.nx) {
            i = 0;
            if (++j == g.ny) {
                j = 0;
                ++l;
            }
        }
    }
    if (Bt) {   // cells k0 .. k0+15 of row s (ldt and k0 multiples of 4: 16-byte aligned)
        float4 *dst = reinterpret_cast<float4 *>(Bt + (int64_t)s * ldt + k0);
        const int nq = (k1 - k0 + 3) / 4;
#pragma unroll
        for (int u = 0; u < kNysCells / 4; ++u)
            if (u < nq) dst[u] = make_float4(vals[4 * u], vals[4 * u + 1], vals[4 * u + 2], vals[4 * u + 3]);
    }
}

// Adds the near-field correction table of the coarse plan (exact prism minus
// the far term, per unit gamma V) to the block; one warp per station, each
// (station, cell) pair is touched by one lane only.
__global__ void __launch_bounds__(256) k_nys_near(int nx, int ny, int nz, NearGeo ng, int64_t N, int64_t ldb,
                                                  const float *__restrict__ dG, const int *__restrict__ st_i0,
                                                  const int *__restrict__ st_j0, int64_t c0, int cb,
                                                  const float *__restrict__ fac, float *__restrict__ B,
                                                  float *__restrict__ Bt, int64_t ldt) {
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= N) return;
    const int i0 = st_i0[s], j0 = st_j0[s];
    for (int t = lane; t < ng.slots; t += 32) {
        const int i = i0 + t % ng.bx, j = j0 + (t / ng.bx) % ng.by, l = t / (ng.bx * ng.by);
        if (i < 0 || i >= nx || j < 0 || j >= ny || l >= nz) continue;
        const int64_t k = (int64_t)i + (int64_t)nx * (j + (int64_t)ny * l) - c0;
        if (k < 0 || k >= cb) continue;
        const float d = dG[s * ng.ld + t];
        if (d != 0.0f) {
            const float v = d * fac[l];
            B[k * ldb + s] += v;
            if (Bt) Bt[s * ldt + k] += v;
        }
    }
}

inline int64_t pad4(int64_t v) { return (v + 3) / 4 * 4; }

}  // namespace

// Automatic sizes (0).  The sketch costs 4 N M_c ell FP32 GEMM flops plus a
// double-float Gram of ell^2 (N + M_c) products and an ell^3 / 3 FP64 factor; a CG
// iteration costs two products with the fine operator, ~0.28 s (mixed) or
// ~0.9 s (FP64) at the sizes below, so FP64 solves sketch the uncoarsened
// operator.  With the Gram matrices on the FP32 pipe the mixed rank rose from
// N / 60 (max 3000) to N / 45 (max 4000): at 210 x 210 x 75 x 178,797, ranks
// 2980 / 3500 / 4000 / 4500 took 103 / 90 / 79 / 79 iterations and 37.4 /
// 35.5 / 33.8 / 36.1 s (set-up 9.7 s at 4000).
//   mixed: rank N / 45 in [100, 4000], coarsening min(3, smallest cell count / 8);
//   FP64:  rank min(3000, N / 2), coarsening 1.
// Measured (inversion to 1e-6; without a preconditioner in brackets):
//   210 x 210 x 75 cells x 178,797 stations, mixed, rank 2980, coarsening 2 / 3 / 4:
//   96 / 103 / 122 iterations, 49.2 / 37.9 / 40.4 s [539, 153 s];
//   80 x 80 x 40 x 6,561, FP64, rank 3000, coarsening 1 / 2: 13 / 26 iterations,
//   16.1 / 23.6 s [128, 99 s]; 150 x 150 x 60 x 22,801, FP64, coarsening 1: 38
//   iterations, 543 s.
void nys_sizes(const grav_plan *p, int *ell, int *cf) {
    const bool f64 = p->opt.precision == GRAV_FP64;
    const int64_t N = p->N;
    const int mmin = std::min(p->nx, std::min(p->ny, p->nz));
    if (*ell <= 0)
        *ell = f64 ? (int)std::min<int64_t>(3000, std::max<int64_t>(1, N / 2))
                   : (int)std::min<int64_t>(4000, std::max<int64_t>(100, (N + 22) / 45));
    if (*cf <= 0) *cf = f64 ? 1 : std::max(1, std::min(3, mmin / 8));
    *ell = (int)std::min<int64_t>(*ell, N);
}

size_t nys_bytes(int64_t N, int ell) {
    // persistent part: Y (FP32, ldy x ell), L^-1 (ell x ell), t, u, v (ell doubles),
    // vh, vl (ell floats), rh, rl (ldy floats), the row-chunk partials of Y^T r
    const size_t ldy = (size_t)pad4(N);
    return 4ull * ldy * ell + 8ull * ell * ell + 24ull * ell + 8ull * ell + 8ull * ldy +
           8ull * ell * (size_t)nys_tpart_chunks(N) + 10 * 256;
}

// Explicit-block width: cells per block of the coarse operator (multiple of 4).
static int64_t block_cells(int64_t Mc, int64_t ldy, int k, size_t left) {
    int64_t cb = std::min<int64_t>({Mc, (1ll << 30) / ldy, (1ll << 27) / k, 65535ll * kNysCells,
                                    (int64_t)(left / (4ull * ldy + 4ull * k + 64))});
    return cb;
}

size_t nys_peak_bytes(const grav_plan *p) {
    int ell = p->opt.nys_rank, cf = p->opt.nys_coarsen;
    nys_sizes(p, &ell, &cf);
    if (ell < 1 || cf < 1) return 0;
    const int64_t ldy = pad4(p->N);
    const int64_t Mc = (int64_t)((p->nx + cf - 1) / cf) * ((p->ny + cf - 1) / cf) * ((p->nz + cf - 1) / cf);
    const int64_t ellp = pad4(ell);
    const int64_t cb = pad4(std::min<int64_t>({Mc, (1ll << 30) / ldy, (1ll << 27) / ellp, 65535ll * kNysCells}));
    // persistent + Omega (FP32) + the two Gram matrices + one explicit block in two layouts and Z_b
    return nys_bytes(p->N, ell) + 4ull * ldy * ellp + 16ull * ell * ell + 8ull * cb * ldy + 4ull * cb * ellp +
           (1u << 20);
}

namespace {

// The plan of p's mesh coarsened cf x cf x cf (cells cf a x cf b x cf c of
// the same origin; it may reach past the fine mesh by less than one coarse
// cell on each axis), mixed precision with a near window of 3 cells, same
// stations and z0.
int coarse_plan(grav_plan *p, int cf, grav_plan **cp, cudaStream_t s) {
    const int nxc = (p->nx + cf - 1) / cf, nyc = (p->ny + cf - 1) / cf, nzc = (p->nz + cf - 1) / cf;
    std::vector<double> xc(nxc + 1), yc(nyc + 1), zc(nzc + 1);
    for (int i = 0; i <= nxc; ++i) xc[i] = p->xe[0] + (double)i * cf * p->cell_a;
    for (int j = 0; j <= nyc; ++j) yc[j] = p->ye[0] + (double)j * cf * p->cell_b;
    for (int l = 0; l <= nzc; ++l) zc[l] = p->ze[0] + (double)l * cf * p->cell_c;
    const grav_mesh cm{nxc, nyc, nzc, xc.data(), yc.data(), zc.data()};
    const grav_survey sv{p->N, p->sx, p->sy, p->sz};
    grav_options oc;
    grav_options_default(&oc);
    oc.precision = GRAV_MIXED;
    oc.near_cells = 3.0;
    oc.z0 = p->opt.z0;
    oc.timeout_s = p->opt.timeout_s;
    return plan_create(p->ctx, &cm, &sv, oc, cp, s);
}

// Y32 = K_c X32 = B (B^T X32) (ldy x k, FP32, column-major: Y32[s + ldy j])
// with B = G_c W_c^-1 / cf^(3/2) formed explicitly one block of cells at a
// time (FP32).  X32 is station-major (X32[j + ldx s], x_nmajor: the sketch's
// Omega) or station-fastest (X32[s + ldx j]); rows s >= N must be 0.  With a
// station-major X32 the block is formed in both layouts, so that neither GEMM
// transposes a tile: Z_b = B_b^T X32 reads the cell-fastest copy and X32 with
// the station index slow and writes Z_b column-fastest (Z_b[j + kp c]); Y32
// += B_b Z_b reads the station-fastest copy and Z_b with the cell index slow.
// When M is given, M (k x k, FP64, lower triangle) = Z^T Z (exact FP32
// products, double-float sums).  Scratch comes from the context's pool and
// the context's HBM budget.
int coarse_products(grav_plan *cp, int cf, double z0, const float *X32, int64_t ldx, bool x_nmajor, int k,
                    float *Y32, double *M, cudaStream_t s) {
    grav_ctx *ctx = cp->ctx;
    const int64_t N = cp->N, Mc = cp->M, ldy = pad4(N), kp = pad4(k);
    const int nzc = cp->nz;
    const int layouts = x_nmajor ? 2 : 1;
    const size_t used = ctx->hbm_used.load() + 4ull * nzc + 5 * 256;
    const size_t left = ctx->hbm_budget > used ? ctx->hbm_budget - used : 0;
    int64_t cb = block_cells(Mc, ldy, (int)kp, left / layouts);
    if (cb < std::min<int64_t>(Mc, 64))
        return set_error(ctx, GRAV_ENOMEM, "explicit coarse operator block (%d columns) exceeds the HBM budget", k);
    const int64_t nblk = (Mc + cb - 1) / cb;
    cb = (Mc + nblk - 1) / nblk;   // equal blocks
    const int64_t cbp = pad4(cb);   // GEMM inner dimension, zero columns at the end
    const size_t bytes = 4ull * nzc + 4ull * layouts * cbp * ldy + 4ull * cbp * kp + 5 * 256;
    char *mem = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&mem, bytes, ctx->pool, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "explicit coarse operator block");
    ctx->hbm_used += bytes;
    Arena ta;
    ta.base = mem; ta.size = bytes;
    float *fac = (float *)ta.take(4ull * nzc);
    float *Bb = (float *)ta.take(4ull * ldy * cbp);                      // B_b[c ldy + s]
    float *Bt = x_nmajor ? (float *)ta.take(4ull * ldy * cbp) : nullptr;  // B_b[s cbp + c]
    float *Zb = (float *)ta.take(4ull * cbp * kp);   // x_nmajor: Z_b[c kp + j]; else Z_b[j cbp + c]
    if (ta.overflow) {
        cudaFreeAsync(mem, s);
        ctx->hbm_used -= bytes;
        return set_error(ctx, GRAV_EDEVICE, "explicit coarse operator layout");
    }
    // fac[l] = gamma V_c (zc_l + z0) / cf^(3/2): K ~ G_c W_c^-2 G_c^T / cf^3 = B B^T
    std::vector<float> hfac(nzc);
    const double vol_mgal = kGammaMgal * cp->cell_a * cp->cell_b * cp->cell_c;
    for (int l = 0; l < nzc; ++l)
        hfac[l] = (float)(vol_mgal * (0.5 * (cp->ze[l] + cp->ze[l + 1]) - cp->ze[0] + z0) / std::pow((double)cf, 1.5));
    cudaMemcpyAsync(fac, hfac.data(), 4ull * nzc, cudaMemcpyHostToDevice, s);
    int rc = GRAV_OK;
    for (int64_t b = 0; b < nblk && !rc; ++b) {
        const int64_t c0 = b * cb;
        const int nb = (int)std::min<int64_t>(cb, Mc - c0);
        // zero blocks: padding rows (stations >= N) and columns (cells >= nb) stay 0
        cudaMemsetAsync(Bb, 0, 4ull * ldy * cbp, s);
        if (Bt) cudaMemsetAsync(Bt, 0, 4ull * ldy * cbp, s);
        dim3 gf((unsigned)((N + 255) / 256), (unsigned)((nb + kNysCells - 1) / kNysCells));
        if (cp->cubic)
            k_nys_far<false><<<gf, 256, 0, s>>>(cp->mg, cp->st32, cp->stz, N, ldy, c0, nb, fac, Bb, Bt, cbp);
        else
            k_nys_far<true><<<gf, 256, 0, s>>>(cp->mg, cp->st32, cp->stz, N, ldy, c0, nb, fac, Bb, Bt, cbp);
        k_nys_near<<<(unsigned)((N * 32 + 255) / 256), 256, 0, s>>>(cp->nx, cp->ny, nzc, cp->ng, N, ldy, cp->dG,
                                                                  cp->st_i0, cp->st_j0, c0, nb, fac, Bb, Bt, cbp);
        note_launches(2);
        bool ok;
        if (x_nmajor) {
            // Z_b = B_b^T X32 (cbp x k, column-fastest), Y32 (+)= B_b Z_b, M (+)= Z_b^T Z_b
            ok = launch_sgemm(false, (int)cbp, k, (int)ldy, Bt, cbp, X32, ldx, Zb, kp, false, s, true, true) == 0;
            ok = ok && launch_sgemm(false, (int)ldy, k, (int)cbp, Bb, ldy, Zb, kp, Y32, ldy, b > 0, s, true, false) == 0;
            if (M) ok = ok && launch_gram_df(k, (int)cbp, Zb, kp, M, b > 0, s, true) == 0;
        } else {
            ok = launch_sgemm(true, (int)cbp, k, (int)ldy, Bb, ldy, X32, ldx, Zb, cbp, false, s) == 0;
            ok = ok && launch_sgemm(false, (int)ldy, k, (int)cbp, Bb, ldy, Zb, cbp, Y32, ldy, b > 0, s) == 0;
            if (M) ok = ok && launch_gram_df(k, (int)cbp, Zb, cbp, M, b > 0, s) == 0;
        }
        if (!ok) rc = set_error(ctx, GRAV_EINVAL, "explicit coarse products: unsupported layout");
    }
    cudaFreeAsync(mem, s);
    ctx->hbm_used -= bytes;
    return rc;
}

}  // namespace

int nys_coarse_apply(grav_plan *p, int cf, const double *X, int k, double *Y, cudaStream_t s) {
    grav_ctx *ctx = p->ctx;
    if (!p->uniform) return set_error(ctx, GRAV_EINVAL, "the coarse operator needs a mesh of uniform cells");
    if (cf < 1 || cf > 8 || k < 1) return set_error(ctx, GRAV_EINVAL, "coarsening must lie in [1, 8] and k >= 1");
    const int64_t N = p->N, ldy = pad4(N);
    grav_plan *cp = nullptr;
    int rc = coarse_plan(p, cf, &cp, s);
    if (rc) return rc;
    const size_t bytes = 8ull * ldy * k + 2 * 256;
    char *mem = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&mem, bytes, ctx->pool, s);
    if (e != cudaSuccess) {
        plan_destroy(cp, s);
        return cuda_error(ctx, e, "coarse operator vectors");
    }
    ctx->hbm_used += bytes;
    Arena ta;
    ta.base = mem; ta.size = bytes;
    float *X32 = (float *)ta.take(4ull * ldy * k);
    float *Y32 = (float *)ta.take(4ull * ldy * k);
    k_narrow<<<grid_n(ldy * k), 256, 0, s>>>(X, N, k, X32, ldy);
    note_launches(1);
    rc = coarse_products(cp, cf, p->opt.z0, X32, ldy, false, k, Y32, nullptr, s);
    if (!rc) {
        k_widen<<<grid_n(N * k), 256, 0, s>>>(Y32, ldy, N, k, Y);
        note_launches(1);
    }
    cudaFreeAsync(mem, s);
    ctx->hbm_used -= bytes;
    plan_destroy(cp, s);
    return rc;
}

int nys_build(grav_plan *p, double lam, int ell, int cf, uint64_t seed, NysState *st, cudaStream_t s) {
    grav_ctx *ctx = p->ctx;
    NvtxRange nv("grav::nystrom_build");
    const int64_t N = p->N, ldy = pad4(N);
    if (!p->uniform) return set_error(ctx, GRAV_EINVAL, "precond = 2 (Nystrom) needs a mesh of uniform cells");
    nys_sizes(p, &ell, &cf);
    if (ell < 1 || cf < 1) return set_error(ctx, GRAV_EINVAL, "Nystrom rank and coarsening must be >= 1");
    *st = NysState{};
    st->ell = ell;
    st->N = N;
    st->ldy = ldy;
    grav_plan *cp = nullptr;
    int rc = coarse_plan(p, cf, &cp, s);
    if (rc) return rc;
    // persistent block; temporary block: Omega (FP32, ldy x ell), M and Y^T Y
    // (ell x ell FP64); the explicit blocks take what the budget leaves
    st->bytes = nys_bytes(N, ell);
    const int64_t ellp = pad4(ell);
    const size_t tmp_bytes = 4ull * ldy * ellp + 24ull * ell * ell + 5 * 256;
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
    st->Y = (float *)pa.take(4ull * ldy * ell);
    st->Linv = (double *)pa.take(8ull * ell * ell);
    st->t = (double *)pa.take(8ull * ell);
    st->u = (double *)pa.take(8ull * ell);
    st->v = (double *)pa.take(8ull * ell);
    st->vh = (float *)pa.take(4ull * ell);
    st->vl = (float *)pa.take(4ull * ell);
    st->rh = (float *)pa.take(4ull * ldy);
    st->rl = (float *)pa.take(4ull * ldy);
    st->tp = (double *)pa.take(8ull * ell * nys_tpart_chunks(N));
    Arena ta;
    ta.base = tmp; ta.size = tmp_bytes;
    float *Om32 = (float *)ta.take(4ull * ldy * ellp);   // station-major: Om32[j + ellp s]
    double *Mm = (double *)ta.take(8ull * ell * ell);
    double *Gy = (double *)ta.take(8ull * ell * ell);
    double *Tm = (double *)ta.take(8ull * ell * ell);   // T, factored in place into L
    int *d_fail = (int *)ta.take(256);
    int *h_fail = nullptr;
    cudaMallocHost((void **)&h_fail, sizeof(int));
    cudaEvent_t ev = nullptr;
    do {
        if (pa.overflow || ta.overflow) {
            rc = set_error(ctx, GRAV_EDEVICE, "Nystrom scratch layout");
            break;
        }
        k_randn32_t<<<grid_n(ldy * ellp), 256, 0, s>>>(Om32, N, ldy, ell, ellp, seed, 1.0 / std::sqrt((double)N));
        note_launches(1);
        // Y = K_c Omega and M = Z^T Z, Z = B^T Omega
        if ((rc = coarse_products(cp, cf, p->opt.z0, Om32, ellp, true, ell, st->Y, Mm, s))) break;
        if (launch_gram_df(ell, (int)ldy, st->Y, ldy, Gy, false, s) != 0) {
            rc = set_error(ctx, GRAV_EINVAL, "Nystrom Gram matrix: unsupported layout");
            break;
        }
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        // T = mu (M + nu I) + Y^T Y (column-major lower, as the Gram matrices),
        // factored on the device.  nu starts at 1e-3 lambda and grows tenfold
        // (to at most 10 lambda) while the factorisation meets a pivot that is
        // not positive; the host reads one flag per attempt.
        st->mu = lam;
        bool factored = false;
        for (double nu = 1e-3 * lam; !factored && nu <= 10.0 * lam * 1.0000001; nu *= 10.0) {
            launch_form_T(ell, lam, nu, Mm, Gy, Tm, s);
            cudaMemsetAsync(d_fail, 0, sizeof(int), s);
            launch_potrf_lower(Tm, ell, d_fail, s);
            cudaMemcpyAsync(h_fail, d_fail, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaEventRecord(ev, s);
            if ((rc = host_wait(ctx, ev, p->opt.timeout_s, "Nystrom factorisation"))) break;
            st->nu = nu;
            factored = (*h_fail == 0);
        }
        if (rc) break;
        if (!factored) {
            rc = set_error(ctx, GRAV_EDEVICE, "Nystrom matrix T is not positive definite (rank %d)", ell);
            break;
        }
        launch_trinv_lower(Tm, st->Linv, ell, s);
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) rc = cuda_error(ctx, le, "Nystrom factorisation launch");
    } while (false);
    if (ev) cudaEventDestroy(ev);
    if (h_fail) cudaFreeHost(h_fail);
    cudaFreeAsync(tmp, s);
    ctx->hbm_used -= tmp_bytes;
    plan_destroy(cp, s);
    if (rc) nys_free(p, st, s);
    return rc;
}

void nys_apply(const NysState &st, const double *r, double *z, cudaStream_t s) {
    launch_nys_apply(st.Y, st.ldy, st.N, st.ell, st.Linv, st.mu, r, z, st.rh, st.rl, st.tp, st.t, st.u, st.v, st.vh, st.vl,
                     s);
}

void nys_free(grav_plan *p, NysState *st, cudaStream_t s) {
    if (st->mem) {
        cudaFreeAsync(st->mem, s);
        p->ctx->hbm_used -= st->bytes;
    }
    *st = NysState{};
}

}  // namespace grav
