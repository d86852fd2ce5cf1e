// Device factorisation of the randomized Nystrom preconditioner's ell x ell
// matrix T = lambda (M + nu I) + Y^T Y (FP64, column-major lower triangle,
// element (i, j), i >= j, at i + ell j): a blocked right-looking Cholesky
// T = L L^T (blocks of 32: the diagonal block factored by one warp, the
// panel below it by a triangular solve per row, the trailing matrix by a
// SYRK-shaped update on 64 x 64 tiles), then the explicit inverse L^-1 block
// row by block row (Li[I, J] = -L_II^-1 sum_{J <= K < I} L[I, K] Li[K, J]),
// which the preconditioner applies as two triangular matrix-vector products
// per CG iteration.  ell^3 / 3 FMAs in all, on the FP64 pipe; no host work
// and no transfer of the ell x ell matrices.
#include <algorithm>
#include <cmath>

#include "device_common.cuh"
#include "internal.h"

namespace grav {
namespace {

constexpr int kCb = 32;    // block size of the factorisation and the inverse
constexpr int kSyT = 64;   // output tile of the trailing update

// T = lam (M + nu I) + G on the lower triangle, 0 above it
__global__ void k_form_T(int n, double lam, double nu, const double *__restrict__ M, const double *__restrict__ G,
                         double *__restrict__ T) {
    const int64_t total = (int64_t)n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % n), j = (int)(t / n);
        T[t] = (i >= j) ? lam * (M[t] + (i == j ? nu : 0.0)) + G[t] : 0.0;
    }
}

// Cholesky of the diagonal block A[k0 .. k0+nb) x [k0 .. k0+nb) in shared
// memory, one warp, lane = row; a pivot that is not positive (or not finite)
// sets *fail and continues with 1 (the caller retries with a larger shift).
__global__ void k_potrf_diag(double *__restrict__ A, int n, int k0, int *__restrict__ fail) {
    __shared__ double a[kCb][kCb + 1];
    const int nb = min(kCb, n - k0);
    const int lane = threadIdx.x;
    for (int c = 0; c < nb; ++c)
        if (lane < nb) a[lane][c] = (lane >= c) ? A[(int64_t)(k0 + lane) + (int64_t)n * (k0 + c)] : 0.0;
    __syncwarp();
    for (int j = 0; j < nb; ++j) {
        double d = a[j][j];
        if (!(d > 0.0) || !isfinite(d)) {
            if (lane == 0) atomicOr(fail, 1);
            d = 1.0;
        }
        const double ljj = sqrt(d), inv = 1.0 / ljj;
        __syncwarp();
        if (lane == j) a[j][j] = ljj;
        if (lane > j && lane < nb) a[lane][j] *= inv;
        __syncwarp();
        if (lane > j && lane < nb) {
            const double lij = a[lane][j];
            for (int c = j + 1; c <= lane; ++c) a[lane][c] = fma(-lij, a[c][j], a[lane][c]);
        }
        __syncwarp();
    }
    for (int c = 0; c < nb; ++c)
        if (lane < nb && lane >= c) A[(int64_t)(k0 + lane) + (int64_t)n * (k0 + c)] = a[lane][c];
}

// Panel below the diagonal block: row i of L[k0+nb.., k0..k0+nb) solves
// x L_kk^T = A[i, k0..k0+nb) by forward substitution (thread per row).
__global__ void __launch_bounds__(128) k_trsm_panel(double *__restrict__ A, int n, int k0) {
    __shared__ double L[kCb][kCb + 1];
    const int nb = min(kCb, n - k0);
    for (int t = threadIdx.x; t < kCb * kCb; t += blockDim.x) {
        const int r = t % kCb, c = t / kCb;
        L[r][c] = (r < nb && c <= r) ? A[(int64_t)(k0 + r) + (int64_t)n * (k0 + c)] : (r == c ? 1.0 : 0.0);
    }
    __syncthreads();
    const int64_t i = (int64_t)k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[kCb];
#pragma unroll
    for (int j = 0; j < kCb; ++j) {
        double v = (j < nb) ? A[i + (int64_t)n * (k0 + j)] : 0.0;
#pragma unroll
        for (int c = 0; c < j; ++c) v = fma(-x[c], L[j][c], v);
        x[j] = v / L[j][j];
    }
#pragma unroll
    for (int j = 0; j < kCb; ++j)
        if (j < nb) A[i + (int64_t)n * (k0 + j)] = x[j];
}

// Trailing update A[k1.., k1..] -= P P^T on the lower triangle, P =
// A[k1.., k0..k0+nb), k1 = k0 + nb: a CTA per 64 x 64 output tile (tile row
// >= tile column, index t -> (bi, bj) with t = bi (bi + 1) / 2 + bj), 4 x 4
// outputs per thread, consecutive threads on consecutive rows.
__global__ void __launch_bounds__(256) k_syrk_lower(double *__restrict__ A, int n, int k0) {
    __shared__ double Pr[kCb][kSyT + 1], Pc[kCb][kSyT + 1];
    const int nb = min(kCb, n - k0);
    const int k1 = k0 + nb, m = n - k1;
    const int64_t t = blockIdx.x;
    int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)bi * (bi + 1) / 2 > t) --bi;
    while ((int64_t)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
    const int bj = (int)(t - (int64_t)bi * (bi + 1) / 2);
    const int r0 = bi * kSyT, c0 = bj * kSyT;
    for (int q = threadIdx.x; q < kCb * kSyT; q += blockDim.x) {
        const int r = q % kSyT, c = q / kSyT;
        const bool okc = c < nb;
        Pr[c][r] = (okc && r0 + r < m) ? A[(int64_t)(k1 + r0 + r) + (int64_t)n * (k0 + c)] : 0.0;
        Pc[c][r] = (okc && c0 + r < m) ? A[(int64_t)(k1 + c0 + r) + (int64_t)n * (k0 + c)] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int c = 0; c < nb; ++c) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            a[i] = Pr[c][tx + 16 * i];
            b[i] = Pc[c][ty + 16 * i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = c0 + ty + 16 * j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = r0 + tx + 16 * i;
            if (row < m && col < m && row >= col) {
                double *p = A + (int64_t)(k1 + row) + (int64_t)n * (k1 + col);
                *p -= acc[i][j];
            }
        }
    }
}

// Li[I, I] = L_II^-1 for the diagonal block at i0: one warp, lane = column
// of the inverse, forward substitution on the unit vector.
__global__ void k_trinv_diag(const double *__restrict__ L, double *__restrict__ Li, int n, int i0) {
    __shared__ double a[kCb][kCb + 1];
    const int nb = min(kCb, n - i0);
    const int lane = threadIdx.x;
    for (int c = 0; c < kCb; ++c)
        a[lane][c] = (lane < nb && c <= lane) ? L[(int64_t)(i0 + lane) + (int64_t)n * (i0 + c)] : (lane == c ? 1.0 : 0.0);
    __syncwarp();
    double x[kCb];
#pragma unroll
    for (int r = 0; r < kCb; ++r) {
        double v = (r == lane) ? 1.0 : 0.0;
#pragma unroll
        for (int c = 0; c < r; ++c) v = fma(-a[r][c], x[c], v);
        x[r] = v / a[r][r];
    }
    if (lane >= nb) return;
#pragma unroll
    for (int r = 0; r < kCb; ++r)
        if (r < nb) Li[(int64_t)(i0 + r) + (int64_t)n * (i0 + lane)] = (r >= lane) ? x[r] : 0.0;
}

// Li[I, J] = -Li_II sum_{J <= K < I} L[I, K] Li[K, J] for the column blocks
// J < I (J0 = 32 blockIdx.x): 256 threads, thread = (row r, columns cq + 8q).
__global__ void __launch_bounds__(256) k_trinv_row(const double *__restrict__ L, double *__restrict__ Li, int n,
                                                   int i0) {
    __shared__ double Ls[kCb][kCb + 1], Ks[kCb][kCb + 1];
    const int nbI = min(kCb, n - i0);
    const int j0 = blockIdx.x * kCb;
    const int r = threadIdx.x % kCb, cq = threadIdx.x / kCb;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k0 = j0; k0 < i0; k0 += kCb) {
        for (int q = threadIdx.x; q < kCb * kCb; q += blockDim.x) {
            const int rr = q % kCb, cc = q / kCb;
            Ls[rr][cc] = (rr < nbI) ? L[(int64_t)(i0 + rr) + (int64_t)n * (k0 + cc)] : 0.0;
            Ks[rr][cc] = Li[(int64_t)(k0 + rr) + (int64_t)n * (j0 + cc)];
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kCb; ++k) {
            const double l = Ls[r][k];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(l, Ks[k][cq + 8 * q], acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) Ks[r][cq + 8 * q] = acc[q];
    for (int q = threadIdx.x; q < kCb * kCb; q += blockDim.x) {
        const int rr = q % kCb, cc = q / kCb;
        Ls[rr][cc] = (rr < nbI && cc < nbI) ? Li[(int64_t)(i0 + rr) + (int64_t)n * (i0 + cc)] : 0.0;
    }
    __syncthreads();
    double out[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k <= r; ++k) {
        const double l = Ls[r][k];
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = fma(l, Ks[k][cq + 8 * q], out[q]);
    }
    if (r < nbI)
#pragma unroll
        for (int q = 0; q < 4; ++q) Li[(int64_t)(i0 + r) + (int64_t)n * (j0 + cq + 8 * q)] = -out[q];
}

}  // namespace

void launch_form_T(int n, double lam, double nu, const double *M, const double *G, double *T, cudaStream_t s) {
    const int64_t total = (int64_t)n * n;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148LL * 16);
    k_form_T<<<blocks, 256, 0, s>>>(n, lam, nu, M, G, T);
    note_launches(1);
}

void launch_potrf_lower(double *A, int n, int *fail, cudaStream_t s) {
    int launches = 0;
    for (int k0 = 0; k0 < n; k0 += kCb) {
        k_potrf_diag<<<1, 32, 0, s>>>(A, n, k0, fail);
        ++launches;
        const int m = n - k0 - std::min(kCb, n - k0);
        if (m > 0) {
            k_trsm_panel<<<(m + 127) / 128, 128, 0, s>>>(A, n, k0);
            const int64_t nt = (m + kSyT - 1) / kSyT;
            k_syrk_lower<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(A, n, k0);
            launches += 2;
        }
    }
    note_launches(launches);
}

void launch_trinv_lower(const double *L, double *Li, int n, cudaStream_t s) {
    cudaMemsetAsync(Li, 0, 8ull * n * n, s);
    int launches = 0;
    for (int i0 = 0; i0 < n; i0 += kCb) {
        k_trinv_diag<<<1, 32, 0, s>>>(L, Li, n, i0);
        ++launches;
        if (i0 > 0) {
            k_trinv_row<<<i0 / kCb, 256, 0, s>>>(L, Li, n, i0);
            ++launches;
        }
    }
    note_launches(launches);
}

}  // namespace grav
