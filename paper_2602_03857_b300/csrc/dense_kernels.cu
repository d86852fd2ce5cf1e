// Dense kernels of the randomized Nystrom preconditioner (nystrom.cu): the
// sketch products, the two Gram matrices and the application of the
// preconditioner.  Plain CUDA cores, no tensor cores and no library.
//
// * k_sgemm: C (+)= A B in FP32 (FP32 products and sums, as the sketch's
//   explicit coarse operator is FP32).  128 x 128 output tiles, 16-deep k
//   slices staged in shared memory (double-buffered through registers),
//   8 x 8 outputs per thread computed with the packed fma.rn.f32x2
//   instruction (two FMAs per issue slot; the FMA pipe, not the issue rate,
//   is the limit).
// * k_gram_df: G (+)= X^T X, lower triangle, for FP32 X.  Every product of
//   two FP32 numbers is exact as p + e (p = a b rounded, e = fma(a, b, -p));
//   the sums run in double-float arithmetic (a pair hi + lo of FP32 numbers,
//   Knuth's TwoSum for hi, e and the TwoSum error into lo) over runs of 128
//   products, and each run's hi + lo is added into an FP64 sum.  The low
//   word is itself an FP32 sum, so a run of n products carries about n u^2
//   (u = 2^-24) relative error: 128-term runs keep it near 5e-13 (FP64-class),
//   where one run over all 178,797 stations of the paper-scale survey would
//   reach 6e-10.  The products and runs use the FP32 pipe, which this GPU
//   runs at 64 times its FP64 rate; the FP64 adds are one per 128 products.
// * k_gemv_t_df / k_gemv_n_df: t = Y^T r and z = (r - Y v) / mu for an FP32
//   matrix Y and FP64 vectors split into FP32 pairs, with the same exact
//   products and double-float sums; k_trmv_lo / k_trmv_lo_t: lower-triangular
//   FP64 products with the explicit inverse factor.
// Every reduction runs in a fixed order: results are bitwise repeatable.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_common.cuh"
#include "internal.h"

namespace grav {
namespace {

constexpr int kGmBM = 128, kGmBN = 128, kGmBK = 16, kGmThreads = 256;
static_assert(kGmBM == 128 && kGmBN == 128 && kGmBK == 16 && kGmThreads == 256, "tile load mapping");
constexpr int kGmPad = 4;   // row stride 132 floats: 16-byte aligned rows
#ifndef GRAV_GEMM_MINB
#define GRAV_GEMM_MINB 2        // CTAs per SM the GEMM's register budget is sized for
#endif

__device__ __forceinline__ f2_t f2_dup(float a) { return f2_pack(a, a); }

// C (+)= A B, m < M, n < N, k < K:
//   A_KMAJ: A(m, k) = A[k + lda m]; else A(m, k) = A[m + lda k].
//   B_NMAJ: B(k, n) = B[n + ldb k]; else B(k, n) = B[k + ldb n].
//   C_NMAJ: C(m, n) = C[n + ldc m]; else C(m, n) = C[m + ldc n].
// An operand whose k index is the slow one (A m-major, B n-major) moves into
// shared memory as it is; a k-fastest one is transposed on the way (four
// scalar stores per float4).  Requirements (checked by the launcher): lda,
// ldb, ldc, K and M multiples of 4, 16-byte aligned bases (float4 loads and
// stores), and for B_NMAJ / C_NMAJ rows of at least N rounded up to 4 (a
// float4 that starts below N may cover padding columns, whose results are
// not stored, and C_NMAJ writes them).
template <bool A_KMAJ, bool B_NMAJ, bool C_NMAJ>
__global__ void __launch_bounds__(kGmThreads, GRAV_GEMM_MINB) k_sgemm(int M, int N, int K, const float *__restrict__ A, int64_t lda,
                                                         const float *__restrict__ B, int64_t ldb, float *__restrict__ C,
                                                         int64_t ldc, int accumulate) {
    __shared__ __align__(16) float As[2][kGmBK][kGmBM + kGmPad];
    __shared__ __align__(16) float Bs[2][kGmBK][kGmBN + kGmPad];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * kGmBM, n0 = blockIdx.y * kGmBN;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ra[2], rb[2];
    auto load_tile = [&](int k0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int idx = tid + kGmThreads * i;
            if (A_KMAJ) {   // lanes take consecutive rows: the transposed stores below are conflict-free
                const int mm = idx & (kGmBM - 1), kq = idx >> 7;
                const int m = m0 + mm, k = k0 + 4 * kq;
                ra[i] = (m < M && k < K) ? __ldg(reinterpret_cast<const float4 *>(A + (int64_t)m * lda + k)) : zero4;
            } else {
                const int mq = idx & 31, kk = idx >> 5;
                const int m = m0 + 4 * mq, k = k0 + kk;
                ra[i] = (m < M && k < K) ? __ldg(reinterpret_cast<const float4 *>(A + (int64_t)k * lda + m)) : zero4;
            }
            if (B_NMAJ) {
                const int nq = idx & 31, kk = idx >> 5;
                const int n = n0 + 4 * nq, k = k0 + kk;
                rb[i] = (n < N && k < K) ? __ldg(reinterpret_cast<const float4 *>(B + (int64_t)k * ldb + n)) : zero4;
            } else {
                const int nn = idx & (kGmBN - 1), kq = idx >> 7;
                const int n = n0 + nn, k = k0 + 4 * kq;
                rb[i] = (n < N && k < K) ? __ldg(reinterpret_cast<const float4 *>(B + (int64_t)n * ldb + k)) : zero4;
            }
        }
    };
    auto store_tile = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int idx = tid + kGmThreads * i;
            if (A_KMAJ) {
                const int mm = idx & (kGmBM - 1), kq = idx >> 7;
                As[buf][4 * kq + 0][mm] = ra[i].x;
                As[buf][4 * kq + 1][mm] = ra[i].y;
                As[buf][4 * kq + 2][mm] = ra[i].z;
                As[buf][4 * kq + 3][mm] = ra[i].w;
            } else {
                const int mq = idx & 31, kk = idx >> 5;
                *reinterpret_cast<float4 *>(&As[buf][kk][4 * mq]) = ra[i];
            }
            if (B_NMAJ) {
                const int nq = idx & 31, kk = idx >> 5;
                *reinterpret_cast<float4 *>(&Bs[buf][kk][4 * nq]) = rb[i];
            } else {
                const int nn = idx & (kGmBN - 1), kq = idx >> 7;
                Bs[buf][4 * kq + 0][nn] = rb[i].x;
                Bs[buf][4 * kq + 1][nn] = rb[i].y;
                Bs[buf][4 * kq + 2][nn] = rb[i].z;
                Bs[buf][4 * kq + 3][nn] = rb[i].w;
            }
        }
    };
    // acc[i][p]: row r(i) = (i < 4 ? ty*4 + i : 64 + ty*4 + i - 4), columns of pair p:
    // p < 2: tx*4 + 2p, +1;  p >= 2: 64 + tx*4 + 2(p-2), +1
    f2_t acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[i][p] = 0ull;
    const int nk = (K + kGmBK - 1) / kGmBK;
    load_tile(0);
    store_tile(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) load_tile((kt + 1) * kGmBK);
#pragma unroll
        for (int kk = 0; kk < kGmBK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + 4 * tx]);
            const f2_t b[4] = {f2_pack(b0.x, b0.y), f2_pack(b0.z, b0.w), f2_pack(b1.x, b1.y), f2_pack(b1.z, b1.w)};
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const f2_t ai = f2_dup(a[i]);
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[i][p] = f2_fma(ai, b[p], acc[i][p]);
            }
        }
        if (kt + 1 < nk) store_tile(buf ^ 1);
        __syncthreads();
    }
    if (C_NMAJ) {   // rows m, four consecutive columns per float4
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
            if (m >= M) continue;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int n = n0 + 64 * half + 4 * tx;
                if (n >= N) continue;
                float a0, a1, a2, a3;
                f2_unpack(acc[i][2 * half], a0, a1);
                f2_unpack(acc[i][2 * half + 1], a2, a3);
                float4 *dst = reinterpret_cast<float4 *>(C + (int64_t)m * ldc + n);
                float4 out = make_float4(a0, a1, a2, a3);
                if (accumulate) {
                    const float4 o = *dst;
                    out.x += o.x; out.y += o.y; out.z += o.z; out.w += o.w;
                }
                *dst = out;
            }
        }
        return;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n = n0 + (p < 2 ? 4 * tx + 2 * p : 64 + 4 * tx + 2 * (p - 2)) + h;
            if (n >= N) continue;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int m = m0 + 64 * r + 4 * ty;
                if (m >= M) continue;
                float v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float lo, hi;
                    f2_unpack(acc[4 * r + i][p], lo, hi);
                    v[i] = h ? hi : lo;
                }
                float4 *dst = reinterpret_cast<float4 *>(C + (int64_t)n * ldc + m);
                float4 out = make_float4(v[0], v[1], v[2], v[3]);
                if (accumulate) {
                    const float4 o = *dst;
                    out.x += o.x; out.y += o.y; out.z += o.z; out.w += o.w;
                }
                *dst = out;
            }
        }
}

// ---------------------------------------------------------------------------
// Double-float accumulation of exact FP32 products.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

// (hi, lo) += a b, with a b = p + e exact and hi + p = s + t exact (TwoSum).
__device__ __forceinline__ void df_acc_prod(DF &x, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = x.hi + p;
    const float bb = s - x.hi;
    const float t = (x.hi - (s - bb)) + (p - bb);
    x.hi = s;
    x.lo += t + e;
}

constexpr int kGrT = 64, kGrBK = 16, kGrThreads = 256;
constexpr int kGrFoldTiles = 8;   // 16-deep k slices per double-float run (128 products)
constexpr int kDfRun = 128;       // terms per double-float run in the GEMVs

// G[i + n j] (+)= sum_k X(k, i) X(k, j) for i >= j (lower triangle), i, j < n,
// k < K, with X(k, i) = X[k + ldx i] (!KSLOW) or X[i + ldx k] (KSLOW); 64 x 64
// tiles of the lower block triangle, 4 x 4 outputs per thread.  ldx and K
// multiples of 4, X 16-byte aligned; for KSLOW rows of at least n rounded up
// to 4 (padding columns may be read; their products are not stored).
template <bool KSLOW>
__global__ void __launch_bounds__(kGrThreads) k_gram_df(int n, int K, const float *__restrict__ X, int64_t ldx,
                                                        double *__restrict__ G, int accumulate) {
    __shared__ __align__(16) float Xi[2][kGrBK][kGrT + 4];
    __shared__ __align__(16) float Xj[2][kGrBK][kGrT + 4];
    // tile (bi, bj), bi >= bj, from the linear block index
    const int t = blockIdx.x;
    int bi = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while (bi * (bi + 1) / 2 > t) --bi;
    const int bj = t - bi * (bi + 1) / 2;
    const int i0 = bi * kGrT, j0 = bj * kGrT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ri, rj;
    // 64 columns x 16 k = 256 float4 per operand: one per thread
    auto load_tile = [&](int k0) {
        if (KSLOW) {   // 16 rows k of 64 consecutive columns: one float4 per thread, stored as is
            const int cq = tid & 15, kk = tid >> 4;
            const int k = k0 + kk;
            const int ci = i0 + 4 * cq, cj = j0 + 4 * cq;
            ri = (ci < n && k < K) ? __ldg(reinterpret_cast<const float4 *>(X + (int64_t)k * ldx + ci)) : zero4;
            rj = (cj < n && k < K) ? __ldg(reinterpret_cast<const float4 *>(X + (int64_t)k * ldx + cj)) : zero4;
            return;
        }
        // lanes take consecutive columns (conflict-free transposed stores)
        const int cc = tid & (kGrT - 1), kq = tid >> 6;
        const int k = k0 + 4 * kq;
        const int ci = i0 + cc, cj = j0 + cc;
        ri = (ci < n && k < K) ? __ldg(reinterpret_cast<const float4 *>(X + (int64_t)ci * ldx + k)) : zero4;
        rj = (cj < n && k < K) ? __ldg(reinterpret_cast<const float4 *>(X + (int64_t)cj * ldx + k)) : zero4;
    };
    auto store_tile = [&](int buf) {
        if (KSLOW) {
            const int cq = tid & 15, kk = tid >> 4;
            *reinterpret_cast<float4 *>(&Xi[buf][kk][4 * cq]) = ri;
            *reinterpret_cast<float4 *>(&Xj[buf][kk][4 * cq]) = rj;
            return;
        }
        const int cc = tid & (kGrT - 1), kq = tid >> 6;
        Xi[buf][4 * kq + 0][cc] = ri.x; Xi[buf][4 * kq + 1][cc] = ri.y;
        Xi[buf][4 * kq + 2][cc] = ri.z; Xi[buf][4 * kq + 3][cc] = ri.w;
        Xj[buf][4 * kq + 0][cc] = rj.x; Xj[buf][4 * kq + 1][cc] = rj.y;
        Xj[buf][4 * kq + 2][cc] = rj.z; Xj[buf][4 * kq + 3][cc] = rj.w;
    };
    DF acc[4][4];
    double acc64[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            acc[a][b] = DF{0.f, 0.f};
            acc64[a][b] = 0.0;
        }
    const int nk = (K + kGrBK - 1) / kGrBK;
    load_tile(0);
    store_tile(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) load_tile((kt + 1) * kGrBK);
#pragma unroll 4
        for (int kk = 0; kk < kGrBK; ++kk) {
            const float4 va = *reinterpret_cast<const float4 *>(&Xi[buf][kk][4 * ty]);
            const float4 vb = *reinterpret_cast<const float4 *>(&Xj[buf][kk][4 * tx]);
            const float a[4] = {va.x, va.y, va.z, va.w};
            const float b[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) df_acc_prod(acc[p][q], a[p], b[q]);
        }
        if ((kt + 1) % kGrFoldTiles == 0 || kt + 1 == nk) {
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc64[p][q] += (double)acc[p][q].hi + (double)acc[p][q].lo;
                    acc[p][q] = DF{0.f, 0.f};
                }
        }
        if (kt + 1 < nk) store_tile(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + 4 * ty + p, j = j0 + 4 * tx + q;
            if (i >= n || j >= n || i < j) continue;
            const double v = acc64[p][q];
            double *dst = G + (int64_t)i + (int64_t)n * j;
            *dst = accumulate ? *dst + v : v;
        }
}

// rh[s] + rl[s] = r[s] to FP32-pair precision (48 bits)
__global__ void k_split_df(const double *__restrict__ r, int64_t n, float *__restrict__ rh, float *__restrict__ rl) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)r[s];
        rh[s] = h;
        rl[s] = (float)(r[s] - (double)h);
    }
}

__device__ __forceinline__ double block_sum_fixed(double v, double *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// tp[c ell + j] = sum over the rows s of chunk c of Y[s + ldy j] (rh[s] + rl[s]):
// a CTA per (16 columns, 8192-row chunk); each thread walks rows s0 + tid,
// s0 + tid + 256, ... and reads rh, rl once for its 16 columns (one
// double-float accumulator per column, runs of 128 rows folded into FP64;
// 18 independent loads per row in flight), then the 256 threads' sums of
// each column are added in a fixed order.  One CTA per column, reading r
// for every column, spent ~8 ms per launch at 178,797 x 3,973 (every CTA
// streamed the same 1.4 MB of r through L2) for 2.8 GB of Y.
constexpr int kGtCols = 16, kGtRows = 8192;
__global__ void __launch_bounds__(256) k_gemv_t_df(const float *__restrict__ Y, int64_t ldy, int64_t n, int ell,
                                                   const float *__restrict__ rh, const float *__restrict__ rl,
                                                   double *__restrict__ tp) {
    __shared__ double red[kGtCols][256 + 1];
    const int j0 = blockIdx.x * kGtCols;
    const int nc = min(kGtCols, ell - j0);
    const int64_t s0 = (int64_t)blockIdx.y * kGtRows, s1 = min(n, s0 + kGtRows);
    DF acc[kGtCols];
    float small[kGtCols];
    double v[kGtCols];
#pragma unroll
    for (int c = 0; c < kGtCols; ++c) {
        acc[c] = DF{0.f, 0.f};
        small[c] = 0.0f;
        v[c] = 0.0;
    }
    int run = 0;
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const float h = rh[s], l = rl[s];
        float a[kGtCols];
#pragma unroll
        for (int c = 0; c < kGtCols; ++c) a[c] = (c < nc) ? __ldcs(Y + s + ldy * (int64_t)(j0 + c)) : 0.0f;
#pragma unroll
        for (int c = 0; c < kGtCols; ++c) {
            df_acc_prod(acc[c], a[c], h);
            small[c] = fmaf(a[c], l, small[c]);
        }
        if (++run == kDfRun) {   // runs of 128 terms into FP64
#pragma unroll
            for (int c = 0; c < kGtCols; ++c) {
                v[c] += (double)acc[c].hi + (double)acc[c].lo + (double)small[c];
                acc[c] = DF{0.f, 0.f};
                small[c] = 0.0f;
            }
            run = 0;
        }
    }
#pragma unroll
    for (int c = 0; c < kGtCols; ++c) red[c][threadIdx.x] = v[c] + ((double)acc[c].hi + (double)acc[c].lo + (double)small[c]);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < nc; c += (int)(blockDim.x >> 5)) {
        double x = 0.0;
        for (int k = lane; k < 256; k += 32) x += red[c][k];
        x = warp_sum(x);
        if (lane == 0) tp[(int64_t)blockIdx.y * ell + j0 + c] = x;
    }
}

// t[j] = sum_c tp[c ell + j] over the row chunks, in chunk order
__global__ void k_sum_chunks(const double *__restrict__ tp, int nch, int ell, double *__restrict__ t) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ell) return;
    double x = 0.0;
    for (int c = 0; c < nch; ++c) x += tp[(int64_t)c * ell + j];
    t[j] = x;
}

// u[i] = sum_{j <= i} Li[i + ell j] t[j]   (thread per row)
__global__ void k_trmv_lo(const double *__restrict__ Li, int ell, const double *__restrict__ t, double *__restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ell) return;
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s = fma(Li[(int64_t)i + (int64_t)ell * j], t[j], s);
    u[i] = s;
}

// v[j] = sum_{i >= j} Li[i + ell j] u[i]   (warp per column)
__global__ void k_trmv_lo_t(const double *__restrict__ Li, int ell, const double *__restrict__ u, double *__restrict__ v) {
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= ell) return;
    double s = 0.0;
    for (int i = j + lane; i < ell; i += 32) s = fma(Li[(int64_t)i + (int64_t)ell * j], u[i], s);
    s = warp_sum(s);
    if (lane == 0) v[j] = s;
}

// z[s] = (r[s] - sum_j Y[s + ldy j] (vh[j] + vl[j])) / mu   (thread per row,
// double-float sums in a fixed column order)
__global__ void __launch_bounds__(256) k_gemv_n_df(const float *__restrict__ Y, int64_t ldy, int64_t n, int ell,
                                                   const float *__restrict__ vh, const float *__restrict__ vl,
                                                   const double *__restrict__ r, double inv_mu,
                                                   double *__restrict__ z) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    DF acc{0.f, 0.f};
    float small = 0.0f;
    double yv = 0.0;
    const float *y = Y + s;
    int j = 0;
    // 16 columns per step: 16 independent loads in flight per thread (4 per
    // step reached ~1.2 TB/s at 178,797 x 3,973, latency-bound)
    for (; j + 16 <= ell; j += 16) {
        if (j % kDfRun == 0 && j > 0) {   // runs of 128 terms into FP64
            yv += (double)acc.hi + (double)acc.lo + (double)small;
            acc = DF{0.f, 0.f};
            small = 0.0f;
        }
        float a[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) a[q] = __ldcs(y + (int64_t)ldy * (j + q));
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            df_acc_prod(acc, a[q], vh[j + q]);
            small = fmaf(a[q], vl[j + q], small);
        }
    }
    if (j % kDfRun == 0 && j > 0 && j < ell) {
        yv += (double)acc.hi + (double)acc.lo + (double)small;
        acc = DF{0.f, 0.f};
        small = 0.0f;
    }
    for (; j < ell; ++j) {
        const float a = __ldcs(y + (int64_t)ldy * j);
        df_acc_prod(acc, a, vh[j]);
        small = fmaf(a, vl[j], small);
    }
    yv += (double)acc.hi + (double)acc.lo + (double)small;
    z[s] = (r[s] - yv) * inv_mu;
}

inline unsigned blocks_for(int64_t n, int threads, int64_t cap = 148 * 32) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

}  // namespace

int launch_sgemm(bool a_kmajor, int M, int N, int K, const float *A, int64_t lda, const float *B, int64_t ldb,
                 float *C, int64_t ldc, bool accumulate, cudaStream_t s, bool b_nmajor, bool c_nmajor) {
    if (M <= 0 || N <= 0) return 0;
    if ((lda | ldb | ldc | K | M) & 3) return -1;
    const int64_t n4 = ((int64_t)N + 3) / 4 * 4;
    if ((b_nmajor && ldb < n4) || (c_nmajor && ldc < n4)) return -1;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15)
        return -1;
    dim3 grid((unsigned)((M + kGmBM - 1) / kGmBM), (unsigned)((N + kGmBN - 1) / kGmBN));
    if (grid.y > 65535) return -1;
    const int acc = accumulate ? 1 : 0;
    auto go = [&](auto kern) { kern<<<grid, kGmThreads, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, acc); };
    if (a_kmajor) {
        if (b_nmajor) c_nmajor ? go(k_sgemm<true, true, true>) : go(k_sgemm<true, true, false>);
        else c_nmajor ? go(k_sgemm<true, false, true>) : go(k_sgemm<true, false, false>);
    } else {
        if (b_nmajor) c_nmajor ? go(k_sgemm<false, true, true>) : go(k_sgemm<false, true, false>);
        else c_nmajor ? go(k_sgemm<false, false, true>) : go(k_sgemm<false, false, false>);
    }
    note_launches(1);
    return 0;
}

int launch_gram_df(int n, int K, const float *X, int64_t ldx, double *G, bool accumulate, cudaStream_t s,
                   bool k_slow) {
    if (n <= 0) return 0;
    if ((ldx | K) & 3 || (reinterpret_cast<uintptr_t>(X) & 15)) return -1;
    if (k_slow && ldx < ((int64_t)n + 3) / 4 * 4) return -1;
    const int nt = (n + kGrT - 1) / kGrT;
    const int64_t tiles = (int64_t)nt * (nt + 1) / 2;
    if (k_slow)
        k_gram_df<true><<<(unsigned)tiles, kGrThreads, 0, s>>>(n, K, X, ldx, G, accumulate ? 1 : 0);
    else
        k_gram_df<false><<<(unsigned)tiles, kGrThreads, 0, s>>>(n, K, X, ldx, G, accumulate ? 1 : 0);
    note_launches(1);
    return 0;
}

int64_t nys_tpart_chunks(int64_t n) { return std::max<int64_t>(1, (n + kGtRows - 1) / kGtRows); }

void launch_nys_apply(const float *Y, int64_t ldy, int64_t n, int ell, const double *Linv, double mu,
                      const double *r, double *z, float *rh, float *rl, double *tp, double *t, double *u, double *v,
                      float *vh, float *vl, cudaStream_t s) {
    k_split_df<<<blocks_for(n, 256), 256, 0, s>>>(r, n, rh, rl);
    const int nch = (int)nys_tpart_chunks(n);
    k_gemv_t_df<<<dim3((unsigned)((ell + kGtCols - 1) / kGtCols), (unsigned)nch), 256, 0, s>>>(Y, ldy, n, ell, rh, rl,
                                                                                              tp);
    k_sum_chunks<<<(unsigned)((ell + 127) / 128), 128, 0, s>>>(tp, nch, ell, t);
    k_trmv_lo<<<(unsigned)((ell + 127) / 128), 128, 0, s>>>(Linv, ell, t, u);
    k_trmv_lo_t<<<(unsigned)((ell * 32 + 255) / 256), 256, 0, s>>>(Linv, ell, u, v);
    k_split_df<<<blocks_for(ell, 256), 256, 0, s>>>(v, ell, vh, vl);
    k_gemv_n_df<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Y, ldy, n, ell, vh, vl, r, 1.0 / mu, z);
    note_launches(7);
}

}  // namespace grav
