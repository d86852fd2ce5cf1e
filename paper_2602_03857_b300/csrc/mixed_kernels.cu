// Mixed-precision prism-gravity operator (GRAV_MIXED), uniform a x b x c cells.
//
// Far field (every cell, FP32): a uniform cube attracts like a point mass
// at its centre up to a relative error O((a/R)^4) (its quadrupole moment
// vanishes), so G_ik ~ gamma V dz / R^3; other boxes carry their quadrupole
// factor (far_kernel_q, the QUAD instantiations).  One MUFU reciprocal square
// root per (station, cell) pair; per-column FP32 sums are folded into a (hi, lo)
// pair by Knuth's two-sum (compensated accumulation), partials are combined
// in FP64 in a fixed order.
//
// Near field (FP64): for every station, the cells whose centre lies within
// near_cells cell widths get the correction dG = G_exact - G_far, where
// G_exact is Eq. 1 evaluated in FP64 with the corner function shared across
// the nodes of the station's window box.  dG is built once per plan and
// applied on every product (forward: per-station row sums; adjoint: a
// deterministic per-cell gather over stations binned by box origin).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cub/device/device_radix_sort.cuh>
#include <type_traits>

#include "device_common.cuh"
#include "internal.h"

namespace grav {

namespace {

// Launch-shape constants (compile-time tunables; the defaults are the measured best).
#ifndef GRAV_MF_T
#define GRAV_MF_T 8
#endif
#ifndef GRAV_MF_MINB
#define GRAV_MF_MINB 4
#endif
#ifndef GRAV_MA_MINB
#define GRAV_MA_MINB 0          // 0: per-TZ default below
#endif
#ifndef GRAV_MA_STAGE
#define GRAV_MA_STAGE 1024
#endif
#ifndef GRAV_MA_TZ
#define GRAV_MA_TZ 0
#endif
#ifndef GRAV_AB_FORCE
#define GRAV_AB_FORCE -1        // -1: choose the adjoint layout by size; 0/1 force it
#endif
constexpr int kMfThreads = 128;
constexpr int kMfT = GRAV_MF_T;          // stations per thread (far forward)
constexpr int kMaWarps = 8;              // warps per CTA (far adjoint)
constexpr int kMaStage = GRAV_MA_STAGE;  // stations per TMA stage (far adjoint)
constexpr int kNsWarps = 8;              // warps per CTA (near set-up)

// CTAs per SM the adjoint is compiled for (register budget 65536 / (256 * minB)):
// measured on B300 at 210 x 210 x 75 -- TZ = 8 is fastest at 3 (79 registers),
// TZ >= 12 at 2 (up to 127 registers; the extra ILP beats the lost occupancy).
template <int TZ>
struct MaMinBlocks {
    static constexpr int value = GRAV_MA_MINB > 0 ? GRAV_MA_MINB : (TZ <= 8 ? 3 : 2);
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct MfwdSmem {
    size_t cx, cy, cz, q, total;
};
__host__ __device__ MfwdSmem mfwd_layout(const MixedGeo &g, int cols_per_stage) {
    MfwdSmem L;
    L.cx = 128;
    L.cy = L.cx + 8ull * g.nx;
    L.cz = align_up(L.cy + 8ull * g.ny, 16);
    L.q = align_up(L.cz + 4ull * g.nzp, 128);
    L.total = L.q + 2ull * cols_per_stage * g.nzp * 4;
    return L;
}

// ---------------------------------------------------------------------------
// The FP32 operands of the mixed products are normalised by the largest
// magnitude of the input vector (m for the forward, r for the adjoint), and
// the FP64 results are multiplied back: the products are homogeneous in
// their input up to rounding at any scale, instead of flushing to zero (or
// overflowing) when the input leaves the range where FP32 products of it
// with dz / R^3 stay normal.
//
// max |v_i| as the bit pattern of a non-negative double (atomicMax on the
// bits orders non-negative doubles numerically); *bits must start at 0.
__global__ void k_absmax(const double *__restrict__ v, int64_t n, unsigned long long *__restrict__ bits) {
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(v[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(bits, (unsigned long long)__double_as_longlong(m));
}

// 1 / max|v| (0 for a zero vector), or 1 without normalisation (bits null)
__device__ __forceinline__ double inv_scale(const unsigned long long *bits) {
    if (!bits) return 1.0;
    const double vm = __longlong_as_double((long long)*bits);
    return vm > 0.0 ? 1.0 / vm : 0.0;
}

// qT[col][l] = gamma*1e5*V * m[i + nx*(j + ny*l)] / max|m|, col = i + nx*j; l >= nz: 0.
// ---------------------------------------------------------------------------
__global__ void k_prep_q(MixedGeo g, const double *__restrict__ m, float scale, const unsigned long long *bits,
                         float *__restrict__ qT) {
    const double sc = scale * inv_scale(bits);
    const int64_t total = (int64_t)g.ncol * g.nzp;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(t % g.nzp);
        const int64_t col = t / g.nzp;
        qT[t] = (l < g.nz) ? (float)(sc * m[col + (int64_t)g.ncol * l]) : 0.0f;
    }
}

// the same FP32 q in the cells' natural order (coalesced gathers of the near field)
__global__ void k_prep_qn(int64_t M, const double *__restrict__ m, float scale, const unsigned long long *bits,
                          float *__restrict__ qn) {
    const double sc = scale * inv_scale(bits);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x)
        qn[k] = (float)(sc * m[k]);
}

// stations: st32 = (xh, xl, yh, yl) of (x - xref, y - yref); stz = (z, r / max|r|) (k_set_rz)
__global__ void k_prep_stations(const double *__restrict__ x, const double *__restrict__ y,
                                const double *__restrict__ z, int64_t n, double xref, double yref,
                                float4 *__restrict__ st32, float2 *__restrict__ stz) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double xr = x[i] - xref, yr = y[i] - yref;
        const float xh = (float)xr, yh = (float)yr;
        st32[i] = make_float4(xh, (float)(xr - (double)xh), yh, (float)(yr - (double)yh));
        stz[i] = make_float2((float)z[i], 0.0f);
    }
}

// stz[i].y = r_i / max|r|
__global__ void k_set_rz(float2 *__restrict__ stz, const double *__restrict__ r, int64_t n,
                         const unsigned long long *bits) {
    const double sc = inv_scale(bits);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        stz[i].y = (float)(sc * r[i]);
}

// The far-field geometry of one (station, cell) pair exactly as every mixed
// kernel computes it (same FP32 operations in the same order).
__device__ __forceinline__ float far_h2(float2 X, float2 Y, float xh, float xl, float yh, float yl) {
    const float dx = (X.x - xh) + (X.y - xl);
    const float dy = (Y.x - yh) + (Y.y - yl);
    return fmaf(dx, dx, dy * dy);
}

// One pair's far-field term in scalar form: the operations of far_pair on
// one half (used for the odd layer left over by the packed layer pairs).
template <bool QUAD>
__device__ __forceinline__ float far_one(float zc, float nzs, float h2, float w, float acc, float qg, float ph) {
    const float dz = zc + nzs;
    const float R2 = fmaf(dz, dz, h2);
    return fmaf(w, far_k<QUAD>(dz, R2, qg, ph), acc);
}

// ---------------------------------------------------------------------------
// Far-field forward.  CTA = (station tile of kMfThreads*T stations, chunk of
// columns).  Column densities qT stream through shared memory by TMA bulk
// copies (double-buffered); stations (hi/lo coordinates, accumulators) stay
// in registers; the inner loop reads 4 layers of q and depth per LDS.128
// (broadcast) and issues per pair: FADD, FFMA, MUFU.RSQ, 3 FMUL, FFMA.
// ---------------------------------------------------------------------------
template <int T, bool QUAD, bool TAIL>
__global__ void __launch_bounds__(kMfThreads, GRAV_MF_MINB) k_mfwd(MixedGeo g, const float *__restrict__ qT,
                                                     const float4 *__restrict__ st32,
                                                     const float2 *__restrict__ stz, int cols_per_chunk,
                                                     int cols_per_stage, double *__restrict__ part,
                                                     int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const MfwdSmem L = mfwd_layout(g, cols_per_stage);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    int *flag = reinterpret_cast<int *>(smem_raw + 16);
    float2 *cxs = reinterpret_cast<float2 *>(smem_raw + L.cx);
    float2 *cys = reinterpret_cast<float2 *>(smem_raw + L.cy);
    float *czs = reinterpret_cast<float *>(smem_raw + L.cz);
    float *qbuf = reinterpret_cast<float *>(smem_raw + L.q);

    const int c0 = blockIdx.y * cols_per_chunk;
    const int c1 = min(g.ncol, c0 + cols_per_chunk);
    const int nst = (c1 > c0) ? (c1 - c0 + cols_per_stage - 1) / cols_per_stage : 0;

    const int64_t s_base = (int64_t)blockIdx.x * (kMfThreads * T) + threadIdx.x;
    float xh[T], xl[T], yh[T], yl[T], hi[T], lo[T];
    f2_t nzs[T];   // (-z, -z) of each station
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t s = s_base + (int64_t)t * kMfThreads;
        const bool ok = s < g.N;
        const float4 P = ok ? st32[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        xh[t] = P.x; xl[t] = P.y; yh[t] = P.z; yl[t] = P.w;
        const float zs = ok ? stz[s].x : -1.0f;
        nzs[t] = f2_pack(-zs, -zs);
        hi[t] = 0.f; lo[t] = 0.f;
    }
    for (int i = threadIdx.x; i < g.nx; i += kMfThreads) cxs[i] = make_float2(g.cx[2 * i], g.cx[2 * i + 1]);
    for (int j = threadIdx.x; j < g.ny; j += kMfThreads) cys[j] = make_float2(g.cy[2 * j], g.cy[2 * j + 1]);
    for (int l = threadIdx.x; l < g.nzp; l += kMfThreads) czs[l] = g.czc[l];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int st) {
        const int buf = st & 1;
        const int ca = c0 + st * cols_per_stage;
        const int cb = min(c1, ca + cols_per_stage);
        const uint32_t bytes = (uint32_t)(cb - ca) * (uint32_t)g.nzp * 4u;
        mbar_arrive_expect_tx(&bar[buf], bytes);
        tma_load_1d(qbuf + (size_t)buf * cols_per_stage * g.nzp, qT + (size_t)ca * g.nzp, bytes, &bar[buf]);
    };
    if (threadIdx.x == 0) {
        if (nst > 0) issue(0);
        if (nst > 1) issue(1);
    }
    // TAIL: whole groups of 4 layers, then the nz mod 4 layers left (a pair
    // and/or one scalar layer through the same operations), so no padded
    // layer costs a reciprocal square root; without TAIL (nz a multiple of 4,
    // and the non-cubic kernels, which would spill registers with the tail
    // code) the last group is zero-padded.  Measured at nz = 75: 135.3 ms
    // against 135.7 ms padded; a tail resolved at compile time took 137.5 ms.
    const int nf4 = TAIL ? (g.nz >> 2) : (g.nzp >> 2);
    const int tail = TAIL ? (g.nz & 3) : 0;
    const f2_t qg2 = f2_pack(g.qg, g.qg);
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        if (threadIdx.x == 0) *flag = mbar_wait_bounded(&bar[buf], (st >> 1) & 1) ? 1 : 0;
        __syncthreads();
        if (!*flag) {
            if (threadIdx.x == 0) {
                set_status(status, kStatusMbarTimeout);
                if (st + 1 < nst) (void)mbar_wait_bounded(&bar[buf ^ 1], ((st + 1) >> 1) & 1);
            }
            return;
        }
        const int ca = c0 + st * cols_per_stage;
        const int cb = min(c1, ca + cols_per_stage);
        const float *qb = qbuf + (size_t)buf * cols_per_stage * g.nzp;
        int i = ca % g.nx, j = ca / g.nx;
        for (int col = ca; col < cb; ++col) {
            const float2 X = cxs[i], Y = cys[j];
            if (++i == g.nx) { i = 0; ++j; }
            // layer pairs (l, l+1) of this column share one packed f32x2 chain per station
            f2_t h2p[T], cs2[T], php[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float h = far_h2(X, Y, xh[t], xl[t], yh[t], yl[t]);
                h2p[t] = f2_pack(h, h);
                cs2[t] = 0ull;
                if (QUAD) {
                    const float ph = far_ph(X, Y, xh[t], xl[t], yh[t], yl[t], g.qa, g.qb);
                    php[t] = f2_pack(ph, ph);
                } else {
                    php[t] = 0ull;
                }
            }
            const float4 *q4 = reinterpret_cast<const float4 *>(qb + (size_t)(col - ca) * g.nzp);
            const float4 *z4 = reinterpret_cast<const float4 *>(czs);
            for (int l4 = 0; l4 < nf4; ++l4) {
                const float4 q = q4[l4], z = z4[l4];
                const f2_t q01 = f2_pack(q.x, q.y), q23 = f2_pack(q.z, q.w);
                const f2_t z01 = f2_pack(z.x, z.y), z23 = f2_pack(z.z, z.w);
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    cs2[t] = far_pair<QUAD>(z01, nzs[t], h2p[t], q01, cs2[t], qg2, php[t]);
                    cs2[t] = far_pair<QUAD>(z23, nzs[t], h2p[t], q23, cs2[t], qg2, php[t]);
                }
            }
            float cs1[T];   // the odd layer left (tail 1 or 3), one term per station
            if (TAIL) {
#pragma unroll
                for (int t = 0; t < T; ++t) cs1[t] = 0.0f;
                if (tail) {
                    const float4 q = q4[nf4], z = z4[nf4];
                    if (tail & 2) {
                        const f2_t q01 = f2_pack(q.x, q.y), z01 = f2_pack(z.x, z.y);
#pragma unroll
                        for (int t = 0; t < T; ++t)
                            cs2[t] = far_pair<QUAD>(z01, nzs[t], h2p[t], q01, cs2[t], qg2, php[t]);
                    }
                    if (tail & 1) {
                        const float ql = (tail == 3) ? q.z : q.x, zl = (tail == 3) ? z.z : z.x;
#pragma unroll
                        for (int t = 0; t < T; ++t) {
                            float nz1, nzu, h2, h2u, ph = 0.0f, phu;
                            f2_unpack(nzs[t], nz1, nzu);
                            f2_unpack(h2p[t], h2, h2u);
                            if (QUAD) f2_unpack(php[t], ph, phu);
                            cs1[t] = far_one<QUAD>(zl, nz1, h2, ql, 0.0f, g.qg, ph);
                        }
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                float a, b, s, e;
                f2_unpack(cs2[t], a, b);
                float c = a + b;
                if (TAIL) c += cs1[t];
                two_sum(hi[t], c, s, e);
                hi[t] = s;
                lo[t] += e;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && st + 2 < nst) {
            fence_proxy_async_smem();
            issue(st + 2);
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t s = s_base + (int64_t)t * kMfThreads;
        if (s < g.N) part[(int64_t)blockIdx.y * g.N + s] = (double)hi[t] + (double)lo[t];
    }
}

// ---------------------------------------------------------------------------
// Far-field adjoint: acc_k = sum_i r_i dz/R^3.  A warp owns TZ cells of one
// column (layers lg*TZ ...); its lanes split the stations of the CTA's chunk
// (x/y hi-lo and (z, r) staged in shared memory by two TMA bulk copies per
// stage).  Layer pairs share one packed f32x2 chain per station (far_pair,
// the forward's per-pair operations).  Each lane sums its stations of one
// stage in FP32, folds that stage sum into (hi, lo) by two-sum, and at the
// end the 32 lane values are reduced by a warp-shuffle butterfly in FP64
// (fixed order: deterministic).
// ---------------------------------------------------------------------------
template <int TZ, bool QUAD>
__global__ void __launch_bounds__(kMaWarps * 32, MaMinBlocks<TZ>::value) k_madj(MixedGeo g, const float4 *__restrict__ st32,
                                                        const float2 *__restrict__ stz, int ngz,
                                                        int64_t schunk_len, double *__restrict__ apart,
                                                        int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    int *flag = reinterpret_cast<int *>(smem_raw + 16);
    float4 *sxy = reinterpret_cast<float4 *>(smem_raw + 128);
    float2 *szr = reinterpret_cast<float2 *>(smem_raw + 128 + 2 * kMaStage * sizeof(float4));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t group = (int64_t)blockIdx.x * kMaWarps + warp;
    const bool gvalid = group < (int64_t)g.ncol * ngz;
    const int col = gvalid ? (int)(group / ngz) : 0;
    const int l0 = gvalid ? (int)(group % ngz) * TZ : 0;
    const int i = col % g.nx, j = col / g.nx;
    const float2 X = make_float2(g.cx[2 * i], g.cx[2 * i + 1]);
    const float2 Y = make_float2(g.cy[2 * j], g.cy[2 * j + 1]);
    static_assert(TZ % 2 == 0, "layer pairs");
    const f2_t qg2 = f2_pack(g.qg, g.qg);
    f2_t zcp[TZ / 2];
    float hi[TZ], lo[TZ];
#pragma unroll
    for (int u = 0; u < TZ / 2; ++u)
        zcp[u] = f2_pack(g.czc[min(l0 + 2 * u, g.nzp - 1)], g.czc[min(l0 + 2 * u + 1, g.nzp - 1)]);
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        hi[t] = 0.f; lo[t] = 0.f;
    }
    const int64_t s0 = (int64_t)blockIdx.y * schunk_len;
    const int64_t s1 = min(g.N, s0 + schunk_len);
    const int nst = (s1 > s0) ? (int)((s1 - s0 + kMaStage - 1) / kMaStage) : 0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int st) {
        const int buf = st & 1;
        const int64_t sa = s0 + (int64_t)st * kMaStage;
        const int cnt = (int)min((int64_t)kMaStage, s1 - sa);
        const uint32_t b1 = (uint32_t)cnt * 16u;
        const uint32_t b2 = (uint32_t)((cnt * 8 + 15) / 16 * 16);
        mbar_arrive_expect_tx(&bar[buf], b1 + b2);
        tma_load_1d(sxy + buf * kMaStage, st32 + sa, b1, &bar[buf]);
        tma_load_1d(szr + buf * kMaStage, stz + sa, b2, &bar[buf]);
    };
    if (threadIdx.x == 0) {
        if (nst > 0) issue(0);
        if (nst > 1) issue(1);
    }
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        if (threadIdx.x == 0) *flag = mbar_wait_bounded(&bar[buf], (st >> 1) & 1) ? 1 : 0;
        __syncthreads();
        if (!*flag) {
            if (threadIdx.x == 0) {
                set_status(status, kStatusMbarTimeout);
                if (st + 1 < nst) (void)mbar_wait_bounded(&bar[buf ^ 1], ((st + 1) >> 1) & 1);
            }
            return;
        }
        const int64_t sa = s0 + (int64_t)st * kMaStage;
        const int cnt = (int)min((int64_t)kMaStage, s1 - sa);
        const float4 *pb = sxy + buf * kMaStage;
        const float2 *zb = szr + buf * kMaStage;
        if (gvalid) {
            f2_t cs2[TZ / 2];
#pragma unroll
            for (int u = 0; u < TZ / 2; ++u) cs2[u] = 0ull;
            for (int k = lane; k < cnt; k += 32) {
                const float4 P = pb[k];
                const float2 Z = zb[k];
                const float h = far_h2(X, Y, P.x, P.y, P.z, P.w);
                const f2_t h2p = f2_pack(h, h), nz2 = f2_pack(-Z.x, -Z.x), w2 = f2_pack(Z.y, Z.y);
                f2_t ph2 = 0ull;
                if (QUAD) {
                    const float ph = far_ph(X, Y, P.x, P.y, P.z, P.w, g.qa, g.qb);
                    ph2 = f2_pack(ph, ph);
                }
#pragma unroll
                for (int u = 0; u < TZ / 2; ++u) cs2[u] = far_pair<QUAD>(zcp[u], nz2, h2p, w2, cs2[u], qg2, ph2);
            }
#pragma unroll
            for (int u = 0; u < TZ / 2; ++u) {
                float a, b, s, e;
                f2_unpack(cs2[u], a, b);
                two_sum(hi[2 * u], a, s, e);
                hi[2 * u] = s;
                lo[2 * u] += e;
                two_sum(hi[2 * u + 1], b, s, e);
                hi[2 * u + 1] = s;
                lo[2 * u + 1] += e;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && st + 2 < nst) {
            fence_proxy_async_smem();
            issue(st + 2);
        }
    }
    if (!gvalid) return;
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        const double v = warp_sum((double)hi[t] + (double)lo[t]);
        if (lane == t % 32 && l0 + t < g.nz)
            apart[(int64_t)blockIdx.y * g.ncol * (int64_t)g.nz + col + (int64_t)g.ncol * (l0 + t)] = v;
    }
}


// ---------------------------------------------------------------------------
// Far-field adjoint, broadcast layout (large meshes): each lane owns TZ cells
// of one column (lanes = consecutive columns, one layer group per CTA), the
// stations of a TMA-staged chunk are read by all lanes at once (shared-memory
// broadcast), and every lane accumulates its own cells: no cross-lane
// reduction.  Sums run in FP32 over 128 stations and are folded into FP64
// accumulators (compensation by wider precision; the FP64 adds run on the
// otherwise idle FP64 pipe).  Every pair's kernel value dz / R^3 comes from
// the same FP32 operations as in the forward (far_pair), so the mixed G^T is
// the transpose of the mixed G term by term: CG on G W^-2 G^T needs that
// symmetry (a variant that folded r into the pair geometry, one FP32
// operation per pair fewer and 2 % faster, perturbed each term by a few ulp
// and took 346 instead of 247 iterations on the 150 x 150 x 60 inversion).
// ---------------------------------------------------------------------------
#ifndef GRAV_AB_MINB
#define GRAV_AB_MINB 2
#endif
constexpr int kAbWarps = 8;
constexpr int kAbStage = 1024;
// FP32 run length before the FP64 fold.  Measured at 210 x 210 x 75 x 178,797:
// 64 / 128 / 256 stations take 142.5 / 139.3 / 138.7 ms, while the rounding
// noise of G^T r (|G^T(a+b) - G^T a - G^T b| / |G^T(a+b)| for white-noise r)
// is 2.1e-7 / ~2.9e-7 / 4.1e-7; the CG on G W^-2 G^T stalls near that noise
// floor, so 128 trades 0.4 % of the adjoint for a lower floor.
constexpr int kAbFold = 128;

// One lane's NL cells (layers l0 .. l0 + NL - 1 of one column): NL / 2 layer
// pairs in packed f32x2 chains and, for odd NL, the last layer alone through
// the same operations in scalar form (far_one), so no padded layer costs a
// reciprocal square root.

template <int NL, bool QUAD>
__device__ __forceinline__ void madj_bc_body(const MixedGeo &g, const float4 *__restrict__ st32,
                                             const float2 *__restrict__ stz, int l0, int cb, int64_t schunk_len,
                                             double *__restrict__ apart, int *status, unsigned char *smem_raw) {
    constexpr int NP = NL / 2;            // packed layer pairs
    constexpr bool ODD = (NL & 1) != 0;   // one more layer, scalar
    constexpr int NPA = NP > 0 ? NP : 1;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    int *flag = reinterpret_cast<int *>(smem_raw + 16);
    float4 *sxy = reinterpret_cast<float4 *>(smem_raw + 128);
    float2 *szr = reinterpret_cast<float2 *>(smem_raw + 128 + 2 * kAbStage * sizeof(float4));

    const int col = cb * (kAbWarps * 32) + threadIdx.x;
    const bool cvalid = col < g.ncol;
    const int cc = cvalid ? col : 0;
    const int i = cc % g.nx, j = cc / g.nx;
    const float2 X = make_float2(g.cx[2 * i], g.cx[2 * i + 1]);
    const float2 Y = make_float2(g.cy[2 * j], g.cy[2 * j + 1]);
    const f2_t qg2 = f2_pack(g.qg, g.qg);
    f2_t zcp[NPA], cs2[NPA];
    double acc[NL];
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        zcp[u] = f2_pack(g.czc[min(l0 + 2 * u, g.nzp - 1)], g.czc[min(l0 + 2 * u + 1, g.nzp - 1)]);
        cs2[u] = 0ull;
    }
#pragma unroll
    for (int t = 0; t < NL; ++t) acc[t] = 0.0;
    const float zc1 = ODD ? g.czc[min(l0 + NL - 1, g.nzp - 1)] : 0.0f;
    float cs1 = 0.0f;
    const int64_t s0 = (int64_t)blockIdx.y * schunk_len;
    const int64_t s1 = min(g.N, s0 + schunk_len);
    const int nst = (s1 > s0) ? (int)((s1 - s0 + kAbStage - 1) / kAbStage) : 0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int st) {
        const int buf = st & 1;
        const int64_t sa = s0 + (int64_t)st * kAbStage;
        const int cnt = (int)min((int64_t)kAbStage, s1 - sa);
        const uint32_t b1 = (uint32_t)cnt * 16u;
        const uint32_t b2 = (uint32_t)((cnt * 8 + 15) / 16 * 16);
        mbar_arrive_expect_tx(&bar[buf], b1 + b2);
        tma_load_1d(sxy + buf * kAbStage, st32 + sa, b1, &bar[buf]);
        tma_load_1d(szr + buf * kAbStage, stz + sa, b2, &bar[buf]);
    };
    if (threadIdx.x == 0) {
        if (nst > 0) issue(0);
        if (nst > 1) issue(1);
    }
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        if (threadIdx.x == 0) *flag = mbar_wait_bounded(&bar[buf], (st >> 1) & 1) ? 1 : 0;
        __syncthreads();
        if (!*flag) {
            if (threadIdx.x == 0) {
                set_status(status, kStatusMbarTimeout);
                if (st + 1 < nst) (void)mbar_wait_bounded(&bar[buf ^ 1], ((st + 1) >> 1) & 1);
            }
            return;
        }
        const int64_t sa = s0 + (int64_t)st * kAbStage;
        const int cnt = (int)min((int64_t)kAbStage, s1 - sa);
        const float4 *pb = sxy + buf * kAbStage;
        const float2 *zb = szr + buf * kAbStage;
        for (int k0 = 0; k0 < cnt; k0 += kAbFold) {
            const int k1 = min(cnt, k0 + kAbFold);
            for (int k = k0; k < k1; ++k) {
                const float4 P = pb[k];
                const float2 Z = zb[k];
                const float h = far_h2(X, Y, P.x, P.y, P.z, P.w);
                const f2_t h2p = f2_pack(h, h), nz2 = f2_pack(-Z.x, -Z.x), w2 = f2_pack(Z.y, Z.y);
                f2_t ph2 = 0ull;
                float ph = 0.0f;
                if (QUAD) {
                    ph = far_ph(X, Y, P.x, P.y, P.z, P.w, g.qa, g.qb);
                    ph2 = f2_pack(ph, ph);
                }
#pragma unroll
                for (int u = 0; u < NP; ++u) cs2[u] = far_pair<QUAD>(zcp[u], nz2, h2p, w2, cs2[u], qg2, ph2);
                if (ODD) cs1 = far_one<QUAD>(zc1, -Z.x, h, Z.y, cs1, g.qg, ph);
            }
#pragma unroll
            for (int u = 0; u < NP; ++u) {
                float a, b;
                f2_unpack(cs2[u], a, b);
                acc[2 * u] += (double)a;
                acc[2 * u + 1] += (double)b;
                cs2[u] = 0ull;
            }
            if (ODD) {
                acc[NL - 1] += (double)cs1;
                cs1 = 0.0f;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && st + 2 < nst) {
            fence_proxy_async_smem();
            issue(st + 2);
        }
    }
    if (!cvalid) return;
#pragma unroll
    for (int t = 0; t < NL; ++t)
        if (l0 + t < g.nz) apart[(int64_t)blockIdx.y * g.ncol * (int64_t)g.nz + col + (int64_t)g.ncol * (l0 + t)] = acc[t];
}

// Layer groups 0 .. ngz-2 hold TZ layers (even), the last group exactly the
// TZL layers left (1 <= TZL <= TZ), so no layer is padded.
template <int TZ, int TZL, bool QUAD>
__global__ void __launch_bounds__(kAbWarps * 32, GRAV_AB_MINB) k_madj_bc(MixedGeo g, const float4 *__restrict__ st32,
                                                                        const float2 *__restrict__ stz, int ngz,
                                                                        int64_t schunk_len,
                                                                        double *__restrict__ apart, int *status) {
    static_assert(TZ % 2 == 0 && TZL >= 1 && TZL <= TZ, "layer groups");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int cblocks = (g.ncol + kAbWarps * 32 - 1) / (kAbWarps * 32);
    const int cb = blockIdx.x % cblocks;
    const int grp = blockIdx.x / cblocks;
    if (TZL == TZ || grp < ngz - 1)
        madj_bc_body<TZ, QUAD>(g, st32, stz, grp * TZ, cb, schunk_len, apart, status, smem_raw);
    else
        madj_bc_body<TZL, QUAD>(g, st32, stz, grp * TZ, cb, schunk_len, apart, status, smem_raw);
}

// ---------------------------------------------------------------------------
// GRAV_MIXED_CORNER forward (diagnostic of the literal FP32 corner-term
// scheme): node weights in FP32 rows, Eq. 2-3 in FP32 once per (station,
// node), FP32 row sums folded by two-sum; structure as the FP64 forward.
// ---------------------------------------------------------------------------
__global__ void k_node_weights32(int nx, int ny, int nz, int ldw, const double *__restrict__ m,
                                 float *__restrict__ w) {
    const int64_t total = (int64_t)(ny + 1) * (nz + 1) * ldw;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t % ldw);
        const int64_t r = t / ldw;
        const int b = (int)(r % (ny + 1));
        const int c = (int)(r / (ny + 1));
        double acc = 0.0;
        if (a <= nx) {
            for (int dc = 0; dc < 2; ++dc) {
                const int l = c - dc;
                if (l < 0 || l >= nz) continue;
                for (int db = 0; db < 2; ++db) {
                    const int j = b - db;
                    if (j < 0 || j >= ny) continue;
                    for (int da = 0; da < 2; ++da) {
                        const int i = a - da;
                        if (i < 0 || i >= nx) continue;
                        const double v = m[i + (int64_t)nx * (j + (int64_t)ny * l)];
                        acc += ((da + db + dc) & 1) ? v : -v;
                    }
                }
            }
        }
        w[t] = (float)acc;
    }
}

constexpr int kCfThreads = 128;
constexpr int kCfT = 4;

template <int T>
__global__ void __launch_bounds__(kCfThreads) k_cfwd32(MixedGeo g, int ldw, const float *__restrict__ w,
                                                      int rows_per_chunk, int rows_per_stage,
                                                      const float4 *__restrict__ st32, const float2 *__restrict__ stz,
                                                      double *__restrict__ part, int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    int *flag = reinterpret_cast<int *>(smem_raw + 16);
    float2 *exs = reinterpret_cast<float2 *>(smem_raw + 128);
    float *wbuf = reinterpret_cast<float *>(smem_raw + 128 + (size_t)((g.nx + 1 + 1) / 2 * 2) * 8);
    const int nrows = (g.ny + 1) * (g.nz + 1);
    const int r0 = blockIdx.y * rows_per_chunk;
    const int r1 = min(nrows, r0 + rows_per_chunk);
    const int nst = (r1 > r0) ? (r1 - r0 + rows_per_stage - 1) / rows_per_stage : 0;
    const int64_t s_base = (int64_t)blockIdx.x * (kCfThreads * T) + threadIdx.x;
    float xh[T], xl[T], yh[T], yl[T], zs[T], hi[T], lo[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t s = s_base + (int64_t)t * kCfThreads;
        const bool ok = s < g.N;
        const float4 P = ok ? st32[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        xh[t] = P.x; xl[t] = P.y; yh[t] = P.z; yl[t] = P.w;
        zs[t] = ok ? stz[s].x : -1.0f;
        hi[t] = 0.f; lo[t] = 0.f;
    }
    for (int a = threadIdx.x; a <= g.nx; a += kCfThreads) exs[a] = make_float2(g.ex[2 * a], g.ex[2 * a + 1]);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int st) {
        const int buf = st & 1;
        const int ra = r0 + st * rows_per_stage;
        const int rb = min(r1, ra + rows_per_stage);
        const uint32_t bytes = (uint32_t)(rb - ra) * (uint32_t)ldw * 4u;
        mbar_arrive_expect_tx(&bar[buf], bytes);
        tma_load_1d(wbuf + (size_t)buf * rows_per_stage * ldw, w + (size_t)ra * ldw, bytes, &bar[buf]);
    };
    if (threadIdx.x == 0) {
        if (nst > 0) issue(0);
        if (nst > 1) issue(1);
    }
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        if (threadIdx.x == 0) *flag = mbar_wait_bounded(&bar[buf], (st >> 1) & 1) ? 1 : 0;
        __syncthreads();
        if (!*flag) {
            if (threadIdx.x == 0) {
                set_status(status, kStatusMbarTimeout);
                if (st + 1 < nst) (void)mbar_wait_bounded(&bar[buf ^ 1], ((st + 1) >> 1) & 1);
            }
            return;
        }
        const float *wb = wbuf + (size_t)buf * rows_per_stage * ldw;
        const int ra = r0 + st * rows_per_stage;
        const int rb = min(r1, ra + rows_per_stage);
        for (int r = ra; r < rb; ++r) {
            const int b = r % (g.ny + 1), c = r / (g.ny + 1);
            const float2 EY = make_float2(g.ey[2 * b], g.ey[2 * b + 1]);
            const float Zc = g.ez[c];
            float dy[T], dz[T], rs[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                dy[t] = (EY.x - yh[t]) + (EY.y - yl[t]);
                dz[t] = Zc - zs[t];
                rs[t] = 0.f;
            }
            const float *wr = wb + (size_t)(r - ra) * ldw;
            for (int a = 0; a <= g.nx; ++a) {
                const float wv = wr[a];
                if (wv == 0.0f) continue;
                const float2 EX = exs[a];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float dx = (EX.x - xh[t]) + (EX.y - xl[t]);
                    rs[t] = fmaf(wv, psi32(dx, dy[t], dz[t]), rs[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                float sum, e;
                two_sum(hi[t], rs[t], sum, e);
                hi[t] = sum;
                lo[t] += e;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && st + 2 < nst) {
            fence_proxy_async_smem();
            issue(st + 2);
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t s = s_base + (int64_t)t * kCfThreads;
        if (s < g.N) part[(int64_t)blockIdx.y * g.N + s] = (double)hi[t] + (double)lo[t];
    }
}

// ---------------------------------------------------------------------------
// Near-field set-up: warp per station.  Psi on those of the (bx+1)(by+1)(bz+1)
// nodes of the station's window box that a cell inside the window radius
// uses (FP64, each node evaluated once), then per box
// cell: dG = G_exact - G_far when the cell centre lies within the window
// radius, else 0.  Also returns the near-field part of diag(G W^-2 G^T),
// sum w2 (G_exact^2 - G_far^2), the box origin and the station's bin key.
// The mesh is uniform: x edges x0 + i a, y edges y0 + j b.
// ---------------------------------------------------------------------------
// MODE: kNsDF (corner function in double-float, the default), kNsF64 (in FP64:
// the near_fp64 option), kNsCorner (FP64 plus the FP32 corner function of the
// GRAV_MIXED_CORNER diagnostic).
constexpr int kNsDF = 0, kNsF64 = 1, kNsCorner = 2;
template <int MODE>
__global__ void __launch_bounds__(kNsWarps * 32) k_near_setup(
    Geo g, MixedGeo mg, NearGeo ng, double x0, double y0, double a, double b, double vol_mgal, double node_r2,
    const double *__restrict__ sx, const double *__restrict__ sy, const double *__restrict__ sz,
    const double *__restrict__ w2, const float4 *__restrict__ st32, const float2 *__restrict__ stz,
    float *__restrict__ dG, int *__restrict__ st_i0, int *__restrict__ st_j0, double *__restrict__ diag_corr,
    unsigned *__restrict__ keys, int *__restrict__ vals, unsigned key_sentinel) {
    constexpr bool CORNER = MODE == kNsCorner, DF = MODE == kNsDF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nbx1 = ng.bx + 1, nby1 = ng.by + 1;
    const int nnode = nbx1 * nby1 * (ng.bz + 1);
    const int nwarps = blockDim.x >> 5;
    double *P = reinterpret_cast<double *>(smem_raw) + (size_t)warp * nnode;
    float *P32 = reinterpret_cast<float *>(reinterpret_cast<double *>(smem_raw) + (size_t)nwarps * nnode) +
                 (size_t)warp * nnode;
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (s >= g.N) return;   // warp-uniform
    const double xs = sx[s], ys = sy[s], zs = sz[s];
    const double lim = 1.0e9;
    // window radius k * width in units of the cell sizes a (x) and b (y)
    // (width = max(a, b, c), so the radius spans >= k columns on each axis)
    const double rad = ng.radius_cells * ng.width;
    const double fx = fmin(fmax((xs - x0) / a - 0.5 - rad / a, -lim), lim);
    const double fy = fmin(fmax((ys - y0) / b - 0.5 - rad / b, -lim), lim);
    const int i0 = (int)floor(fx) + 1;
    const int j0 = (int)floor(fy) + 1;
    // Psi only at the nodes a cell inside the window can use: a cell whose
    // centre lies within the radius has its 8 corners within node_r2 (radius
    // plus half a cell diagonal, squared, with a margin).  The nodes that pass
    // are queued (warp ballot) and evaluated 32 at a time, so the FP64 work
    // follows the window's hemisphere (~half the box) with every lane busy.
    int *queue0 = reinterpret_cast<int *>(reinterpret_cast<double *>(smem_raw) + (size_t)nwarps * nnode) +
                  (CORNER ? (size_t)nwarps * nnode : 0);
    int *queue = queue0 + (size_t)warp * 64;
    // DF: Psi runs in double-float (psi_df, ~2^-45 of R ln R; the FP32 entries
    // of the table need ~2^-39) from the node offsets of the window box, split
    // once per station into double-float in shared memory; P then holds
    // (hi, lo) pairs.  The other modes evaluate the FP64 corner function.
    const int ncrd = nbx1 + nby1 + ng.bz + 1;
    float2 *crd = reinterpret_cast<float2 *>(queue0 + (size_t)nwarps * 64) + (size_t)warp * ncrd;
    float2 *P2 = reinterpret_cast<float2 *>(P);
    const float *Ddf = reinterpret_cast<const float *>(g.fn + kFnDf);
    if (DF) {
        for (int u = lane; u < ncrd; u += 32) {
            double v = 0.0;
            if (u < nbx1) {
                const int ia = i0 + u;
                v = (ia >= 0 && ia <= g.nx) ? g.xe[ia] - xs : 0.0;
            } else if (u < nbx1 + nby1) {
                const int jb = j0 + u - nbx1;
                v = (jb >= 0 && jb <= g.ny) ? g.ye[jb] - ys : 0.0;
            } else {
                const int c = u - nbx1 - nby1;
                v = (c <= g.nz) ? g.ze[c] - zs : 0.0;
            }
            const df32 dv = df_from_double(v);
            crd[u] = make_float2(dv.hi, dv.lo);
        }
        __syncwarp();
    }
    auto psi_node = [&](int t) {
        const int ta = t % nbx1;
        const int tb = (t / nbx1) % nby1;
        const int c = t / (nbx1 * nby1);
        if (!DF) {
            const double x = g.xe[i0 + ta] - xs, y = g.ye[j0 + tb] - ys, z = g.ze[c] - zs;
            P[t] = psi64(x, y, z, x * x, y * y, z * z, g.fn);
        } else {
            const float2 X = crd[ta], Y = crd[nbx1 + tb], Z = crd[nbx1 + nby1 + c];
            const df32 v = psi_df(df_make(X.x, X.y), df_make(Y.x, Y.y), df_make(Z.x, Z.y), Ddf);
            P2[t] = make_float2(v.hi, v.lo);
        }
    };
    int qn = 0;   // queued nodes (warp-uniform)
    for (int t0 = 0; t0 < nnode; t0 += 32) {
        const int t = t0 + lane;
        bool need = false;
        if (t < nnode) {
            const int ia = i0 + t % nbx1;
            const int jb = j0 + (t / nbx1) % nby1;
            const int c = t / (nbx1 * nby1);
            if (ia >= 0 && ia <= g.nx && jb >= 0 && jb <= g.ny && c <= g.nz) {
                const double x = g.xe[ia] - xs, y = g.ye[jb] - ys, z = g.ze[c] - zs;
                need = x * x + y * y + z * z < node_r2;
            }
            if (!need) P[t] = 0.0;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, need);
        if (need) queue[qn + __popc(mask & ((1u << lane) - 1u))] = t;
        qn += __popc(mask);
        __syncwarp();
        if (qn >= 32) {
            psi_node(queue[lane]);
            __syncwarp();
            const int rest = qn - 32;
            const int moved = lane < rest ? queue[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) queue[lane] = moved;
            qn = rest;
            __syncwarp();
        }
    }
    if (lane < qn) psi_node(queue[lane]);
    const float4 S = st32[s];
    const float zf = stz[s].x;
    if (CORNER) {
        // the FP32 corner function at the same nodes, from exactly the FP32
        // coordinates the node-shared FP32 forward uses
        for (int t = lane; t < nnode; t += 32) {
            const int ia = i0 + t % nbx1;
            const int jb = j0 + (t / nbx1) % nby1;
            const int c = t / (nbx1 * nby1);
            float v = 0.0f;
            if (ia >= 0 && ia <= g.nx && jb >= 0 && jb <= g.ny && c <= g.nz) {
                const float dx = (mg.ex[2 * ia] - S.x) + (mg.ex[2 * ia + 1] - S.y);
                const float dy = (mg.ey[2 * jb] - S.z) + (mg.ey[2 * jb + 1] - S.w);
                const float dz = mg.ez[c] - zf;
                v = psi32(dx, dy, dz);
            }
            P32[t] = v;
        }
    }
    __syncwarp();
    const double r2max = (ng.radius_cells * ng.width) * (ng.radius_cells * ng.width);
    const int sxs = 1, sys = nbx1, szs = nbx1 * nby1;
    double dcorr = 0.0;
    const df32 gam_df = df_from_double(kGammaMgal), vol_df = df_from_double(vol_mgal),
               ivol_df = df_from_double(1.0 / vol_mgal);
    for (int t = lane; t < ng.slots; t += 32) {
        const int ai = t % ng.bx;
        const int bj = (t / ng.bx) % ng.by;
        const int l = t / (ng.bx * ng.by);
        const int i = i0 + ai, j = j0 + bj;
        float dgv = 0.0f;
        if (i >= 0 && i < g.nx && j >= 0 && j < g.ny && l < g.nz) {
            const double xc = 0.5 * (g.xe[i] + g.xe[i + 1]) - xs;
            const double yc = 0.5 * (g.ye[j] + g.ye[j + 1]) - ys;
            const double zc = 0.5 * (g.ze[l] + g.ze[l + 1]) - zs;
            if (xc * xc + yc * yc + zc * zc < r2max) {
                const int n0 = ai + sys * bj + szs * l;
                // sigma(n, k) = -(-1)^(da+db+dc) for the vertex (i+da, j+db, l+dc)
                if (!DF) {
                    const double E = -P[n0] + P[n0 + sxs] + P[n0 + sys] - P[n0 + sxs + sys] + P[n0 + szs] -
                                     P[n0 + sxs + szs] - P[n0 + sys + szs] + P[n0 + sxs + sys + szs];
                    const double gex = kGammaMgal * E;
                    double gfar;
                    if (CORNER) {
                        const double E32 = -(double)P32[n0] + (double)P32[n0 + sxs] + (double)P32[n0 + sys] -
                                           (double)P32[n0 + sxs + sys] + (double)P32[n0 + szs] -
                                           (double)P32[n0 + sxs + szs] - (double)P32[n0 + sys + szs] +
                                           (double)P32[n0 + sxs + sys + szs];
                        gfar = kGammaMgal * E32;
                    } else {
                        const float2 X = make_float2(mg.cx[2 * i], mg.cx[2 * i + 1]);
                        const float2 Y = make_float2(mg.cy[2 * j], mg.cy[2 * j + 1]);
                        const float h2 = far_h2(X, Y, S.x, S.y, S.z, S.w);
                        const float ph = far_ph(X, Y, S.x, S.y, S.z, S.w, mg.qa, mg.qb);
                        const float dz = mg.czc[l] - zf;
                        const float R2 = fmaf(dz, dz, h2);
                        gfar = vol_mgal * (double)far_kernel_q(dz, R2, mg.qg, ph);
                    }
                    const double val = gex - gfar;
                    dgv = (float)(val / vol_mgal);
                    dcorr += w2[l] * (gex * gex - gfar * gfar);
                } else {
                    // double-float: neighbouring nodes are differenced first (x,
                    // then the y and z pairs of those), so each subtraction of
                    // nearly equal values is done exactly by TwoSum
                    auto Pd = [&](int n) {
                        const float2 v = P2[n];
                        return df_make(v.x, v.y);
                    };
                    const df32 ex0 = df_sub(Pd(n0 + sxs), Pd(n0));
                    const df32 ex1 = df_sub(Pd(n0 + sxs + sys), Pd(n0 + sys));
                    const df32 ex2 = df_sub(Pd(n0 + sxs + szs), Pd(n0 + szs));
                    const df32 ex3 = df_sub(Pd(n0 + sxs + sys + szs), Pd(n0 + sys + szs));
                    const df32 E = df_sub(df_sub(ex0, ex1), df_sub(ex2, ex3));
                    const df32 gex = df_mul(E, gam_df);
                    const float2 X = make_float2(mg.cx[2 * i], mg.cx[2 * i + 1]);
                    const float2 Y = make_float2(mg.cy[2 * j], mg.cy[2 * j + 1]);
                    const float h2 = far_h2(X, Y, S.x, S.y, S.z, S.w);
                    const float ph = far_ph(X, Y, S.x, S.y, S.z, S.w, mg.qa, mg.qb);
                    const float dz = mg.czc[l] - zf;
                    const float R2 = fmaf(dz, dz, h2);
                    const df32 gfar = df_mulf(vol_df, far_kernel_q(dz, R2, mg.qg, ph));
                    const df32 v = df_sub(gex, gfar);
                    dgv = df_mul(v, ivol_df).hi;
                    // gex^2 - gfar^2 = (gex - gfar)(gex + gfar)
                    dcorr += w2[l] * (double)(v.hi * (gex.hi + gfar.hi));
                }
            }
        }
        // formed in double-float (or FP64), stored in FP32 per unit q = gamma V rho
        // (so the products use the FP32 q of the far field); relative rounding 6e-8
        dG[s * ng.ld + t] = dgv;
    }
    if (lane < ng.ld - ng.slots) dG[s * ng.ld + ng.slots + lane] = 0.0f;   // row padding
    dcorr = warp_sum(dcorr);
    if (lane == 0) {
        diag_corr[s] = dcorr;
        st_i0[s] = i0;
        st_j0[s] = j0;
        const bool hit = (i0 <= g.nx - 1) && (i0 + ng.bx - 1 >= 0) && (j0 <= g.ny - 1) && (j0 + ng.by - 1 >= 0);
        keys[s] = hit ? (unsigned)((i0 + ng.bx - 1) + ng.nbx * (j0 + ng.by - 1)) : key_sentinel;
        vals[s] = (int)s;
    }
}

// bin_start[b] = first position p with key_sorted[p] >= b, b in [0, nbins]
__global__ void k_bin_bounds(const unsigned *__restrict__ ks, int64_t n, int nbins, int *__restrict__ bin_start) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nbins; b += gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (ks[mid] < (unsigned)b) lo = mid + 1; else hi = mid;
        }
        bin_start[b] = (int)lo;
    }
}

// corr[s] = sum_slots dGq[s][slot] * q[cell(s, slot)]   (warp per station),
// q = gamma V rho in FP32 (the far field's values, in natural cell order).  Slot
// t = a + bx (bj + by l); each lane walks t = lane, lane + 32, ... with
// (a, bj, l) stepped incrementally (no divisions in the loop), four slots per
// step so that their loads are independent.  Products and runs of 16 terms
// are FP32 (FMA pipe), folded into an FP64 sum: the FP64 pipe (1/64 of the
// FP32 rate on this GPU) does one addition per 16 terms instead of one FMA
// per term.
//
// Stations whose box lies inside the mesh (all but those near its edges) take
// a fast path: the table row (padded to a multiple of 4 floats) is prefetched
// into L2 whole and streams in 16-byte loads (read once, evict-first), the
// cell of each slot comes from the plan's slot-offset table
// off[t] = a + nx (bj + ny l) (L1-resident), and no slot needs a bounds check.
__global__ void __launch_bounds__(256) k_near_fwd(int nx, int ny, int nz, NearGeo ng, int64_t N,
                                                  const float *__restrict__ dG, const int *__restrict__ st_i0,
                                                  const int *__restrict__ st_j0, const int *__restrict__ off,
                                                  const float *__restrict__ qn, double *__restrict__ corr) {
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= N) return;
    const int i0 = st_i0[s], j0 = st_j0[s];
    const float *gs = dG + s * ng.ld;
    if (i0 >= 0 && i0 + ng.bx <= nx && j0 >= 0 && j0 + ng.by <= ny && ng.bz <= nz) {
        // padded slots hold dG = 0 and offset 0 (the box origin, inside the mesh)
        const float4 *g4 = reinterpret_cast<const float4 *>(gs);
        const int4 *o4 = reinterpret_cast<const int4 *>(off);
        const float *qb = qn + i0 + (int64_t)nx * j0;
        const int n4 = ng.ld >> 2;
        // the whole row requested at once: the loop's loads then hit L2
        if (lane == 0) prefetch_l2_bulk(gs, 4u * (uint32_t)ng.ld);
        double acc = 0.0;
        for (int v = lane; v < n4; v += 64) {   // 8 slots per lane and step, loads issued together
            const bool two = v + 32 < n4;
            const float4 G0 = __ldcs(g4 + v);
            const int4 O0 = __ldg(o4 + v);
            const float4 G1 = two ? __ldcs(g4 + v + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
            const int4 O1 = two ? __ldg(o4 + v + 32) : make_int4(0, 0, 0, 0);
            const float q0 = qb[O0.x], q1 = qb[O0.y], q2 = qb[O0.z], q3 = qb[O0.w];
            const float q4 = qb[O1.x], q5 = qb[O1.y], q6 = qb[O1.z], q7 = qb[O1.w];
            float accf = G0.x * q0;
            accf = fmaf(G0.y, q1, accf);
            accf = fmaf(G0.z, q2, accf);
            accf = fmaf(G0.w, q3, accf);
            accf = fmaf(G1.x, q4, accf);
            accf = fmaf(G1.y, q5, accf);
            accf = fmaf(G1.z, q6, accf);
            accf = fmaf(G1.w, q7, accf);
            acc += (double)accf;   // FP32 runs of 8 terms folded into FP64
        }
        const double v = warp_sum(acc);
        if (lane == 0) corr[s] = v;
        return;
    }
    const int qa = 32 % ng.bx, qr = 32 / ng.bx;
    int a = lane % ng.bx;
    const int r0 = lane / ng.bx;
    int bj = r0 % ng.by, l = r0 / ng.by;
    auto step = [&](int &a_, int &bj_, int &l_) {
        a_ += qa;
        int carry = qr;
        if (a_ >= ng.bx) {
            a_ -= ng.bx;
            ++carry;
        }
        bj_ += carry;
        while (bj_ >= ng.by) {
            bj_ -= ng.by;
            ++l_;
        }
    };
    double acc = 0.0;
    float accf = 0.0f;
    int run = 0;
    for (int t = lane; t < ng.slots; t += 128) {
        float g[4], q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + a, j = j0 + bj;
            const bool ok = t + 32 * u < ng.slots && i >= 0 && i < nx && j >= 0 && j < ny && l < nz;
            g[u] = ok ? gs[t + 32 * u] : 0.0f;
            q[u] = ok ? qn[i + (int64_t)nx * (j + (int64_t)ny * l)] : 0.0f;
            step(a, bj, l);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) accf = fmaf(g[u], q[u], accf);
        if (++run == 4) {   // fold every 16 terms
            acc += (double)accf;
            accf = 0.0f;
            run = 0;
        }
    }
    acc += (double)accf;
    const double v = warp_sum(acc);
    if (lane == 0) corr[s] = v;
}

// out[k] = sum over stations whose window box holds cell k of dG * r, for the
// top bz layers.  A warp owns 32 consecutive cells of one row (y) and layer;
// the stations whose box covers row y have box-origin bins in bin rows
// y-by+1 .. y, and within one bin row the bins of the 32 columns are
// consecutive keys, i.e. one contiguous range of the sorted station list.  For
// each such station the lanes read one box row of dG (consecutive slots:
// coalesced).  Stations are fetched eight at a time (independent loads) and
// accumulated in (bin row, bin, station) order: deterministic.
__global__ void __launch_bounds__(256, 4) k_near_adj(int nx, int ny, NearGeo ng, const float *__restrict__ dG,
                                                  const int *__restrict__ bin_start, const int *__restrict__ bin_st,
                                                  const int *__restrict__ st_i0, const float2 *__restrict__ stz,
                                                  double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int l = blockIdx.z;
    if (y >= ny) return;   // warp-uniform
    const int tx0 = blockIdx.x * 32;
    const int x = tx0 + lane;
    const bool xin = x < nx;
    // shifted bin coordinates: sbi = i0 + bx - 1, sbj = j0 + by - 1
    const int sbi_lo = tx0;
    const int sbi_hi = min(ng.nbx - 1, tx0 + 31 + ng.bx - 1);
    double acc = 0.0;
    for (int sbj = y; sbj <= y + ng.by - 1; ++sbj) {
        const int b = y - (sbj - (ng.by - 1));   // row of the cell inside the station's box
        const int p0 = bin_start[sbi_lo + ng.nbx * sbj];
        const int p1 = bin_start[sbi_hi + ng.nbx * sbj + 1];
        const int64_t row = (int64_t)ng.bx * (b + (int64_t)ng.by * l);
        // runs of up to 8 stations in FP32 (r as the FP32 copy in stz.y), folded
        // into FP64; the run's loads are issued together (independent)
        for (int p = p0; p < p1; p += 8) {
            int sv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) sv[u] = (p + u < p1) ? bin_st[p + u] : -1;
            float g[8], rv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int a = sv[u] >= 0 ? x - st_i0[sv[u]] : -1;
                const bool ok = a >= 0 && a < ng.bx && xin;
                g[u] = ok ? dG[(int64_t)sv[u] * ng.ld + row + a] : 0.0f;
                rv[u] = ok ? stz[sv[u]].y : 0.0f;
            }
            float accf = 0.0f;
#pragma unroll
            for (int u = 0; u < 8; ++u) accf = fmaf(g[u], rv[u], accf);
            acc += (double)accf;
        }
    }
    if (xin) out[x + (int64_t)nx * (y + (int64_t)ny * l)] = acc;
}

// Near-field adjoint, station-streaming form (the default when its shared
// memory fits).  out[k] = sum over stations s whose window box holds cell k of
// dG[s][slot(s, k)] * r_s, for the top lz layers.
//
// CTA = tile of kNaTile x kNaTile station bins (box origins i0, j0); the boxes
// of its stations cover a region of RX x RY x lz cells, RX = kNaTile + bx - 1.
// Each station's table row (ld floats, contiguous, 16-byte padded) is copied
// whole into shared memory by one 1D TMA bulk copy through an ns-stage ring
// completed on mbarriers, so the table is read from HBM exactly once and in
// full rows (the cell-tiled form below reads box rows of 17 floats split over
// 32-column tiles and fetches about twice the table).  Thread t owns slots
// t, t + 256, ...: slot u of station s adds dG * r into region cell
// base(s) + roff[u].  The slots of one station map to distinct cells and a
// barrier separates consecutive stations, so every cell receives its terms in
// station order (bitwise deterministic).  Terms are summed in FP32 in shared
// memory and folded every kNaFold stations into the CTA's FP64 region sums,
// tpart[tile] in global memory (a cell sees at most kNaFold FP32 terms
// between folds); k_near_adj_gather adds, per cell, the tiles whose region
// holds it, in tile order.
constexpr int kNaTile = 8;
constexpr int kNaThreads = 256;
constexpr int kNaFold = 16;
constexpr int kNaMaxStages = 12;
constexpr size_t kNaSmemBudget = 74 * 1024;    // three CTAs per SM
static_assert(8 * kNaMaxStages + 8 <= 128 && 128 + 4 * (2 * kNaTile + 1) <= 256, "near adjoint header");

constexpr int kNaMeta = 256;     // station metadata ring (prefetched 128 stations ahead)

constexpr int kNaMaxKs = 20;      // slots per thread the streaming form handles (rows up to 5120 floats)

struct NearAdjShape {
    bool ok = false;
    int RX = 0, RY = 0, lz = 0, RC = 0, ns = 0, ntx = 0, nty = 0, ks = 0;
    size_t o_sb = 0, o_meta = 0, o_acc32 = 0, o_stage = 0, smem = 0;
};

static NearAdjShape near_adj_shape(const grav_plan *p) {
    NearAdjShape z;
    z.RX = kNaTile + p->ng.bx - 1;
    z.RY = kNaTile + p->ng.by - 1;
    z.lz = std::min(p->ng.bz, p->nz);
    z.RC = z.RX * z.RY * z.lz;
    z.ntx = (p->ng.nbx + kNaTile - 1) / kNaTile;
    z.nty = (p->ng.nby + kNaTile - 1) / kNaTile;
    z.o_sb = 256;                                             // after the header: mbarriers, flags, row table
    z.o_meta = z.o_sb + 2ull * 4 * kNaMaxStages;              // sbase[], srv[]
    z.o_acc32 = z.o_meta + 3ull * 4 * kNaMeta;                // station ring: index, base, r
    z.o_stage = align_up(z.o_acc32 + 4ull * z.RC, 128);
    const size_t row = 4ull * p->ng.ld;
    const int ns = z.o_stage + 2 * row <= kNaSmemBudget ? (int)((kNaSmemBudget - z.o_stage) / row) : 0;
    z.ns = std::min(ns, kNaMaxStages);
    z.smem = z.o_stage + (size_t)z.ns * row;
    const int need = (p->ng.ld + kNaThreads - 1) / kNaThreads;
    z.ks = need <= 4 ? 4 : need <= 8 ? 8 : need <= 12 ? 12 : need <= 16 ? 16 : kNaMaxKs;
    z.ok = z.ns >= 2 && p->ng.ld % 4 == 0 && need <= kNaMaxKs;
    return z;
}

template <int KS>
__global__ void __launch_bounds__(kNaThreads) k_near_adj_rows(
    NearGeo ng, int RX, int RY, int lz, int ns, int ntx, uint32_t o_sb, uint32_t o_meta,
    uint32_t o_acc32, uint32_t o_stage, const float *__restrict__ dG, const int *__restrict__ bin_start,
    const int *__restrict__ bin_st, const int *__restrict__ st_i0, const int *__restrict__ st_j0,
    const float2 *__restrict__ stz, double *__restrict__ tpart, int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // header (256 bytes): mbarriers [0, 96), flags [96, 104), row table [128, 196)
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);                      // [ns], ns <= 12
    volatile int *flag = reinterpret_cast<volatile int *>(smem_raw + 8 * kNaMaxStages);   // [2]
    int *rowinfo = reinterpret_cast<int *>(smem_raw + 128);                       // [2 kNaTile + 1]
    int *sbase = reinterpret_cast<int *>(smem_raw + o_sb);
    float *srv = reinterpret_cast<float *>(smem_raw + o_sb + 4 * kNaMaxStages);
    int *msidx = reinterpret_cast<int *>(smem_raw + o_meta);          // [kNaMeta]
    int *mbase = msidx + kNaMeta;                                      // [kNaMeta]
    float *mrv = reinterpret_cast<float *>(mbase + kNaMeta);          // [kNaMeta]
    float *acc32 = reinterpret_cast<float *>(smem_raw + o_acc32);
    float *stage = reinterpret_cast<float *>(smem_raw + o_stage);
    const int tid = threadIdx.x;
    const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    const int I0 = tx * kNaTile, J0 = ty * kNaTile;
    const int RC = RX * RY * lz;

    // this thread's slots u = tid + 256 k: u = a + bx (b + by l) -> region
    // offset a + RX (b + RY l), kept in registers; padding and layers below
    // the mesh (l >= lz) take no cell (-1)
    int ro[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int u = tid + kNaThreads * k;
        int v = -1;
        if (u < ng.slots) {
            const int a = u % ng.bx, b = (u / ng.bx) % ng.by, l = u / (ng.bx * ng.by);
            if (l < lz) v = a + RX * (b + RY * l);
        }
        ro[k] = v;
    }
    // the CTA's FP64 region sums live in its own block of tpart (L2-resident);
    // thread t alone folds into cells t, t + 256, ..., so the order is fixed
    double *acc64 = tpart + (size_t)blockIdx.x * RC;
    for (int c = tid; c < RC; c += kNaThreads) {
        acc32[c] = 0.0f;
        acc64[c] = 0.0;
    }
    // station ranges of the tile's bin rows: rowinfo[r] = first position in
    // bin_st, rowinfo[kNaTile + 1 + r] = stations before row r (prefix)
    if (tid == 0) {
        int q = 0;
        const int i1 = min(I0 + kNaTile, ng.nbx);
        for (int r = 0; r < kNaTile; ++r) {
            const int sbj = J0 + r;
            int p0 = 0, p1 = 0;
            if (sbj < ng.nby) {
                p0 = bin_start[I0 + ng.nbx * sbj];
                p1 = bin_start[i1 + ng.nbx * sbj];
            }
            rowinfo[r] = p0;
            rowinfo[kNaTile + r] = q;
            q += p1 - p0;
        }
        rowinfo[2 * kNaTile] = q;
        for (int k = 0; k < ns; ++k) mbar_init(&full[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int Q = rowinfo[2 * kNaTile];
    const uint32_t row_bytes = 4u * (uint32_t)ng.ld;

    // station metadata (table row, region base, FP32 r) for stations [u0, u1),
    // into ring slot u % kNaMeta, one station per thread: the dependent global
    // loads run in parallel and ahead of the copies that need them
    auto fetch_meta = [&](int u0, int u1) {
        const int u = u0 + tid;
        if (u < u1) {
            int r = 0;
            while (r + 1 < kNaTile && rowinfo[kNaTile + r + 1] <= u) ++r;
            const int sidx = bin_st[rowinfo[r] + (u - rowinfo[kNaTile + r])];
            const int ri = st_i0[sidx] + ng.bx - 1 - I0;
            const int rj = st_j0[sidx] + ng.by - 1 - J0;
            const int slot = u % kNaMeta;
            msidx[slot] = sidx;
            mbase[slot] = (ri >= 0 && ri < kNaTile && rj >= 0 && rj < kNaTile) ? ri + RX * rj : -1;
            mrv[slot] = stz[sidx].y;
        }
    };
    // thread 0: station q's row into stage q % ns, with its region base and r
    auto issue = [&](int q) {
        const int k = q % ns, slot = q % kNaMeta;
        const int sidx = msidx[slot];
        sbase[k] = mbase[slot];
        srv[k] = mrv[slot];
        mbar_arrive_expect_tx(&full[k], row_bytes);
        tma_load_1d(stage + (size_t)k * ng.ld, dG + (int64_t)sidx * ng.ld, row_bytes, &full[k]);
    };
    static_assert(kNaMeta == kNaThreads, "one metadata slot per thread");
    auto fetch_meta_half = [&](int u0, int u1) {
        if (tid < kNaMeta / 2) fetch_meta(u0, u1);
    };
    fetch_meta(0, min(Q, kNaMeta));
    __syncthreads();
    if (tid == 0)
        for (int q = 0; q < min(Q, ns); ++q) issue(q);

    for (int q = 0; q < Q; ++q) {
        const int k = q % ns;
        if (tid == 0) flag[q & 1] = mbar_wait_spin_bounded(&full[k], (uint32_t)((q / ns) & 1)) ? 1 : 0;
        __syncthreads();   // also orders station q-1's shared-memory sums before station q's
        if (!flag[q & 1]) {
            if (tid == 0) {
                set_status(status, kStatusMbarTimeout);
                for (int u = q + 1; u < min(Q, max(q - 1 + ns, ns)); ++u)   // copies still in flight
                    (void)mbar_wait_bounded(&full[u % ns], (uint32_t)((u / ns) & 1));
            }
            return;
        }
        if (tid == 0 && q >= 1 && q - 1 + ns < Q) {   // stage (q-1) % ns was read before the barrier
            fence_proxy_async_smem();
            issue(q - 1 + ns);
        }
        // refill half of the metadata ring: slots of stations [q + 128, q + 256) held
        // stations [q - 128, q), all issued (ns <= 12); read after >= 1 more barrier
        if (q % (kNaMeta / 2) == 0 && q > 0) fetch_meta_half(q + kNaMeta / 2, min(Q, q + kNaMeta));
        const int base = sbase[k];
        const float rv = srv[k];
        if (base >= 0 && rv != 0.0f) {
            // a station's slots are distinct cells: all loads first, then the
            // stores (independent, so their latencies overlap)
            const float *gr = stage + (size_t)k * ng.ld + tid;
            float gv[KS], av[KS];
#pragma unroll
            for (int j = 0; j < KS; ++j) gv[j] = ro[j] >= 0 ? gr[kNaThreads * j] : 0.0f;
#pragma unroll
            for (int j = 0; j < KS; ++j) av[j] = ro[j] >= 0 ? acc32[base + ro[j]] : 0.0f;
#pragma unroll
            for (int j = 0; j < KS; ++j)
                if (ro[j] >= 0) acc32[base + ro[j]] = fmaf(gv[j], rv, av[j]);
        }
        if ((q + 1) % kNaFold == 0 || q + 1 == Q) {
            __syncthreads();
            for (int c = tid; c < RC; c += kNaThreads) {
                acc64[c] += (double)acc32[c];
                acc32[c] = 0.0f;
            }
        }
    }
}

// Near-field adjoint, warp-private form (the default when its shared memory
// fits).  CTA = tile of kNwTile x kNwTile station bins, region of RX x RY x lz
// cells (RX = kNwTile + bx - 1); each of the 8 warps owns a private FP32
// accumulator over the whole region and takes stations w, w + 8, ... of the
// tile in order.  A warp requests its station's table row (ld floats,
// contiguous) and its next station's row from L2 by bulk prefetch, streams
// the row with 16-byte evict-first loads, kNwChunk per lane in flight,
// and adds dG * r into its own accumulator (one station's slots are distinct
// cells, so no lane races another; no other warp touches this accumulator, so
// no barrier separates stations).  Every kNwPass stations per warp the eight
// accumulators are summed cell by cell in warp order (FP32) and added into
// the tile's FP64 region sums in global memory (tpart[tile], the same
// per-tile layout k_near_adj_gather reads; the first pass writes them), then
// cleared: bitwise deterministic, at most 8 kNwPass FP32 terms per cell
// between FP64 folds.
// The table is read once, in whole rows, with no per-station barrier.
constexpr int kNwTile = 4;
constexpr int kNwWarps = 8;
constexpr int kNwPass = 16;
constexpr int kNwChunk = 8;
constexpr size_t kNwSmemBudget = 112 * 1024;   // two CTAs per SM

struct NearWarpShape {
    bool ok = false;
    int RX = 0, RY = 0, lz = 0, RC = 0, ntx = 0, nty = 0;
    size_t o_meta = 0, o_roff = 0, o_acc = 0, smem = 0;
};

static NearWarpShape near_warp_shape(const grav_plan *p) {
    NearWarpShape z;
    z.RX = kNwTile + p->ng.bx - 1;
    z.RY = kNwTile + p->ng.by - 1;
    z.lz = std::min(p->ng.bz, p->nz);
    z.RC = z.RX * z.RY * z.lz;
    z.ntx = (p->ng.nbx + kNwTile - 1) / kNwTile;
    z.nty = (p->ng.nby + kNwTile - 1) / kNwTile;
    z.o_meta = 128;                                             // header: row table [2 kNwTile + 1]
    z.o_roff = z.o_meta + 3ull * 4 * kNwWarps * kNwPass;        // a pass's stations: row, base, r
    z.o_acc = align_up(z.o_roff + 4ull * p->ng.ld, 16);        // roff[ld]
    z.smem = z.o_acc + 4ull * kNwWarps * z.RC;                 // kNwWarps private accumulators
    z.ok = z.smem <= kNwSmemBudget && p->ng.ld % 4 == 0;
    return z;
}

__global__ void __launch_bounds__(kNwWarps * 32, 2) k_near_adj_warp(
    NearGeo ng, int RX, int RY, int lz, int ntx, uint32_t o_meta, uint32_t o_roff, uint32_t o_acc,
    const float *__restrict__ dG,
    const int *__restrict__ bin_start, const int *__restrict__ bin_st, const int *__restrict__ st_i0,
    const int *__restrict__ st_j0, const float2 *__restrict__ stz, double *__restrict__ tpart) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int *rowinfo = reinterpret_cast<int *>(smem_raw);                  // [2 kNwTile + 1]
    int *msidx = reinterpret_cast<int *>(smem_raw + o_meta);           // [kNwWarps kNwPass]
    int *mbase = msidx + kNwWarps * kNwPass;
    float *mrv = reinterpret_cast<float *>(mbase + kNwWarps * kNwPass);
    int *roff = reinterpret_cast<int *>(smem_raw + o_roff);
    float *acc_all = reinterpret_cast<float *>(smem_raw + o_acc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    const int I0 = tx * kNwTile, J0 = ty * kNwTile;
    const int RC = RX * RY * lz;
    float *accw = acc_all + (size_t)warp * RC;
    double *acc64 = tpart + (size_t)blockIdx.x * RC;
    for (int u = tid; u < ng.ld; u += kNwWarps * 32) {
        int v = -1;
        if (u < ng.slots) {
            const int a = u % ng.bx, b = (u / ng.bx) % ng.by, l = u / (ng.bx * ng.by);
            if (l < lz) v = a + RX * (b + RY * l);
        }
        roff[u] = v;
    }
    for (int c = tid; c < kNwWarps * RC; c += kNwWarps * 32) acc_all[c] = 0.0f;
    if (tid == 0) {
        int q = 0;
        const int i1 = min(I0 + kNwTile, ng.nbx);
        for (int r = 0; r < kNwTile; ++r) {
            const int sbj = J0 + r;
            int p0 = 0, p1 = 0;
            if (sbj < ng.nby) {
                p0 = bin_start[I0 + ng.nbx * sbj];
                p1 = bin_start[i1 + ng.nbx * sbj];
            }
            rowinfo[r] = p0;
            rowinfo[kNwTile + r] = q;
            q += p1 - p0;
        }
        rowinfo[2 * kNwTile] = q;
    }
    __syncthreads();
    const int Q = rowinfo[2 * kNwTile];
    if (Q == 0)   // otherwise the first pass writes the region sums
        for (int c = tid; c < RC; c += kNwWarps * 32) acc64[c] = 0.0;
    const int n4 = ng.ld >> 2;
    const float4 *dG4 = reinterpret_cast<const float4 *>(dG);
    const int4 *roff4 = reinterpret_cast<const int4 *>(roff);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int pass0 = 0; pass0 < Q; pass0 += kNwWarps * kNwPass) {
        const int pass1 = min(Q, pass0 + kNwWarps * kNwPass);
        // the pass's station metadata, one station per thread (the dependent
        // loads run in parallel instead of once per station and warp)
        if (tid < kNwWarps * kNwPass && pass0 + tid < pass1) {
            const int q = pass0 + tid;
            int r = 0;
            while (r + 1 < kNwTile && rowinfo[kNwTile + r + 1] <= q) ++r;
            const int sidx = bin_st[rowinfo[r] + (q - rowinfo[kNwTile + r])];
            const int ri = st_i0[sidx] + ng.bx - 1 - I0;
            const int rj = st_j0[sidx] + ng.by - 1 - J0;
            const float rv = stz[sidx].y;
            msidx[tid] = sidx;
            mbase[tid] = (ri >= 0 && ri < kNwTile && rj >= 0 && rj < kNwTile && rv != 0.0f) ? ri + RX * rj : -1;
            mrv[tid] = rv;
        }
        __syncthreads();
        int pf_q = -1;
        for (int q = pass0 + warp; q < pass1; q += kNwWarps) {
            const int base = mbase[q - pass0];
            if (base < 0) continue;   // warp-uniform
            const int sidx = msidx[q - pass0];
            const float rv = mrv[q - pass0];
            float *acc = accw + base;
            const float4 *row = dG4 + (int64_t)sidx * n4;
            // this row (unless requested one station earlier) and the row of
            // the warp's next station, each requested whole
            const int qnext = q + kNwWarps;
            const bool pf_next = qnext < pass1 && mbase[qnext - pass0] >= 0;
            if (lane == 0) {
                if (pf_q != q) prefetch_l2_bulk(row, 16u * (uint32_t)n4);
                if (pf_next) prefetch_l2_bulk(dG4 + (int64_t)msidx[qnext - pass0] * n4, 16u * (uint32_t)n4);
            }
            pf_q = pf_next ? qnext : -1;
            for (int v0 = 0; v0 < n4; v0 += 32 * kNwChunk) {
                float4 gq[kNwChunk];
#pragma unroll
                for (int c = 0; c < kNwChunk; ++c) {
                    const int v = v0 + lane + 32 * c;
                    gq[c] = v < n4 ? __ldcs(row + v) : zero4;
                }
                int4 oq[kNwChunk];
#pragma unroll
                for (int c = 0; c < kNwChunk; ++c) {
                    const int v = v0 + lane + 32 * c;
                    oq[c] = v < n4 ? roff4[v] : make_int4(-1, -1, -1, -1);
                }
                // a station's slots are distinct cells: all accumulator loads,
                // then all stores (independent, so their latencies overlap)
                float av[4 * kNwChunk];
#pragma unroll
                for (int c = 0; c < kNwChunk; ++c) {
                    av[4 * c + 0] = oq[c].x >= 0 ? acc[oq[c].x] : 0.0f;
                    av[4 * c + 1] = oq[c].y >= 0 ? acc[oq[c].y] : 0.0f;
                    av[4 * c + 2] = oq[c].z >= 0 ? acc[oq[c].z] : 0.0f;
                    av[4 * c + 3] = oq[c].w >= 0 ? acc[oq[c].w] : 0.0f;
                }
#pragma unroll
                for (int c = 0; c < kNwChunk; ++c) {
                    if (oq[c].x >= 0) acc[oq[c].x] = fmaf(gq[c].x, rv, av[4 * c + 0]);
                    if (oq[c].y >= 0) acc[oq[c].y] = fmaf(gq[c].y, rv, av[4 * c + 1]);
                    if (oq[c].z >= 0) acc[oq[c].z] = fmaf(gq[c].z, rv, av[4 * c + 2]);
                    if (oq[c].w >= 0) acc[oq[c].w] = fmaf(gq[c].w, rv, av[4 * c + 3]);
                }
            }
            __syncwarp();   // the next station's lanes read cells these lanes wrote
        }
        __syncthreads();
        for (int c = tid; c < RC; c += kNwWarps * 32) {
            float t = 0.0f;
#pragma unroll
            for (int w = 0; w < kNwWarps; ++w) {
                t += acc_all[(size_t)w * RC + c];
                acc_all[(size_t)w * RC + c] = 0.0f;
            }
            acc64[c] = pass0 == 0 ? (double)t : acc64[c] + (double)t;
        }
        __syncthreads();
    }
}

// Near-field adjoint, layer-split form (the default when its shared memory
// fits).  CTA = tile of kNwTile x kNwTile station bins with one FP32
// accumulator over its region (RX x RY x lz cells), as in k_near_adj_warp,
// but warp w owns the region's layers w, w + W, ... (W = min(lz, 8) warps):
// a station's slots in layer l only touch region layer l, so the warps never
// share a cell and need no private copies (8x less shared memory, several
// CTAs per SM).  Every warp walks all of the tile's stations in order and,
// for each, streams the contiguous bx*by-float segment of its layer in the
// station's table row (lane-consecutive slots, evict-first, the next
// station's segment prefetched into L2) into its planes.  Every kNlPass
// stations each warp adds its FP32 planes into the tile's FP64 region sums
// in global memory (the first pass writes them; same layout as
// k_near_adj_warp, read by k_near_adj_gather) and clears them: each cell sees
// its stations in tile order, at most kNlPass FP32 terms between FP64 folds,
// bitwise deterministic.
constexpr int kNlPass = 128;
constexpr int kNlUnroll = 10;   // slots per lane in flight (bx*by = 289 at the default window)
constexpr size_t kNlSmemBudget = 64 * 1024;

struct NearLayerShape {
    bool ok = false;
    int RX = 0, RY = 0, SX = 0, lz = 0, RC = 0, ntx = 0, nty = 0, nwarps = 0;
    size_t o_meta = 0, o_roff = 0, o_acc = 0, smem = 0;
};

static NearLayerShape near_layer_shape(const grav_plan *p) {
    NearLayerShape z;
    z.RX = kNwTile + p->ng.bx - 1;
    z.RY = kNwTile + p->ng.by - 1;
    z.lz = std::min(p->ng.bz, p->nz);
    z.RC = z.RX * z.RY * z.lz;
    z.ntx = (p->ng.nbx + kNwTile - 1) / kNwTile;
    z.nty = (p->ng.nby + kNwTile - 1) / kNwTile;
    z.nwarps = std::min(z.lz, 8);
    z.o_meta = 128;                                              // header: row table [2 kNwTile + 1]
    z.o_roff = z.o_meta + 3ull * 4 * kNlPass;                    // a pass's stations: index, base, r
    z.o_acc = align_up(z.o_roff + 4ull * p->ng.bx * p->ng.by, 16);   // in-layer slot -> region offset
    // shared-memory row stride SX = bx (mod 32): 32 consecutive slots of a
    // layer then fall on 32 distinct banks; RX when the padded planes do not fit
    z.SX = z.RX + ((p->ng.bx - z.RX) % 32 + 32) % 32;
    if (z.o_acc + 4ull * z.SX * z.RY * z.lz > kNlSmemBudget) z.SX = z.RX;
    z.smem = z.o_acc + 4ull * z.SX * z.RY * z.lz;               // FP32 accumulator over the region
    z.ok = z.smem <= kNlSmemBudget;
    return z;
}

__global__ void __launch_bounds__(256) k_near_adj_layer(
    NearGeo ng, int RX, int RY, int SX, int lz, int ntx, uint32_t o_meta, uint32_t o_roff, uint32_t o_acc,
    const float *__restrict__ dG, const int *__restrict__ bin_start, const int *__restrict__ bin_st,
    const int *__restrict__ st_i0, const int *__restrict__ st_j0, const float2 *__restrict__ stz,
    double *__restrict__ tpart) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int *rowinfo = reinterpret_cast<int *>(smem_raw);                  // [2 kNwTile + 1]
    int *msidx = reinterpret_cast<int *>(smem_raw + o_meta);           // [kNlPass]
    int *mbase = msidx + kNlPass;
    float *mrv = reinterpret_cast<float *>(mbase + kNlPass);
    int *roff = reinterpret_cast<int *>(smem_raw + o_roff);
    float *acc = reinterpret_cast<float *>(smem_raw + o_acc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x, nw = nthr >> 5;
    const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    const int I0 = tx * kNwTile, J0 = ty * kNwTile;
    const int plane = RX * RY, RC = plane * lz, bxy = ng.bx * ng.by;
    const int splane = SX * RY;   // a layer in shared memory (rows of SX >= RX)
    double *acc64 = tpart + (size_t)blockIdx.x * RC;
    for (int u = tid; u < bxy; u += nthr) roff[u] = u % ng.bx + SX * (u / ng.bx);
    for (int c = tid; c < splane * lz; c += nthr) acc[c] = 0.0f;
    if (tid == 0) {
        int q = 0;
        const int i1 = min(I0 + kNwTile, ng.nbx);
        for (int r = 0; r < kNwTile; ++r) {
            const int sbj = J0 + r;
            int p0 = 0, p1 = 0;
            if (sbj < ng.nby) {
                p0 = bin_start[I0 + ng.nbx * sbj];
                p1 = bin_start[i1 + ng.nbx * sbj];
            }
            rowinfo[r] = p0;
            rowinfo[kNwTile + r] = q;
            q += p1 - p0;
        }
        rowinfo[2 * kNwTile] = q;
    }
    __syncthreads();
    const int Q = rowinfo[2 * kNwTile];
    if (Q == 0)   // otherwise the first pass writes the region sums
        for (int c = tid; c < RC; c += nthr) acc64[c] = 0.0;
    for (int pass0 = 0; pass0 < Q; pass0 += kNlPass) {
        const int pass1 = min(Q, pass0 + kNlPass);
        for (int t = tid; t < pass1 - pass0; t += nthr) {
            const int q = pass0 + t;
            int r = 0;
            while (r + 1 < kNwTile && rowinfo[kNwTile + r + 1] <= q) ++r;
            const int sidx = bin_st[rowinfo[r] + (q - rowinfo[kNwTile + r])];
            const int ri = st_i0[sidx] + ng.bx - 1 - I0;
            const int rj = st_j0[sidx] + ng.by - 1 - J0;
            const float rv = stz[sidx].y;
            msidx[t] = sidx;
            mbase[t] = (ri >= 0 && ri < kNwTile && rj >= 0 && rj < kNwTile && rv != 0.0f) ? ri + SX * rj : -1;
            mrv[t] = rv;
        }
        __syncthreads();
        for (int l = warp; l < lz; l += nw) {
            float *accl = acc + (size_t)l * splane;
            // [lo16, hi16): this layer's segment of a row, widened to 16-byte bounds
            const uint32_t lo16 = (4u * (uint32_t)(l * bxy)) & ~15u;
            const uint32_t hi16 = (4u * (uint32_t)((l + 1) * bxy) + 15u) & ~15u;
            for (int q = 0; q < pass1 - pass0; ++q) {
                const int base = mbase[q];
                if (base < 0) continue;   // warp-uniform
                const float rv = mrv[q];
                const float *seg = dG + (int64_t)msidx[q] * ng.ld + (int64_t)l * bxy;
                if (lane == 0) {
                    if (q == 0) prefetch_l2_bulk(reinterpret_cast<const char *>(dG + (int64_t)msidx[q] * ng.ld) + lo16,
                                                 hi16 - lo16);
                    if (q + 1 < pass1 - pass0 && mbase[q + 1] >= 0)
                        prefetch_l2_bulk(reinterpret_cast<const char *>(dG + (int64_t)msidx[q + 1] * ng.ld) + lo16,
                                         hi16 - lo16);
                }
                float *a = accl + base;
                for (int t0 = 0; t0 < bxy; t0 += 32 * kNlUnroll) {
                    float gv[kNlUnroll];
                    int ov[kNlUnroll];
#pragma unroll
                    for (int u = 0; u < kNlUnroll; ++u) {
                        const int t = t0 + lane + 32 * u;
                        gv[u] = t < bxy ? __ldcs(seg + t) : 0.0f;
                        ov[u] = t < bxy ? roff[t] : -1;
                    }
                    float av[kNlUnroll];
#pragma unroll
                    for (int u = 0; u < kNlUnroll; ++u) av[u] = ov[u] >= 0 ? a[ov[u]] : 0.0f;
#pragma unroll
                    for (int u = 0; u < kNlUnroll; ++u)
                        if (ov[u] >= 0) a[ov[u]] = fmaf(gv[u], rv, av[u]);
                }
                __syncwarp();   // the next station's lanes read cells these lanes wrote
            }
            double *p64 = acc64 + (size_t)l * plane;
            for (int c = lane; c < plane; c += 32) {
                const int sc = c % RX + SX * (c / RX);
                p64[c] = pass0 == 0 ? (double)accl[sc] : p64[c] + (double)accl[sc];
                accl[sc] = 0.0f;
            }
            __syncwarp();
        }
        __syncthreads();   // the metadata is rewritten by the next pass
    }
}

// Near-field forward, tile form (the default when its shared memory fits):
// corr[s] = sum over slots of dG[s][t] q[cell(s, t)], the stations taken per
// tile of kNwTile x kNwTile station bins as in k_near_adj_warp.  The tile's
// q values over its region (RX x RY x lz cells, zero outside the mesh, whose
// table entries are zero anyway) and the slot -> region offset table are
// staged in shared memory once, so a station's gathers are shared-memory
// loads instead of scattered L2 sectors.  Each warp takes stations w, w + 8,
// ... of the tile, requests each row whole from L2 by bulk prefetch (one row
// per warp in flight keeps the requests within L2) and streams it in 16-byte
// evict-first loads, kNfChunk per lane in flight.  FP32 runs of 16 terms are summed in double-float per lane
// and across the warp (fixed butterfly): bitwise deterministic, no FP64
// operation per term or per run.  Stations whose box misses the mesh (sorted
// after every bin) get 0 from the first CTA.
constexpr int kNfChunk = 4;
constexpr size_t kNfSmemBudget = 64 * 1024;

struct NearFwdShape {
    bool ok = false;
    int RX = 0, RY = 0, lz = 0, RC = 0, ntx = 0, nty = 0;
    size_t o_meta = 0, o_roff = 0, o_q = 0, smem = 0;
};

static NearFwdShape near_fwd_shape(const grav_plan *p) {
    NearFwdShape z;
    z.RX = kNwTile + p->ng.bx - 1;
    z.RY = kNwTile + p->ng.by - 1;
    z.lz = std::min(p->ng.bz, p->nz);
    z.RC = z.RX * z.RY * z.lz;
    z.ntx = (p->ng.nbx + kNwTile - 1) / kNwTile;
    z.nty = (p->ng.nby + kNwTile - 1) / kNwTile;
    z.o_meta = 128;                                             // header: row table [2 kNwTile + 1]
    z.o_roff = z.o_meta + 2ull * 4 * kNwWarps * kNwPass;        // a pass's stations: index, base
    z.o_q = align_up(z.o_roff + 4ull * p->ng.ld, 16);          // roff[ld]
    z.smem = z.o_q + 4ull * z.RC;                              // q over the region
    z.ok = z.smem <= kNfSmemBudget && p->ng.ld % 4 == 0;
    return z;
}

__global__ void __launch_bounds__(kNwWarps * 32) k_near_fwd_tile(
    int nx, int ny, NearGeo ng, int RX, int RY, int lz, int ntx, uint32_t o_meta, uint32_t o_roff, uint32_t o_q,
    const float *__restrict__ dG, const int *__restrict__ bin_start, const int *__restrict__ bin_st,
    const int *__restrict__ st_i0, const int *__restrict__ st_j0, const float *__restrict__ qn, int64_t N,
    double *__restrict__ corr) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int *rowinfo = reinterpret_cast<int *>(smem_raw);                  // [2 kNwTile + 1]
    int *msidx = reinterpret_cast<int *>(smem_raw + o_meta);           // [kNwWarps kNwPass]
    int *mbase = msidx + kNwWarps * kNwPass;
    int *roff = reinterpret_cast<int *>(smem_raw + o_roff);
    float *qreg = reinterpret_cast<float *>(smem_raw + o_q);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    const int I0 = tx * kNwTile, J0 = ty * kNwTile;
    const int RC = RX * RY * lz;
    // slot -> region offset; slots of layers below lz and row padding hold
    // dG = 0 and point at region cell 0
    for (int u = tid; u < ng.ld; u += kNwWarps * 32) {
        int v = 0;
        if (u < ng.slots) {
            const int a = u % ng.bx, b = (u / ng.bx) % ng.by, l = u / (ng.bx * ng.by);
            if (l < lz) v = a + RX * (b + RY * l);
        }
        roff[u] = v;
    }
    // region cell (x, y, l) is mesh cell (I0 - bx + 1 + x, J0 - by + 1 + y, l)
    const int X0 = I0 - ng.bx + 1, Y0 = J0 - ng.by + 1;
    for (int c = tid; c < RC; c += kNwWarps * 32) {
        const int x = c % RX, y = (c / RX) % RY, l = c / (RX * RY);
        const int i = X0 + x, j = Y0 + y;
        qreg[c] = (i >= 0 && i < nx && j >= 0 && j < ny) ? qn[i + (int64_t)nx * (j + (int64_t)ny * l)] : 0.0f;
    }
    if (tid == 0) {
        int q = 0;
        const int i1 = min(I0 + kNwTile, ng.nbx);
        for (int r = 0; r < kNwTile; ++r) {
            const int sbj = J0 + r;
            int p0 = 0, p1 = 0;
            if (sbj < ng.nby) {
                p0 = bin_start[I0 + ng.nbx * sbj];
                p1 = bin_start[i1 + ng.nbx * sbj];
            }
            rowinfo[r] = p0;
            rowinfo[kNwTile + r] = q;
            q += p1 - p0;
        }
        rowinfo[2 * kNwTile] = q;
    }
    if (blockIdx.x == 0)   // stations whose box misses the mesh
        for (int64_t p = bin_start[ng.nbx * ng.nby] + (int64_t)tid; p < N; p += kNwWarps * 32) corr[bin_st[p]] = 0.0;
    __syncthreads();
    const int Q = rowinfo[2 * kNwTile];
    const int n4 = ng.ld >> 2;
    const float4 *dG4 = reinterpret_cast<const float4 *>(dG);
    const int4 *roff4 = reinterpret_cast<const int4 *>(roff);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int pass0 = 0; pass0 < Q; pass0 += kNwWarps * kNwPass) {
        const int pass1 = min(Q, pass0 + kNwWarps * kNwPass);
        if (pass0 > 0) __syncthreads();   // the previous pass's metadata is consumed
        if (tid < kNwWarps * kNwPass && pass0 + tid < pass1) {
            const int q = pass0 + tid;
            int r = 0;
            while (r + 1 < kNwTile && rowinfo[kNwTile + r + 1] <= q) ++r;
            const int sidx = bin_st[rowinfo[r] + (q - rowinfo[kNwTile + r])];
            const int ri = st_i0[sidx] + ng.bx - 1 - I0;
            const int rj = st_j0[sidx] + ng.by - 1 - J0;
            msidx[tid] = sidx;
            mbase[tid] = ri + RX * rj;
        }
        __syncthreads();
        for (int q = pass0 + warp; q < pass1; q += kNwWarps) {
            const int sidx = msidx[q - pass0];
            const float *qb = qreg + mbase[q - pass0];
            const float4 *row = dG4 + (int64_t)sidx * n4;
            if (lane == 0) prefetch_l2_bulk(row, 16u * (uint32_t)n4);
            float hi = 0.0f, lo = 0.0f;
            for (int v0 = 0; v0 < n4; v0 += 32 * kNfChunk) {
                float4 gq[kNfChunk];
#pragma unroll
                for (int c = 0; c < kNfChunk; ++c) {
                    const int v = v0 + lane + 32 * c;
                    gq[c] = v < n4 ? __ldcs(row + v) : zero4;
                }
                float run = 0.0f;
#pragma unroll
                for (int c = 0; c < kNfChunk; ++c) {
                    const int v = v0 + lane + 32 * c;
                    const int4 o = v < n4 ? roff4[v] : make_int4(0, 0, 0, 0);
                    run = fmaf(gq[c].x, qb[o.x], run);
                    run = fmaf(gq[c].y, qb[o.y], run);
                    run = fmaf(gq[c].z, qb[o.z], run);
                    run = fmaf(gq[c].w, qb[o.w], run);
                }
                float e;
                two_sum(hi, run, hi, e);
                lo += e;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ho = __shfl_xor_sync(0xffffffffu, hi, o), lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
                float e;
                two_sum(hi, ho, hi, e);
                lo += lo2 + e;
            }
            if (lane == 0) corr[sidx] = (double)hi + (double)lo;
        }
    }
}

// out[x + nx (y + ny l)] = sum over the station tiles (tx, ty) whose region holds
// the cell, ty then tx ascending (fixed order).
__global__ void k_near_adj_gather(int nx, int ny, int lz, int bx, int by, int RX, int RY, int ntx, int tile,
                                  const double *__restrict__ tpart, double *__restrict__ out) {
    const int64_t total = (int64_t)nx * ny * lz;
    const int64_t RC = (int64_t)RX * RY * lz;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx);
        const int y = (int)((k / nx) % ny);
        const int l = (int)(k / ((int64_t)nx * ny));
        double s = 0.0;
        for (int ty = y / tile; ty <= (y + by - 1) / tile; ++ty)
            for (int tx = x / tile; tx <= (x + bx - 1) / tile; ++tx) {
                const int ri = x - (tx * tile - bx + 1), rj = y - (ty * tile - by + 1);
                s += tpart[(int64_t)(ty * ntx + tx) * RC + ri + (int64_t)RX * (rj + (int64_t)RY * l)];
            }
        out[k] = s;
    }
}

// out[k] = vol * fs * (sum_c apart[c][k] + near[k] (top bz layers)) [* w2_l] [+ add[k]],
// fs = max|r| (bits in *fbits): the partials are in units of max|r|
__global__ void k_madj_finish(int nx, int ny, int nz, int bz, const double *__restrict__ apart, int nschunk,
                              const unsigned long long *__restrict__ fbits, double vol,
                              const double *__restrict__ near, const double *__restrict__ w2,
                              const double *__restrict__ add, double *__restrict__ out) {
    const int64_t M = (int64_t)nx * ny * nz;
    const int64_t plane = (int64_t)nx * ny;
    const double fs = fbits ? __longlong_as_double((long long)*fbits) : 1.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(k / plane);
        double s = 0.0;
        for (int c = 0; c < nschunk; ++c) s += apart[(int64_t)c * M + k];
        if (l < bz) s += near[k];
        s *= fs;
        s *= vol;
        if (w2) s *= w2[l];
        if (add) s += add[k];
        out[k] = s;
    }
}

// Far-field part of diag(G W^-2 G^T): sum_k w2_l (dz/R^3)^2 per station
// (times vol^2 later); thread = T stations, grid.y = column chunks.
template <int T, bool QUAD>
__global__ void __launch_bounds__(kMfThreads) k_mdiag(MixedGeo g, const float *__restrict__ w2f,
                                                      const float4 *__restrict__ st32,
                                                      const float2 *__restrict__ stz, int cols_per_chunk,
                                                      double *__restrict__ part) {
    const int64_t s_base = (int64_t)blockIdx.x * (kMfThreads * T) + threadIdx.x;
    float xh[T], xl[T], yh[T], yl[T], zs[T], hi[T], lo[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t s = s_base + (int64_t)t * kMfThreads;
        const bool ok = s < g.N;
        const float4 P = ok ? st32[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        xh[t] = P.x; xl[t] = P.y; yh[t] = P.z; yl[t] = P.w;
        zs[t] = ok ? stz[s].x : -1.0f;
        hi[t] = 0.f; lo[t] = 0.f;
    }
    const int c0 = blockIdx.y * cols_per_chunk;
    const int c1 = min(g.ncol, c0 + cols_per_chunk);
    for (int col = c0; col < c1; ++col) {
        const int i = col % g.nx, j = col / g.nx;
        const float2 X = make_float2(g.cx[2 * i], g.cx[2 * i + 1]);
        const float2 Y = make_float2(g.cy[2 * j], g.cy[2 * j + 1]);
        float h2[T], ph[T], cs[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            h2[t] = far_h2(X, Y, xh[t], xl[t], yh[t], yl[t]);
            ph[t] = QUAD ? far_ph(X, Y, xh[t], xl[t], yh[t], yl[t], g.qa, g.qb) : 0.0f;
            cs[t] = 0.f;
        }
        for (int l = 0; l < g.nz; ++l) {
            const float zc = g.czc[l], wl = w2f[l];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float dz = zc - zs[t];
                const float k = far_k<QUAD>(dz, fmaf(dz, dz, h2[t]), g.qg, ph[t]);
                cs[t] = fmaf(wl, k * k, cs[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            float s, e;
            two_sum(hi[t], cs[t], s, e);
            hi[t] = s;
            lo[t] += e;
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t s = s_base + (int64_t)t * kMfThreads;
        if (s < g.N) part[(int64_t)blockIdx.y * g.N + s] = (double)hi[t] + (double)lo[t];
    }
}

inline int grid_for(int64_t n, int threads, int cap = 148 * 32) {
    int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

constexpr int kMfColsPerStage = 32;

// Layer groups of the broadcast adjoint: 16 layers (8 packed pairs; measured
// fastest per layer among 8/12/16/20 at 2 CTAs per SM), the last group
// exactly the layers left (an odd count ends with one scalar layer).  At
// nz = 75 that is 16, 16, 16, 16, 11: the 12-layer last group used before (a
// multiple of 4) spent one reciprocal square root in 76 on a padded layer.
#ifndef GRAV_AB_TZ
#define GRAV_AB_TZ 16
#endif
constexpr int kAbTz = GRAV_AB_TZ;
static_assert(kAbTz % 4 == 0 && kAbTz >= 16, "layer group: a multiple of 4, at least 16");
int adj_tz_bc(int nz) { (void)nz; return kAbTz; }
int adj_tzl_bc(int nz) {
    const int tz = adj_tz_bc(nz);
    return nz - tz * ((nz + tz - 1) / tz - 1);
}

// Layer group of the shuffle adjoint layout (small meshes): TZ in
// {8, 10, 12, 14, 16} minimising the modelled time
//   waves x TZ x stations per chunk x CTAs per SM x per-layer cost(TZ),
// waves = ceil(CTAs / (148 x CTAs per SM)) with the station chunking that
// mixed_sizes() applies.  It accounts for padded layers (ceil(nz/TZ) TZ >= nz)
// and for a nearly empty last wave.  Per-layer costs measured on the packed
// kernel (17 serving-sized meshes, 1.7k-43.9k columns, 2k-20k stations):
// 8 and 10: 1.03, 12 and 14: 1.00, 16: 0.96; the model's choice was within
// 0.4 % of the best of the five on average (4.9 % at worst).
int adj_tz(int nz, int ncol, int64_t N) {
    if (GRAV_MA_TZ == 8 || GRAV_MA_TZ == 10 || GRAV_MA_TZ == 12 || GRAV_MA_TZ == 14 || GRAV_MA_TZ == 16)
        return GRAV_MA_TZ;
    const int tzs[5] = {8, 10, 12, 14, 16};
    const double cost[5] = {1.03, 1.03, 1.00, 1.00, 0.96};
    int best = 8;
    double bc = 1e300;
    for (int q = 0; q < 5; ++q) {
        const int T = tzs[q];
        const int minb = T <= 8 ? 3 : 2;   // MaMinBlocks<T>
        const int64_t ngz = (nz + T - 1) / T;
        const int64_t ctas = ((int64_t)ncol * ngz + kMaWarps - 1) / kMaWarps;
        int64_t nsch = std::max<int64_t>(1, (148LL * 8 + ctas - 1) / ctas);
        nsch = std::min<int64_t>(nsch, std::max<int64_t>(1, (N + kMaStage - 1) / kMaStage));
        int64_t len = (N + nsch - 1) / nsch;
        len = (len + kMaStage - 1) / kMaStage * kMaStage;
        nsch = (N + len - 1) / len;
        const int64_t waves = (ctas * nsch + 148LL * minb - 1) / (148LL * minb);
        const double c = (double)waves * T * (double)std::min<int64_t>(len, N) * minb * cost[q];
        if (c < bc) { bc = c; best = T; }
    }
    return best;
}

}  // namespace

// Plan-time sizing and device set-up of the mixed path.  Allocations come from
// the plan's arena (see api.cu, which calls mixed_scratch_bytes first).
struct MixedSizes {
    int cols_per_chunk, nchunk, tz, ngz, nschunk, bc;
    int64_t schunk_len;
    size_t cub_temp;
    int nbins;
    int key_bits;
};

static MixedSizes mixed_sizes(const grav_plan *p) {
    MixedSizes z{};
    const int ncol = p->nx * p->ny;
    const int tiles = (int)((p->N + kMfThreads * kMfT - 1) / (kMfThreads * kMfT));
    // aim at >= 16 waves of ~6 resident CTAs per SM, each CTA >= 16 columns
    const int64_t target = 148LL * 6 * 16;   // (32 or 48 waves: measured no faster)
    int nchunk = (int)std::min<int64_t>(std::max<int64_t>(1, (target + tiles - 1) / tiles), std::max(1, ncol / 16));
    z.cols_per_chunk = (ncol + nchunk - 1) / nchunk;
    z.nchunk = (ncol + z.cols_per_chunk - 1) / z.cols_per_chunk;
    // broadcast layout when the cells alone fill the GPU (>= 2 CTAs per SM);
    // station chunks then add waves (>= 32) to trim the tail: measured at
    // 210 x 210 x 75 x 178,797, 2 chunks (5.8 waves) 143.2 ms, 6 chunks
    // 138.9 ms, 12 chunks (35 waves) 137.5 ms; the partials (chunks x M
    // doubles) are capped at 512 MB
    //
    // Smaller meshes (serving-sized) get the broadcast layout too when station
    // chunks of >= 64 stations can fill one wave: measured on the first 24
    // jobs of the serving stream, the shuffle layout reached 65 % of the MUFU
    // peak (pairs-weighted) and the broadcast layout 76 % with 1024-station
    // chunks; the chunk count is then chosen by a wave model (below).
    const int tz_bc = adj_tz_bc(p->nz);
    const int64_t slots = 148LL * GRAV_AB_MINB;
    const int64_t bc_ctas = (int64_t)((ncol + kAbWarps * 32 - 1) / (kAbWarps * 32)) * ((p->nz + tz_bc - 1) / tz_bc);
    const int64_t part_cap = std::max<int64_t>(1, (512ll << 20) / (8 * std::max<int64_t>(p->M, 1)));
    const bool bc_fills = bc_ctas >= slots || bc_ctas * std::min<int64_t>(part_cap, p->N / 64) >= slots;
    z.bc = (GRAV_AB_FORCE >= 0) ? GRAV_AB_FORCE : (bc_fills ? 1 : 0);
    // run-time override of the layout choice: GRAV_ADJOINT_LAYOUT=broadcast|shuffle|auto
    if (const char *env = std::getenv("GRAV_ADJOINT_LAYOUT")) {
        if (std::strcmp(env, "broadcast") == 0) z.bc = 1;
        else if (std::strcmp(env, "shuffle") == 0) z.bc = 0;
    }
    z.tz = z.bc ? tz_bc : adj_tz(p->nz, ncol, p->N);
    z.ngz = (p->nz + z.tz - 1) / z.tz;
    int64_t nsch, stage;
    bool modelled = false;
    if (z.bc) {
        nsch = std::max<int64_t>(1, (32 * slots + bc_ctas - 1) / bc_ctas);
        nsch = std::min<int64_t>(nsch, part_cap);
        stage = kAbStage;
        const int64_t nsch_stages = std::min<int64_t>(nsch, (p->N + stage - 1) / stage);
        if (bc_ctas * nsch_stages < 8 * slots && p->N >= 64) {
            // fewer than 8 waves with whole 1024-station stages: chunks of any
            // multiple of 32 stations (>= 64), the count minimising a list-
            // scheduling model in units of one station through a full
            // 16-layer group: total work / slots + the longest CTA (the
            // groups differ in size, so one tight wave leaves slots idle) +
            // each CTA's fixed cost (~32 stations) + the finish kernel's read
            // of the chunk partials (M doubles per chunk, ~M / 2e5)
            const int ngz_bc = (p->nz + tz_bc - 1) / tz_bc;
            const double layers = (double)(tz_bc * (ngz_bc - 1) + adj_tzl_bc(p->nz)) / tz_bc;   // groups' work
            const int64_t cblocks = (ncol + kAbWarps * 32 - 1) / (kAbWarps * 32);
            double best = 1e300;
            int64_t best_n = 1;
            // (more than 64 waves of chunks gains nothing: the search stays short)
            const int64_t hi = std::min<int64_t>(std::min<int64_t>(part_cap, p->N / 64), 64 * slots / bc_ctas + 1);
            for (int64_t n = 1; n <= std::max<int64_t>(1, hi); ++n) {
                int64_t len = (p->N + n - 1) / n;
                len = (len + 31) / 32 * 32;
                const int64_t ns = (p->N + len - 1) / len;
                const double work = (double)ns * (double)cblocks * layers * (double)(len + 32);
                const double c = work / (double)slots + (double)(len + 32) + (double)ns * (double)p->M / 2e5;
                if (c < best) { best = c; best_n = n; }
            }
            nsch = best_n;
            stage = 32;
            modelled = true;
        }
    } else {
        const int64_t groups_ctas = ((int64_t)ncol * z.ngz + kMaWarps - 1) / kMaWarps;
        nsch = std::max<int64_t>(1, (148LL * 8 + groups_ctas - 1) / groups_ctas);
        stage = kMaStage;
    }
    if (!modelled) nsch = std::min<int64_t>(nsch, (p->N + stage - 1) / stage);
    int64_t len = (p->N + nsch - 1) / nsch;
    len = (len + stage - 1) / stage * stage;   // keeps every chunk start 16-byte aligned (stage even)
    z.schunk_len = len;
    z.nschunk = (int)((p->N + len - 1) / len);
    z.nbins = p->ng.nbx * p->ng.nby;
    int bits = 1;
    while ((1LL << bits) <= (int64_t)z.nbins) ++bits;
    z.key_bits = bits;
    size_t tmp = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tmp, (unsigned *)nullptr, (unsigned *)nullptr, (int *)nullptr,
                                    (int *)nullptr, (int)p->N, 0, bits);
    z.cub_temp = tmp;
    return z;
}

// GRAV_MIXED_CORNER forward sizing: FP32 node-weight rows padded to 16 bytes,
// row chunks so that the grid holds >= 8 CTAs per SM.
struct CornerSizes {
    int ldw, rows_per_chunk, nchunk;
};
constexpr int kCfRowsPerStage = 8;

static CornerSizes corner_sizes(const grav_plan *p) {
    CornerSizes c{};
    c.ldw = (p->nx + 1 + 3) / 4 * 4;
    const int nrows = (p->ny + 1) * (p->nz + 1);
    const int64_t tiles = (p->N + kCfThreads * kCfT - 1) / (kCfThreads * kCfT);
    const int64_t want = std::max<int64_t>(1, (148LL * 8 + tiles - 1) / tiles);
    const int nchunk = (int)std::min<int64_t>(want, std::max(1, nrows / kCfRowsPerStage));
    c.rows_per_chunk = (nrows + nchunk - 1) / nchunk;
    c.nchunk = (nrows + c.rows_per_chunk - 1) / c.rows_per_chunk;
    return c;
}

static size_t cfwd_smem(const grav_plan *p) {
    return 128 + (size_t)((p->nx + 2) / 2 * 2) * 8 + 2ull * kCfRowsPerStage * corner_sizes(p).ldw * 4;
}

size_t mixed_scratch_bytes(const grav_plan *p) {
    const MixedSizes z = mixed_sizes(p);
    const int64_t N = p->N, M = p->M;
    const int nzp = (p->nz + 3) / 4 * 4;
    const int64_t lz = std::min(p->ng.bz, p->nz);
    size_t b = 0;
    auto add = [&](size_t v) { b += (v + 255) / 256 * 256 + 256; };
    add(8ull * p->nx); add(8ull * p->ny); add(4ull * nzp); add(4ull * nzp);   // cx, cy, czc, w2f
    add(4ull * p->nx * p->ny * nzp);                                       // qT
    add(4ull * M);                                                          // qN
    add(16ull * (N + 2)); add(8ull * (N + 4));                             // st32, stz (padded)
    add(8); add(8);                                                         // max|r|, max|m|
    add(8ull * z.nchunk * N);                                               // m_part
    add(8ull * z.nschunk * M);                                              // m_apart
    add(4ull * N * p->ng.ld);                                               // dG (FP32, padded rows)
    add(4ull * N); add(4ull * N);                                           // i0, j0
    add(4ull * p->ng.ld);                                                   // slot -> cell offset
    add(8ull * N); add(8ull * N);                                           // diag_corr, near_corr
    add(8ull * p->nx * p->ny * lz);                                         // near adjoint
    {
        const NearAdjShape na = near_adj_shape(p);
        const NearWarpShape nw = near_warp_shape(p);
        const NearLayerShape nl = near_layer_shape(p);
        const size_t tb = std::max(std::max(na.ok ? 8ull * na.ntx * na.nty * na.RC : 0ull,
                                            nw.ok ? 8ull * nw.ntx * nw.nty * nw.RC : 0ull),
                                   nl.ok ? 8ull * nl.ntx * nl.nty * nl.RC : 0ull);
        if (tb) add(tb);                                                    // per-tile near sums
    }
    add(4ull * N); add(4ull * N); add(4ull * N); add(4ull * N);             // keys, keys_sorted, vals, bin_st
    add(4ull * (z.nbins + 2));                                              // bin_start
    add(z.cub_temp);
    add(8ull * std::max<int64_t>(N, 1) * std::max(z.nchunk, 1));            // diag partials
    if (p->opt.precision == GRAV_MIXED_CORNER) {
        const CornerSizes c = corner_sizes(p);
        add(8ull * (p->nx + 1)); add(8ull * (p->ny + 1)); add(4ull * (p->nz + 1));   // ex, ey, ez
        add(4ull * (p->ny + 1) * (p->nz + 1) * c.ldw);                              // FP32 node weights
        add(8ull * c.nchunk * N);                                                   // row-chunk partials
    }
    return b;
}

static void *take(grav_plan *p, size_t bytes) {
    void *q = p->arena.take(bytes);
    return q;
}

int near_setup_warps(const grav_plan *p) {
    const size_t per_node = p->opt.precision == GRAV_MIXED_CORNER ? 12 : 8;   // FP64 (+ FP32) or double-float values
    const size_t per_warp = (size_t)(p->ng.bx + 1) * (p->ng.by + 1) * (p->ng.bz + 1) * per_node + 256 +   // + node queue
                            8ull * (p->ng.bx + p->ng.by + p->ng.bz + 3);   // + box node offsets (double-float)
    const size_t cap = 200 * 1024;
    return (int)std::min<size_t>(kNsWarps, cap / per_warp);
}

int mixed_setup(grav_plan *p, cudaStream_t s) {
    const MixedSizes z = mixed_sizes(p);
    const int ns_warps = near_setup_warps(p);
    if (ns_warps < 1) return GRAV_EINVAL;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const int nzp = (nz + 3) / 4 * 4;
    const double a = p->xe[1] - p->xe[0];
    const double xref = 0.5 * (p->xe.front() + p->xe.back());
    const double yref = 0.5 * (p->ye.front() + p->ye.back());
    std::vector<float> hcx(2 * nx), hcy(2 * ny), hcz(nzp), hw2(nzp, 0.0f);
    for (int i = 0; i < nx; ++i) {
        const double v = 0.5 * (p->xe[i] + p->xe[i + 1]) - xref;
        hcx[2 * i] = (float)v;
        hcx[2 * i + 1] = (float)(v - (double)(float)v);
    }
    for (int j = 0; j < ny; ++j) {
        const double v = 0.5 * (p->ye[j] + p->ye[j + 1]) - yref;
        hcy[2 * j] = (float)v;
        hcy[2 * j + 1] = (float)(v - (double)(float)v);
    }
    for (int l = 0; l < nzp; ++l) {
        const int ll = std::min(l, nz - 1);
        hcz[l] = (float)(0.5 * (p->ze[ll] + p->ze[ll + 1]));
        if (l < nz) {
            const double zc = 0.5 * (p->ze[l] + p->ze[l + 1]) - p->ze[0];
            hw2[l] = (float)((zc + p->opt.z0) * (zc + p->opt.z0));
        }
    }
    p->m_cx = (float *)take(p, 8ull * nx);
    p->m_cy = (float *)take(p, 8ull * ny);
    p->m_czc = (float *)take(p, 4ull * nzp);
    float *w2f = (float *)take(p, 4ull * nzp);
    p->qT = (float *)take(p, 4ull * nx * ny * nzp);
    p->qN = (float *)take(p, 4ull * p->M);
    p->st32 = (float4 *)take(p, 16ull * (p->N + 2));
    p->stz = (float2 *)take(p, 8ull * (p->N + 4));
    p->rmax_bits = (unsigned long long *)take(p, 8);
    p->mmax_bits = (unsigned long long *)take(p, 8);
    p->m_fwd_cols_per_chunk = z.cols_per_chunk;
    p->m_fwd_nchunk = z.nchunk;
    p->m_adj_tz = z.tz;
    p->m_adj_ngz = z.ngz;
    p->m_adj_nschunk = z.nschunk;
    p->m_adj_schunk_len = (int)z.schunk_len;
    p->m_adj_bc = z.bc;
    p->m_part = (double *)take(p, 8ull * z.nchunk * p->N);
    p->m_apart = (double *)take(p, 8ull * z.nschunk * p->M);
    p->dG = (float *)take(p, 4ull * p->N * p->ng.ld);
    p->st_i0 = (int *)take(p, 4ull * p->N);
    p->st_j0 = (int *)take(p, 4ull * p->N);
    p->near_off = (int *)take(p, 4ull * p->ng.ld);
    p->diag_corr = (double *)take(p, 8ull * p->N);
    p->near_corr = (double *)take(p, 8ull * p->N);
    const int64_t lz = std::min(p->ng.bz, nz);
    p->m_cellacc = (double *)take(p, 8ull * nx * ny * lz);
    {
        // form: layer-split if its shared memory fits, else warp-private, else
        // station-streaming, else cell-tiled; GRAV_NEAR_ADJ=warp|rows|tiles
        // restricts the choice
        const NearAdjShape na = near_adj_shape(p);
        const NearWarpShape nw = near_warp_shape(p);
        const NearLayerShape nl = near_layer_shape(p);
        const char *ev = std::getenv("GRAV_NEAR_ADJ");
        const bool want_tiles = ev && std::strcmp(ev, "tiles") == 0;
        const bool want_rows = ev && std::strcmp(ev, "rows") == 0;
        const bool want_warp = ev && std::strcmp(ev, "warp") == 0;
        p->near_adj_rows = 0;
        if (!want_tiles && !want_rows && !want_warp && nl.ok) p->near_adj_rows = 3;
        else if (!want_tiles && !want_rows && nw.ok) p->near_adj_rows = 2;
        else if (!want_tiles && na.ok) p->near_adj_rows = 1;
        // near forward: tile form when it fits; GRAV_NEAR_FWD=warp forces a warp per station
        const char *fv = std::getenv("GRAV_NEAR_FWD");
        p->near_fwd_tile = near_fwd_shape(p).ok && !(fv && std::strcmp(fv, "warp") == 0);
        if (p->near_adj_rows == 3) p->near_tpart = (double *)take(p, 8ull * nl.ntx * nl.nty * nl.RC);
        if (p->near_adj_rows == 2) p->near_tpart = (double *)take(p, 8ull * nw.ntx * nw.nty * nw.RC);
        if (p->near_adj_rows == 1) p->near_tpart = (double *)take(p, 8ull * na.ntx * na.nty * na.RC);
    }
    unsigned *keys = (unsigned *)take(p, 4ull * p->N);
    unsigned *keys_sorted = (unsigned *)take(p, 4ull * p->N);
    int *vals = (int *)take(p, 4ull * p->N);
    p->bin_st = (int *)take(p, 4ull * p->N);
    p->bin_start = (int *)take(p, 4ull * (z.nbins + 2));
    void *cub_tmp = take(p, std::max<size_t>(z.cub_temp, 16));
    p->m_w2f = w2f;
    const bool corner = p->opt.precision == GRAV_MIXED_CORNER;
    std::vector<float> hex, hey, hez;
    if (corner) {
        const CornerSizes c = corner_sizes(p);
        p->cr_ldw = c.ldw;
        p->cr_rows_per_chunk = c.rows_per_chunk;
        p->cr_nchunk = c.nchunk;
        hex.resize(2 * (nx + 1));
        hey.resize(2 * (ny + 1));
        hez.resize(nz + 1);
        for (int i = 0; i <= nx; ++i) {
            const double v = p->xe[i] - xref;
            hex[2 * i] = (float)v;
            hex[2 * i + 1] = (float)(v - (double)(float)v);
        }
        for (int j = 0; j <= ny; ++j) {
            const double v = p->ye[j] - yref;
            hey[2 * j] = (float)v;
            hey[2 * j + 1] = (float)(v - (double)(float)v);
        }
        for (int l = 0; l <= nz; ++l) hez[l] = (float)p->ze[l];
        p->mg.ex = (const float *)take(p, 8ull * (nx + 1));
        p->mg.ey = (const float *)take(p, 8ull * (ny + 1));
        p->mg.ez = (const float *)take(p, 4ull * (nz + 1));
        p->cr_w32 = (float *)take(p, 4ull * (ny + 1) * (nz + 1) * c.ldw);
        p->cr_part = (double *)take(p, 8ull * c.nchunk * p->N);
    }
    if (p->arena.overflow) return GRAV_EDEVICE;
    if (corner) {
        cudaMemcpyAsync((void *)p->mg.ex, hex.data(), 8ull * (nx + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync((void *)p->mg.ey, hey.data(), 8ull * (ny + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync((void *)p->mg.ez, hez.data(), 4ull * (nz + 1), cudaMemcpyHostToDevice, s);
    }

    p->mg.nx = nx; p->mg.ny = ny; p->mg.nz = nz; p->mg.nzp = nzp; p->mg.ncol = nx * ny;
    p->mg.cx = p->m_cx; p->mg.cy = p->m_cy; p->mg.czc = p->m_czc; p->mg.N = p->N;
    {
        const double a2 = p->cell_a * p->cell_a, b2 = p->cell_b * p->cell_b, c2 = p->cell_c * p->cell_c;
        p->mg.qa = p->cubic ? 0.0f : (float)((12.0 * a2 - 3.0 * b2 - 9.0 * c2) / 24.0);
        p->mg.qb = p->cubic ? 0.0f : (float)((12.0 * b2 - 3.0 * a2 - 9.0 * c2) / 24.0);
        p->mg.qg = p->cubic ? 0.0f : (float)((6.0 * c2 - 3.0 * a2 - 3.0 * b2) / 24.0);
    }

    {
        // slot t = a + bx (bj + by l) of a station's window box -> cell offset from its box origin
        std::vector<int> hoff(p->ng.ld, 0);   // padding slots: offset 0
        for (int l = 0; l < p->ng.bz; ++l)
            for (int bj = 0; bj < p->ng.by; ++bj)
                for (int a = 0; a < p->ng.bx; ++a)
                    hoff[a + p->ng.bx * (bj + p->ng.by * l)] = a + nx * (bj + ny * l);
        cudaMemcpyAsync(p->near_off, hoff.data(), 4ull * p->ng.ld, cudaMemcpyHostToDevice, s);
    }
    cudaMemcpyAsync(p->m_cx, hcx.data(), 8ull * nx, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->m_cy, hcy.data(), 8ull * ny, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->m_czc, hcz.data(), 4ull * nzp, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(w2f, hw2.data(), 4ull * nzp, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(p->stz, 0, 8ull * (p->N + 4), s);
    k_prep_stations<<<grid_for(p->N, 256), 256, 0, s>>>(p->sx, p->sy, p->sz, p->N, xref, yref, p->st32, p->stz);

    const int nnode = (p->ng.bx + 1) * (p->ng.by + 1) * (p->ng.bz + 1);
    const size_t smem = (size_t)ns_warps * (nnode * (corner ? 12 : 8) + 256 + 8ull * (p->ng.bx + p->ng.by + p->ng.bz + 3));
    const double vol_mgal = kGammaMgal * p->cell_a * p->cell_b * p->cell_c;
    // nodes within the window radius plus half a cell diagonal (relative margin 1e-9)
    const double node_r = (p->ng.radius_cells * p->ng.width +
                           0.5 * std::sqrt(p->cell_a * p->cell_a + p->cell_b * p->cell_b + p->cell_c * p->cell_c)) *
                          (1.0 + 1e-9);
    auto setup = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        kern<<<(unsigned)((p->N + ns_warps - 1) / ns_warps), ns_warps * 32, smem, s>>>(
            make_geo(p), p->mg, p->ng, p->xe[0], p->ye[0], a, p->ye[1] - p->ye[0], vol_mgal, node_r * node_r,
            p->sx, p->sy, p->sz,
            p->d_w2, p->st32,
            p->stz, p->dG, p->st_i0, p->st_j0, p->diag_corr, keys, vals, (unsigned)z.nbins);
    };
    if (corner) setup(k_near_setup<kNsCorner>);
    else if (p->opt.near_fp64) setup(k_near_setup<kNsF64>);
    else setup(k_near_setup<kNsDF>);
    size_t tmp = z.cub_temp;
    cub::DeviceRadixSort::SortPairs(cub_tmp, tmp, keys, keys_sorted, vals, p->bin_st, (int)p->N, 0, z.key_bits, s);
    k_bin_bounds<<<grid_for(z.nbins + 1, 256), 256, 0, s>>>(keys_sorted, p->N, z.nbins, p->bin_start);
    note_launches(4);
    // the diagonal's far-field partials reuse m_part (same chunking as the forward)
    return GRAV_OK;
}

int mixed_adj_last_group(const grav_plan *p) { return p->m_adj_bc ? adj_tzl_bc(p->nz) : p->m_adj_tz; }

size_t mfwd_smem(const grav_plan *p) { return mfwd_layout(p->mg, kMfColsPerStage).total; }

void launch_absmax(const double *v, int64_t n, unsigned long long *bits, cudaStream_t s) {
    cudaMemsetAsync(bits, 0, 8, s);
    k_absmax<<<grid_for(n, 256, 148 * 4), 256, 0, s>>>(v, n, bits);
    note_launches(1);
}

void launch_mixed_prep_q(const grav_plan *p, const double *m, cudaStream_t s, bool normalize) {
    const float scale = (float)(kGammaMgal * p->cell_a * p->cell_b * p->cell_c);
    const int64_t total = (int64_t)p->mg.ncol * p->mg.nzp;
    const unsigned long long *bits = normalize ? p->mmax_bits : nullptr;
    if (normalize) {
        cudaMemsetAsync(p->mmax_bits, 0, 8, s);
        k_absmax<<<grid_for(p->M, 256, 148 * 4), 256, 0, s>>>(m, p->M, p->mmax_bits);
        note_launches(1);
    }
    k_prep_q<<<grid_for(total, 256), 256, 0, s>>>(p->mg, m, scale, bits, p->qT);
    k_prep_qn<<<grid_for(p->M, 256), 256, 0, s>>>(p->M, m, scale, bits, p->qN);
    note_launches(2);
}

int mixed_fwd_tail(const grav_plan *p) { return (p->cubic && (p->nz & 3)) ? 1 : 0; }

void launch_mixed_fwd(const grav_plan *p, cudaStream_t s) {
    const int tiles = (int)((p->N + kMfThreads * kMfT - 1) / (kMfThreads * kMfT));
    dim3 grid(tiles, p->m_fwd_nchunk);
    const size_t smem = mfwd_smem(p);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        stage_begin(p, kStageFwdMain, s);
        kern<<<grid, kMfThreads, smem, s>>>(p->mg, p->qT, p->st32, p->stz, p->m_fwd_cols_per_chunk, kMfColsPerStage,
                                            p->m_part, p->ctx->d_status);
        stage_end(p, kStageFwdMain, s);
    };
    if (!p->cubic) go(k_mfwd<kMfT, true, false>);
    else if (mixed_fwd_tail(p)) go(k_mfwd<kMfT, false, true>);
    else go(k_mfwd<kMfT, false, false>);
    note_launches(1);
}

void launch_corner_fwd(const grav_plan *p, const double *m, cudaStream_t s) {
    const int64_t total = (int64_t)(p->ny + 1) * (p->nz + 1) * p->cr_ldw;
    k_node_weights32<<<grid_for(total, 256), 256, 0, s>>>(p->nx, p->ny, p->nz, p->cr_ldw, m, p->cr_w32);
    const int tiles = (int)((p->N + kCfThreads * kCfT - 1) / (kCfThreads * kCfT));
    dim3 grid(tiles, p->cr_nchunk);
    cudaFuncSetAttribute(k_cfwd32<kCfT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    stage_begin(p, kStageFwdMain, s);
    k_cfwd32<kCfT><<<grid, kCfThreads, cfwd_smem(p), s>>>(p->mg, p->cr_ldw, p->cr_w32, p->cr_rows_per_chunk,
                                                          kCfRowsPerStage, p->st32, p->stz, p->cr_part,
                                                          p->ctx->d_status);
    stage_end(p, kStageFwdMain, s);
    note_launches(2);
}

void launch_mixed_near_fwd(const grav_plan *p, const double *m, cudaStream_t s) {
    const int64_t threads = p->N * 32;
    stage_begin(p, kStageFwdNear, s);
    (void)m;   // the near field reads the FP32 q that launch_mixed_prep_q formed from m
    if (p->near_fwd_tile) {
        const NearFwdShape nf = near_fwd_shape(p);
        cudaFuncSetAttribute(k_near_fwd_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nf.smem);
        k_near_fwd_tile<<<(unsigned)(nf.ntx * nf.nty), kNwWarps * 32, nf.smem, s>>>(
            p->nx, p->ny, p->ng, nf.RX, nf.RY, nf.lz, nf.ntx, (uint32_t)nf.o_meta, (uint32_t)nf.o_roff,
            (uint32_t)nf.o_q, p->dG, p->bin_start, p->bin_st, p->st_i0, p->st_j0, p->qN, p->N, p->near_corr);
        stage_end(p, kStageFwdNear, s);
        note_launches(1);
        return;
    }
    k_near_fwd<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(p->nx, p->ny, p->nz, p->ng, p->N, p->dG,
                                                                p->st_i0, p->st_j0, p->near_off, p->qN,
                                                                p->near_corr);
    stage_end(p, kStageFwdNear, s);
    note_launches(1);
}

// k_madj_bc<TZ, tzl> for the run-time last-group size tzl (1 <= tzl <= TZ)
template <int TZ, int L, bool Q, typename F>
void pick_bc_last(int tzl, F &gob) {
    if constexpr (L < TZ) {
        if (tzl == L) { gob(k_madj_bc<TZ, L, Q>); return; }
        pick_bc_last<TZ, L + 1, Q>(tzl, gob);
    } else {
        gob(k_madj_bc<TZ, TZ, Q>);
    }
}

void launch_mixed_adj(const grav_plan *p, const double *r, cudaStream_t s) {
    cudaMemsetAsync(p->rmax_bits, 0, 8, s);
    k_absmax<<<grid_for(p->N, 256, 148 * 4), 256, 0, s>>>(r, p->N, p->rmax_bits);
    k_set_rz<<<grid_for(p->N, 256), 256, 0, s>>>(p->stz, r, p->N, p->rmax_bits);
    note_launches(2);
    const int64_t groups = (int64_t)p->mg.ncol * p->m_adj_ngz;
    dim3 grid((unsigned)((groups + kMaWarps - 1) / kMaWarps), p->m_adj_nschunk);
    const size_t smem = 128 + 2ull * kMaStage * (sizeof(float4) + sizeof(float2));
    note_launches(1);
    stage_begin(p, kStageAdjMain, s);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        kern<<<grid, kMaWarps * 32, smem, s>>>(p->mg, p->st32, p->stz, p->m_adj_ngz, p->m_adj_schunk_len,
                                              p->m_apart, p->ctx->d_status);
    };
    if (p->m_adj_bc) {
        const int cblocks = (p->mg.ncol + kAbWarps * 32 - 1) / (kAbWarps * 32);
        dim3 gbc((unsigned)(cblocks * p->m_adj_ngz), p->m_adj_nschunk);
        const size_t sm_bc = 128 + 2ull * kAbStage * (sizeof(float4) + sizeof(float2));
        auto gob = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            kern<<<gbc, kAbWarps * 32, sm_bc, s>>>(p->mg, p->st32, p->stz, p->m_adj_ngz, p->m_adj_schunk_len,
                                                  p->m_apart, p->ctx->d_status);
        };
        const int tzl = adj_tzl_bc(p->nz);
        auto pick = [&](auto quad) {
            constexpr bool Q = decltype(quad)::value;
            pick_bc_last<kAbTz, 1, Q>(tzl, gob);
        };
        if (p->cubic) pick(std::false_type{}); else pick(std::true_type{});
    } else {
        auto pick = [&](auto quad) {
            constexpr bool Q = decltype(quad)::value;
            switch (p->m_adj_tz) {
                case 16: go(k_madj<16, Q>); break;
                case 14: go(k_madj<14, Q>); break;
                case 12: go(k_madj<12, Q>); break;
                case 10: go(k_madj<10, Q>); break;
                default: go(k_madj<8, Q>); break;
            }
        };
        if (p->cubic) pick(std::false_type{}); else pick(std::true_type{});
    }
    stage_end(p, kStageAdjMain, s);
    const int lz = std::min(p->ng.bz, p->nz);
    stage_begin(p, kStageAdjNear, s);
    if (p->near_adj_rows == 3) {
        const NearLayerShape nl = near_layer_shape(p);
        cudaFuncSetAttribute(k_near_adj_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nl.smem);
        k_near_adj_layer<<<(unsigned)(nl.ntx * nl.nty), 32 * nl.nwarps, nl.smem, s>>>(
            p->ng, nl.RX, nl.RY, nl.SX, nl.lz, nl.ntx, (uint32_t)nl.o_meta, (uint32_t)nl.o_roff, (uint32_t)nl.o_acc,
            p->dG, p->bin_start, p->bin_st, p->st_i0, p->st_j0, p->stz, p->near_tpart);
        const int64_t cells = (int64_t)p->nx * p->ny * lz;
        k_near_adj_gather<<<grid_for(cells, 256), 256, 0, s>>>(p->nx, p->ny, lz, p->ng.bx, p->ng.by, nl.RX, nl.RY,
                                                               nl.ntx, kNwTile, p->near_tpart, p->m_cellacc);
        note_launches(1);
    } else if (p->near_adj_rows == 2) {
        const NearWarpShape nw = near_warp_shape(p);
        cudaFuncSetAttribute(k_near_adj_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nw.smem);
        k_near_adj_warp<<<(unsigned)(nw.ntx * nw.nty), kNwWarps * 32, nw.smem, s>>>(
            p->ng, nw.RX, nw.RY, nw.lz, nw.ntx, (uint32_t)nw.o_meta, (uint32_t)nw.o_roff, (uint32_t)nw.o_acc, p->dG,
            p->bin_start,
            p->bin_st, p->st_i0, p->st_j0, p->stz, p->near_tpart);
        const int64_t cells = (int64_t)p->nx * p->ny * lz;
        k_near_adj_gather<<<grid_for(cells, 256), 256, 0, s>>>(p->nx, p->ny, lz, p->ng.bx, p->ng.by, nw.RX, nw.RY,
                                                               nw.ntx, kNwTile, p->near_tpart, p->m_cellacc);
        note_launches(1);
    } else if (p->near_adj_rows == 1) {
        const NearAdjShape na = near_adj_shape(p);
        auto go = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)na.smem);
            kern<<<(unsigned)(na.ntx * na.nty), kNaThreads, na.smem, s>>>(
                p->ng, na.RX, na.RY, na.lz, na.ns, na.ntx, (uint32_t)na.o_sb, (uint32_t)na.o_meta,
                (uint32_t)na.o_acc32, (uint32_t)na.o_stage, p->dG, p->bin_start, p->bin_st,
                p->st_i0, p->st_j0, p->stz, p->near_tpart, p->ctx->d_status);
        };
        switch (na.ks) {
            case 4: go(k_near_adj_rows<4>); break;
            case 8: go(k_near_adj_rows<8>); break;
            case 12: go(k_near_adj_rows<12>); break;
            case 16: go(k_near_adj_rows<16>); break;
            default: go(k_near_adj_rows<kNaMaxKs>); break;
        }
        const int64_t cells = (int64_t)p->nx * p->ny * lz;
        k_near_adj_gather<<<grid_for(cells, 256), 256, 0, s>>>(p->nx, p->ny, lz, p->ng.bx, p->ng.by, na.RX, na.RY,
                                                               na.ntx, kNaTile, p->near_tpart, p->m_cellacc);
        note_launches(1);
    } else {
        dim3 gna((unsigned)((p->nx + 31) / 32), (unsigned)((p->ny + 7) / 8), (unsigned)lz);
        k_near_adj<<<gna, 256, 0, s>>>(p->nx, p->ny, p->ng, p->dG, p->bin_start, p->bin_st, p->st_i0, p->stz,
                                       p->m_cellacc);
    }
    stage_end(p, kStageAdjNear, s);
    note_launches(2);
}

void launch_mixed_adj_finish(const grav_plan *p, const double *r, int depth_weighted, const double *add,
                             double *out, cudaStream_t s) {
    (void)r;
    k_madj_finish<<<grid_for(p->M, 256), 256, 0, s>>>(p->nx, p->ny, p->nz, std::min(p->ng.bz, p->nz), p->m_apart,
                                                      p->m_adj_nschunk,
                                                      p->rmax_bits,
                                                      kGammaMgal * p->cell_a * p->cell_b * p->cell_c, p->m_cellacc,
                                                      depth_weighted ? p->d_w2 : nullptr, add, out);
    note_launches(1);
}

void launch_mixed_diag(const grav_plan *p, double *diag, cudaStream_t s) {
    const int tiles = (int)((p->N + kMfThreads * kMfT - 1) / (kMfThreads * kMfT));
    dim3 grid(tiles, p->m_fwd_nchunk);
    if (p->cubic)
        k_mdiag<kMfT, false><<<grid, kMfThreads, 0, s>>>(p->mg, p->m_w2f, p->st32, p->stz, p->m_fwd_cols_per_chunk,
                                                         p->m_part);
    else
        k_mdiag<kMfT, true><<<grid, kMfThreads, 0, s>>>(p->mg, p->m_w2f, p->st32, p->stz, p->m_fwd_cols_per_chunk,
                                                        p->m_part);
    note_launches(1);
    const double v = kGammaMgal * p->cell_a * p->cell_b * p->cell_c;
    launch_reduce_rows(p->m_part, p->m_fwd_nchunk, p->N, v * v, nullptr, 0.0, p->diag_corr, diag, s);
}

}  // namespace grav
