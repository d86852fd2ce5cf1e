// FP64 node-shared prism-gravity operator (GRAV_FP64).
//
// Summation by parts of Eq. 1 + Eq. 5: the 8-corner parity sum of every cell
// is regrouped per mesh node, so the corner function Psi (Eq. 2-3) is
// evaluated ONCE per (station, node) instead of once per (station, cell,
// corner):
//     d_i    = gamma * sum_n Psi(n - s_i) w_n,   w_n = sum_{cells k at n} sigma(n,k) m_k
//     (G^T r)_k = gamma * sum_{n corner of k} sigma(n,k) u_n,   u_n = sum_i Psi(n - s_i) r_i
// with sigma(n,k) = (-1)^(p+q+r) and p = 1 (2) when n is the lower (upper)
// x-vertex of cell k (same for q along y, r along z).  w is the mixed third
// difference of the zero-padded density; D^T is its transpose.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace grav {

namespace {

constexpr int kFwdThreads = 128;
constexpr int kFwdT = 2;            // stations per thread
constexpr int kFwdSmemLimit = 200 * 1024;   // dynamic shared memory k_fwd64 may use
constexpr int kAdjWarps = 8;        // warps per CTA in the adjoint
constexpr int kAdjTZ = 8;           // node levels per warp
constexpr int kAdjStage = 256;      // stations per TMA stage
constexpr int kDiagZC = 4;          // cell layers per sweep in the diagonal kernel
constexpr int kDiagDfZC = 16;       // cell layers per sweep in the double-float diagonal kernel
constexpr int kDiagKMax = 7;        // cells per lane of the warp-per-station diagonal (nx <= 224)

// ---------------------------------------------------------------------------
// w = D m, laid out as node rows r = b + (ny+1) c of ldw doubles (x fastest,
// entries a > nx are zero padding so that every row starts 16-byte aligned).
// ---------------------------------------------------------------------------
__global__ void k_node_weights(int nx, int ny, int nz, int ldw, const double *__restrict__ m,
                               double *__restrict__ w) {
    const int64_t rows = (int64_t)(ny + 1) * (nz + 1);
    const int64_t total = rows * ldw;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t % ldw);
        const int64_t r = t / ldw;
        const int b = (int)(r % (ny + 1));
        const int c = (int)(r / (ny + 1));
        double acc = 0.0;
        if (a <= nx) {
#pragma unroll
            for (int dc = 0; dc < 2; ++dc) {
                const int l = c - dc;
                if (l < 0 || l >= nz) continue;
#pragma unroll
                for (int db = 0; db < 2; ++db) {
                    const int j = b - db;
                    if (j < 0 || j >= ny) continue;
#pragma unroll
                    for (int da = 0; da < 2; ++da) {
                        const int i = a - da;
                        if (i < 0 || i >= nx) continue;
                        // node = cell vertex (i+da, j+db, l+dc): sigma = (-1)^(da+db+dc+3)
                        const double v = m[i + (int64_t)nx * (j + (int64_t)ny * l)];
                        acc += ((da + db + dc) & 1) ? v : -v;
                    }
                }
            }
        }
        w[t] = acc;
    }
}

// ---------------------------------------------------------------------------
// Forward: CTA = (station tile of kFwdThreads*T stations, chunk of node rows).
// Node-weight rows stream through shared memory by 1D TMA bulk copies
// (double-buffered, mbarrier-completed); stations stay in registers; every
// thread reads the same node (shared-memory broadcast).  Zero node weights are
// skipped (warp-uniform branch: every lane sees the same node).
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(kFwdThreads) k_fwd64(Geo g, int ldw, const double *__restrict__ w,
                                                       int rows_per_chunk, int rows_per_stage,
                                                       const double *__restrict__ sx,
                                                       const double *__restrict__ sy,
                                                       const double *__restrict__ sz,
                                                       double *__restrict__ part, int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    int *flag = reinterpret_cast<int *>(smem_raw + 16);
    double *Xs = reinterpret_cast<double *>(smem_raw + 128);
    double *wbuf = Xs + ldw;

    const int nrows = (g.ny + 1) * (g.nz + 1);
    const int r0 = blockIdx.y * rows_per_chunk;
    const int r1 = min(nrows, r0 + rows_per_chunk);
    const int nst = (r1 > r0) ? (r1 - r0 + rows_per_stage - 1) / rows_per_stage : 0;

    const int64_t s_base = (int64_t)blockIdx.x * (kFwdThreads * T) + threadIdx.x;
    // a warp whose first station is past N has no station at all (t adds
    // whole CTAs of threads): it skips the evaluation and only keeps the
    // CTA's barriers (surveys of a few stations, e.g. the FP64 error check)
    const bool live = s_base - (threadIdx.x & 31) < g.N;
    double xs[T], ys[T], zs[T], acc[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t s = s_base + (int64_t)t * kFwdThreads;
        const bool ok = s < g.N;
        xs[t] = ok ? sx[s] : 0.0;
        ys[t] = ok ? sy[s] : 0.0;
        zs[t] = ok ? sz[s] : g.ze[0] - 1.0;
        acc[t] = 0.0;
    }
    for (int a = threadIdx.x; a < ldw; a += kFwdThreads) Xs[a] = (a <= g.nx) ? g.xe[a] : 0.0;
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
        const uint32_t bytes = (uint32_t)(rb - ra) * (uint32_t)ldw * 8u;
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
        const double *wb = wbuf + (size_t)buf * rows_per_stage * ldw;
        const int ra = r0 + st * rows_per_stage;
        const int rb = min(r1, ra + rows_per_stage);
        for (int r = ra; live && r < rb; ++r) {
            const int b = r % (g.ny + 1);
            const int c = r / (g.ny + 1);
            const double Yb = g.ye[b], Zc = g.ze[c];
            double dy[T], dz[T], y2[T], z2[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                dy[t] = Yb - ys[t];
                dz[t] = Zc - zs[t];
                y2[t] = dy[t] * dy[t];
                z2[t] = dz[t] * dz[t];
            }
            const double *wr = wb + (size_t)(r - ra) * ldw;
            for (int a = 0; a <= g.nx; ++a) {
                const double wv = wr[a];
                if (wv == 0.0) continue;
                const double xa = Xs[a];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const double dx = xa - xs[t];
                    acc[t] = fma(wv, psi64(dx, dy[t], dz[t], dx * dx, y2[t], z2[t], g.fn), acc[t]);
                }
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
        const int64_t s = s_base + (int64_t)t * kFwdThreads;
        if (s < g.N) part[(int64_t)blockIdx.y * g.N + s] = acc[t];
    }
}

// out[i] = scale * sum_c part[c][i] + add_scale * add[i] + add2[i]  (fixed order)
// One CTA per 32 consecutive rows i: lane = row, the 8 warps split the
// chunks c (warp w sums c = w, w + 8, ...; each load is 32 consecutive
// doubles), then warp 0 adds the 8 warp sums in order: deterministic, and
// parallel over chunks as well as rows (surveys of a few thousand stations
// have thousands of forward chunks).
constexpr int kRedWarps = 8;
__global__ void __launch_bounds__(kRedWarps * 32) k_reduce_rows(const double *__restrict__ part, int nchunk, int64_t n,
                                                              double scale, const double *__restrict__ add,
                                                              double add_scale, const double *__restrict__ add2,
                                                              const unsigned long long *__restrict__ fbits,
                                                              double *__restrict__ out) {
    __shared__ double ws[kRedWarps][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    double s = 0.0;
    if (i < n)
        for (int c = warp; c < nchunk; c += kRedWarps) s += part[(int64_t)c * n + i];
    ws[warp][lane] = s;
    __syncthreads();
    if (warp != 0 || i >= n) return;
    s = ws[0][lane];
#pragma unroll
    for (int w = 1; w < kRedWarps; ++w) s += ws[w][lane];
    s *= scale;
    if (add2) s += add2[i];
    if (fbits) s *= __longlong_as_double((long long)*fbits);
    if (add) s = fma(add_scale, add[i], s);
    out[i] = s;
}

// st4[s].w = r[s]
__global__ void k_set_r(double4_16a *__restrict__ st4, const double *__restrict__ r, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        st4[i].w = r[i];
}

__global__ void k_init_st4(double4_16a *__restrict__ st4, const double *__restrict__ x, const double *__restrict__ y,
                           const double *__restrict__ z, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        st4[i] = make_double4_16a(x[i], y[i], z[i], 0.0);
}

// ---------------------------------------------------------------------------
// Adjoint: u_n = sum_i Psi(n - s_i) r_i.  A warp owns TZ nodes of one node
// column (a, b) at levels c0..c0+TZ-1; its 32 lanes split the stations of the
// CTA's station chunk (staged in shared memory by TMA), each lane accumulates
// its own stations, and a warp-shuffle butterfly reduces the 32 lane partials
// per node at the end (fixed order: deterministic).
// ---------------------------------------------------------------------------
template <int TZ>
__global__ void __launch_bounds__(kAdjWarps * 32) k_adj64(Geo g, const double4_16a *__restrict__ st4,
                                                          int64_t schunk_len, double *__restrict__ upart,
                                                          int64_t Nn, int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    int *flag = reinterpret_cast<int *>(smem_raw + 16);
    double4_16a *sbuf = reinterpret_cast<double4_16a *>(smem_raw + 128);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ngz = (g.nz + 1 + TZ - 1) / TZ;
    const int64_t ncolumns = (int64_t)(g.nx + 1) * (g.ny + 1);
    const int64_t group = (int64_t)blockIdx.x * kAdjWarps + warp;
    const bool gvalid = group < ncolumns * ngz;
    const int64_t col = gvalid ? group / ngz : 0;
    const int c0 = gvalid ? (int)(group % ngz) * TZ : 0;
    const int a = (int)(col % (g.nx + 1));
    const int b = (int)(col / (g.nx + 1));
    const double Xa = g.xe[a], Yb = g.ye[b];
    double Zt[TZ], acc[TZ];
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        Zt[t] = g.ze[min(c0 + t, g.nz)];
        acc[t] = 0.0;
    }

    const int64_t s0 = (int64_t)blockIdx.y * schunk_len;
    const int64_t s1 = min(g.N, s0 + schunk_len);
    const int nst = (s1 > s0) ? (int)((s1 - s0 + kAdjStage - 1) / kAdjStage) : 0;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int st) {
        const int buf = st & 1;
        const int64_t sa = s0 + (int64_t)st * kAdjStage;
        const int cnt = (int)min((int64_t)kAdjStage, s1 - sa);
        const uint32_t bytes = (uint32_t)cnt * 32u;
        mbar_arrive_expect_tx(&bar[buf], bytes);
        tma_load_1d(sbuf + buf * kAdjStage, st4 + sa, bytes, &bar[buf]);
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
        const int64_t sa = s0 + (int64_t)st * kAdjStage;
        const int cnt = (int)min((int64_t)kAdjStage, s1 - sa);
        const double4_16a *sb = sbuf + buf * kAdjStage;
        if (gvalid) {
            for (int k = lane; k < cnt; k += 32) {
                const double4_16a S = sb[k];
                if (S.w == 0.0) continue;
                const double dx = Xa - S.x, dy = Yb - S.y;
                const double x2 = dx * dx, y2 = dy * dy;
#pragma unroll
                for (int t = 0; t < TZ; ++t) {
                    const double dz = Zt[t] - S.z;
                    acc[t] = fma(S.w, psi64(dx, dy, dz, x2, y2, dz * dz, g.fn), acc[t]);
                }
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
        const double v = warp_sum(acc[t]);
        if (lane == t % 32 && c0 + t <= g.nz)
            upart[(int64_t)blockIdx.y * Nn + a + (int64_t)(g.nx + 1) * (b + (int64_t)(g.ny + 1) * (c0 + t))] = v;
    }
}

// out[k] = scale * sum_{8 corners n of k} sigma(n,k) u_n  [* (zc_l + z0)^2]  [+ add[k]]
__global__ void k_adj_finish(int nx, int ny, int nz, const double *__restrict__ u, double scale,
                             const double *__restrict__ w2, const double *__restrict__ add,
                             double *__restrict__ out) {
    const int64_t M = (int64_t)nx * ny * nz;
    const int64_t sx = 1, sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx);
        const int j = (int)((k / nx) % ny);
        const int l = (int)(k / ((int64_t)nx * ny));
        const int64_t n0 = i + sy * j + sz * l;
        // sigma = -(-1)^(da+db+dc)
        const double v = -u[n0] + u[n0 + sx] + u[n0 + sy] - u[n0 + sx + sy] + u[n0 + sz] - u[n0 + sx + sz] -
                         u[n0 + sy + sz] + u[n0 + sx + sy + sz];
        double o = scale * v;
        if (w2) o *= w2[l];
        if (add) o += add[k];
        out[k] = o;
    }
}

// ---------------------------------------------------------------------------
// diag_i = sum_k G_ik^2 (zc_k + z0)^2 in FP64.  Thread = station; grid.y =
// ranges of y-rows of cells.  Along x the right node column of one cell is the
// left node column of the next, so each step evaluates Psi on 2 new node
// columns (levels l0..l0+ZC) for ZC cells: 2(ZC+1)/ZC evaluations per cell.
// ---------------------------------------------------------------------------
template <int ZC, bool WRITE_G>
__global__ void __launch_bounds__(128) k_diag64(Geo g, const double *__restrict__ w2, int jrows,
                                                const double *__restrict__ sx, const double *__restrict__ sy,
                                                const double *__restrict__ sz, double *__restrict__ part,
                                                float2 *__restrict__ Gout) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.N) return;
    const double xs = sx[s], ys = sy[s], zs = sz[s];
    const int j0 = blockIdx.y * jrows;
    const int j1 = min(g.ny, j0 + jrows);
    double acc = 0.0;
    for (int j = j0; j < j1; ++j) {
        const double dy0 = g.ye[j] - ys, dy1 = g.ye[j + 1] - ys;
        const double y20 = dy0 * dy0, y21 = dy1 * dy1;
        for (int l0 = 0; l0 < g.nz; l0 += ZC) {
            const int nl = min(ZC, g.nz - l0);
            double dz[ZC + 1], z2[ZC + 1], w2l[ZC];
#pragma unroll
            for (int c = 0; c <= ZC; ++c) {
                dz[c] = g.ze[l0 + min(c, nl)] - zs;
                z2[c] = dz[c] * dz[c];
            }
#pragma unroll
            for (int c = 0; c < ZC; ++c) w2l[c] = w2[l0 + min(c, nl - 1)];
            double P0[ZC + 1], P1[ZC + 1];
            {
                const double dx = g.xe[0] - xs, x2 = dx * dx;
#pragma unroll
                for (int c = 0; c <= ZC; ++c) {
                    P0[c] = (c <= nl) ? psi64(dx, dy0, dz[c], x2, y20, z2[c], g.fn) : 0.0;
                    P1[c] = (c <= nl) ? psi64(dx, dy1, dz[c], x2, y21, z2[c], g.fn) : 0.0;
                }
            }
            for (int i = 0; i < g.nx; ++i) {
                const double dx = g.xe[i + 1] - xs, x2 = dx * dx;
                double E[ZC + 1];
#pragma unroll
                for (int c = 0; c <= ZC; ++c) {
                    double q0 = 0.0, q1 = 0.0;
                    if (c <= nl) {
                        q0 = psi64(dx, dy0, dz[c], x2, y20, z2[c], g.fn);
                        q1 = psi64(dx, dy1, dz[c], x2, y21, z2[c], g.fn);
                    }
                    E[c] = P0[c] - q0 - P1[c] + q1;
                    P0[c] = q0;
                    P1[c] = q1;
                }
#pragma unroll
                for (int c = 0; c < ZC; ++c) {
                    if (c < nl) {
                        const double G = kGammaMgal * (E[c + 1] - E[c]);
                        acc = fma(G * G, w2l[c], acc);
                        if (WRITE_G) {   // the FP64 value as a double-float pair (48-bit significand)
                            const float gh = __double2float_rn(G);
                            Gout[(i + (int64_t)g.nx * (j + (int64_t)g.ny * (l0 + c))) * g.N + s] =
                                make_float2(gh, __double2float_rn(G - (double)gh));
                        }
                    }
                }
            }
        }
    }
    part[(int64_t)blockIdx.y * g.N + s] = acc;
}

// The same diagonal with a warp per station: lane l owns the K cells
// l K .. l K + K - 1 along x (K = ceil(nx / 32) <= KMAX) and keeps Psi at its
// K + 1 x nodes on the previous y edge (levels l0..l0+ZC) in registers, so a
// node is evaluated once per layer group instead of once per y edge of each
// of its two rows: (K + 1)/K (ZC + 1)/ZC evaluations per cell (1.43 at
// nx = 210, against 2.5 for the thread-per-station form).  Same differences
// of Psi in another order.
template <int ZC, int KMAX>
__global__ void __launch_bounds__(128) k_diag64w(Geo g, const double *__restrict__ w2, int jrows,
                                                 const double *__restrict__ sx, const double *__restrict__ sy,
                                                 const double *__restrict__ sz, double *__restrict__ part) {
    // Psi on the previous y edge, [warp][node a][level c][lane] (lane fastest: conflict-free)
    __shared__ double prev_s[4][KMAX + 1][ZC + 1][32];
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (s >= g.N) return;   // warp-uniform
    double(*prev)[ZC + 1][32] = prev_s[wid];
    const double xs = sx[s], ys = sy[s], zs = sz[s];
    const int K = (g.nx + 31) / 32;   // cells per lane (<= KMAX, checked by the launcher)
    const int a0 = lane * K;          // first x node of this lane
    const int j0 = blockIdx.y * jrows;
    const int j1 = min(g.ny, j0 + jrows);
    double acc = 0.0;
    for (int l0 = 0; l0 < g.nz; l0 += ZC) {
        const int nl = min(ZC, g.nz - l0);
        double dz[ZC + 1], z2[ZC + 1], w2l[ZC];
#pragma unroll
        for (int c = 0; c <= ZC; ++c) {
            dz[c] = g.ze[l0 + min(c, nl)] - zs;
            z2[c] = dz[c] * dz[c];
        }
#pragma unroll
        for (int c = 0; c < ZC; ++c) w2l[c] = w2[l0 + min(c, nl - 1)];
        {
            const double dy = g.ye[j0] - ys, y2 = dy * dy;
            for (int a = 0; a <= K; ++a) {
                const bool ok = a0 + a <= g.nx;
                const double dx = g.xe[min(a0 + a, g.nx)] - xs, x2 = dx * dx;
#pragma unroll
                for (int c = 0; c <= ZC; ++c)
                    prev[a][c][lane] = (ok && c <= nl) ? psi64(dx, dy, dz[c], x2, y2, z2[c], g.fn) : 0.0;
            }
        }
        for (int j = j0; j < j1; ++j) {
            const double dy = g.ye[j + 1] - ys, y2 = dy * dy;
            double eprev[ZC + 1];
            for (int a = 0; a <= K; ++a) {
                const bool ok = a0 + a <= g.nx;
                const double dx = g.xe[min(a0 + a, g.nx)] - xs, x2 = dx * dx;
                double ey[ZC + 1];
#pragma unroll
                for (int c = 0; c <= ZC; ++c) {
                    const double v = (ok && c <= nl) ? psi64(dx, dy, dz[c], x2, y2, z2[c], g.fn) : 0.0;
                    ey[c] = v - prev[a][c][lane];   // y difference at node a
                    prev[a][c][lane] = v;
                }
                if (a >= 1 && ok) {   // cell a0 + a - 1
#pragma unroll
                    for (int c = 0; c < ZC; ++c)
                        if (c < nl) {
                            const double G = kGammaMgal * ((ey[c + 1] - eprev[c + 1]) - (ey[c] - eprev[c]));
                            acc = fma(G * G, w2l[c], acc);
                        }
                }
#pragma unroll
                for (int c = 0; c <= ZC; ++c) eprev[c] = ey[c];
            }
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) part[(int64_t)blockIdx.y * g.N + s] = acc;
}

// The diagonal with the corner function in double-float (psi_df: pairs of
// FP32 numbers on the FP32 pipe, 64x the FP64 rate here; ~2^-45 of
// R (|ln R| + 1) per node value).  A diagonal entry is a sum of squares, so
// the per-node errors do not meet the node-shared products' cancellation
// across the mesh: emulated at that error bound they move an entry by
// ~1e-13 of its value (tested against the FP64 kernel and the oracle).
// A warp per station: lane t holds x node a0 + t of a 32-node segment and
// owns the cell a0 + t (lanes 0..30), whose right node comes from lane t + 1
// by a shuffle; Psi of the lane's node on the previous y edge, at the ZC + 1
// levels of a layer group, is kept in shared memory (lane fastest).
// Evaluations per cell: (32/31) ((ZC + 1)/ZC) (1 + 1/rows).  Differences in
// the order of k_diag64w (y, then x, then z; adjacent nodes first, so each
// cancellation is exact in TwoSum); G^2 w2 is summed in double-float over a
// sweep (segment x layer group x rows) and folded into FP64 per sweep.  The
// y offsets of 32 rows are split by the lanes and broadcast by shuffles, and
// the levels' offsets and weights sit in shared memory, so no FP64
// operation runs per node.  The level loop is not unrolled (one inlined
// corner function keeps the loop body in the instruction cache).
template <int ZC>
__global__ void __launch_bounds__(128) k_diagdf(Geo g, const double *__restrict__ w2, int jrows,
                                                const double *__restrict__ sx, const double *__restrict__ sy,
                                                const double *__restrict__ sz, double *__restrict__ part) {
    __shared__ float2 zw_s[4][2 * ZC + 1];    // per warp: level offsets (ZC + 1), then w2 of the ZC layers
    __shared__ float2 prev_s[4][ZC + 1][32];  // per warp: Psi on the previous y edge [level][lane]
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (s >= g.N) return;   // warp-uniform
    float2 *zw = zw_s[wid];
    float2(*prev)[32] = prev_s[wid];
    const float *D = reinterpret_cast<const float *>(g.fn + kFnDf);
    const double xs = sx[s], ys = sy[s], zs = sz[s];
    const int j0 = blockIdx.y * jrows;
    const int j1 = min(g.ny, j0 + jrows);
    const df32 gam = df_from_double(kGammaMgal);
    const unsigned full = 0xffffffffu;
    double acc = 0.0;
    for (int a0 = 0; a0 < g.nx; a0 += 31) {
        const int a = min(a0 + lane, g.nx);   // lanes past the last node repeat it (their values are not used)
        const bool own = lane < 31 && a0 + lane < g.nx;
        const df32 X = df_from_double(g.xe[a] - xs);
        for (int l0 = 0; l0 < g.nz; l0 += ZC) {
            const int nl = min(ZC, g.nz - l0);
            __syncwarp();
            for (int u = lane; u <= 2 * ZC; u += 32) {   // 2 ZC + 1 entries (more than a warp for ZC >= 16)
                const df32 v = u <= ZC ? df_from_double(g.ze[l0 + min(u, nl)] - zs)
                                       : df_from_double(w2[l0 + min(u - ZC - 1, nl - 1)]);
                zw[u] = make_float2(v.hi, v.lo);
            }
            __syncwarp();
            {
                const df32 Y = df_from_double(g.ye[j0] - ys);
#pragma unroll 1
                for (int c = 0; c <= nl; ++c) {
                    const float2 z = zw[c];
                    const df32 v = psi_df(X, Y, df_make(z.x, z.y), D);
                    prev[c][lane] = make_float2(v.hi, v.lo);
                }
            }
            df32 sacc = df_make(0.0f, 0.0f);
            for (int jb = j0; jb < j1; jb += 32) {
                const df32 Yl = df_from_double(g.ye[min(jb + 1 + lane, g.ny)] - ys);   // edge jb + 1 + lane
                const int nrow = min(32, j1 - jb);
                for (int r = 0; r < nrow; ++r) {
                    const df32 Y = df_make(__shfl_sync(full, Yl.hi, r), __shfl_sync(full, Yl.lo, r));
                    df32 exl = df_make(0.0f, 0.0f);   // x difference at the level below
#pragma unroll 1
                    for (int c = 0; c <= nl; ++c) {
                        const float2 z = zw[c];
                        const df32 v = psi_df(X, Y, df_make(z.x, z.y), D);
                        const float2 pv = prev[c][lane];
                        prev[c][lane] = make_float2(v.hi, v.lo);
                        const df32 ey = df_sub(v, df_make(pv.x, pv.y));   // y difference at this lane's node
                        const df32 er = df_make(__shfl_down_sync(full, ey.hi, 1), __shfl_down_sync(full, ey.lo, 1));
                        const df32 ex = df_sub(er, ey);                    // then x: right node minus left
                        if (c >= 1 && own) {                               // cell layer l0 + c - 1: then z
                            const df32 G = df_mul(df_sub(ex, exl), gam);
                            const float2 wv = zw[ZC + c];
                            sacc = df_add(sacc, df_mul(df_sqr(G), df_make(wv.x, wv.y)));
                        }
                        exl = ex;
                    }
                }
            }
            acc += df_to_double(sacc);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) part[(int64_t)blockIdx.y * g.N + s] = acc;
}

inline int grid_for(int64_t n, int threads, int cap = 148 * 32) {
    int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}


int fwd_rows_per_stage(const grav_plan *p) {
    // ~16 KB of node weights per stage
    return std::max(1, std::min(p->f64_rows_per_chunk, (16384 / 8) / p->ldw));
}

// ---------------------------------------------------------------------------
// Stored-G products (G formed once in FP64 with node-shared differencing,
// cell-major Gc[k][i], station i fastest).  An FP64 GEMV on this GPU is
// bound by the FP64 pipe, not by HBM: one DFMA per 8-byte entry at
// 1.65 DFMA/clk/SM is 4.96e11 entries/s against HBM's 8.1e11 (measured:
// FP64 pipe 93-96 % busy, DRAM 57 %).  G is therefore kept as double-float
// pairs (hi, lo FP32: the FP64 value to a 48-bit significand, same 8 bytes)
// and the products run in double-float arithmetic on the FP32 pipe (~18
// FP32 operations per entry, 64x the FP64 rate), which leaves HBM the bound.
// The input vector is split into pairs once per product (k_split_df).
// d: CTA = (128 stations, chunk of cells) -> FP64 partials [chunk][N].
// G^T r: warp per cell, lanes over stations, FP64 shuffle reduction.
// ---------------------------------------------------------------------------
__global__ void k_split_df(const double *__restrict__ x, int64_t n, float2 *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        const float h = __double2float_rn(v);
        y[i] = make_float2(h, __double2float_rn(v - (double)h));
    }
}

__device__ __forceinline__ df32 df_of(float2 v) { return df_make(v.x, v.y); }

// d partials: CTA = 4,096 consecutive stations (thread t: t + 256 j, j < 16)
// x a chunk of cells, so each row of G is read as one 32 KB contiguous run
// with 16 independent loads per thread; double-float sums in registers, each
// station's cells in order.
constexpr int kGfJ = 16;
constexpr int kGfTile = 256 * kGfJ;
__global__ void __launch_bounds__(256) k_gemv_cached(const float2 *__restrict__ Gc, int64_t N, int64_t M,
                                                     int64_t cells_per_chunk, const float2 *__restrict__ m,
                                                     double *__restrict__ part) {
    const int64_t ib = (int64_t)blockIdx.x * kGfTile + threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * cells_per_chunk;
    const int64_t k1 = min(M, k0 + cells_per_chunk);
    df32 a[kGfJ];
#pragma unroll
    for (int j = 0; j < kGfJ; ++j) a[j] = df_make(0.0f, 0.0f);
    for (int64_t k = k0; k < k1; ++k) {
        const float2 *row = Gc + k * N;
        const df32 mk = df_of(m[k]);
        float2 g[kGfJ];
#pragma unroll
        for (int j = 0; j < kGfJ; ++j) {
            const int64_t i = ib + 256 * j;
            g[j] = i < N ? row[i] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int j = 0; j < kGfJ; ++j) a[j] = df_add(a[j], df_mul(df_of(g[j]), mk));
    }
#pragma unroll
    for (int j = 0; j < kGfJ; ++j) {
        const int64_t i = ib + 256 * j;
        if (i < N) part[(int64_t)blockIdx.y * N + i] = df_to_double(a[j]);
    }
}

// sum_k G_ik^2 w2[layer(k)] (the diagonal of G W^-2 G^T), once per plan: FP64
__global__ void __launch_bounds__(128) k_gemv_cached_sq(const float2 *__restrict__ Gc, int64_t N, int64_t M,
                                                        int64_t plane, int64_t cells_per_chunk,
                                                        const double *__restrict__ w2, double *__restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * cells_per_chunk;
    const int64_t k1 = min(M, k0 + cells_per_chunk);
    if (i >= N) return;
    double a = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
        const float2 gv = Gc[k * N + i];
        const double g = (double)gv.x + (double)gv.y;
        a = fma(g * g, w2[k / plane], a);
    }
    part[(int64_t)blockIdx.y * N + i] = a;
}

__global__ void __launch_bounds__(256) k_gemvt_cached(const float2 *__restrict__ Gc, int64_t N, int64_t M, int nx,
                                                      int ny, const float2 *__restrict__ r,
                                                      const double *__restrict__ w2, const double *__restrict__ add,
                                                      double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= M) return;
    const float2 *row = Gc + k * N;
    df32 a = df_make(0.0f, 0.0f);
    for (int64_t i = lane; i < N; i += 32) a = df_add(a, df_mul(df_of(row[i]), df_of(r[i])));
    double s = warp_sum(df_to_double(a));
    if (lane == 0) {
        if (w2) s *= w2[k / ((int64_t)nx * ny)];
        if (add) s += add[k];
        out[k] = s;
    }
}

}  // namespace

int cached_fwd_tiles(int64_t N) { return (int)((N + kGfTile - 1) / kGfTile); }

int cached_fwd_ctas_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gemv_cached, 256, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

void launch_build_g64(const grav_plan *p, float2 *Gc, double *diag, cudaStream_t s) {
    const int tiles = (int)((p->N + 127) / 128);
    dim3 grid(tiles, p->f64_diag_nchunk);
    k_diag64<kDiagZC, true><<<grid, 128, 0, s>>>(make_geo(p), p->d_w2, p->f64_diag_jrows, p->sx, p->sy, p->sz,
                                                 p->part, Gc);
    note_launches(1);
    if (diag) launch_reduce_rows(p->part, p->f64_diag_nchunk, p->N, 1.0, nullptr, 0.0, nullptr, diag, s);
}

void launch_cached_fwd(const grav_plan *p, const double *m, const double *add, double add_scale, double *d,
                       cudaStream_t s) {
    const int64_t per = (p->M + p->c_nchunk - 1) / p->c_nchunk;
    dim3 grid((unsigned)cached_fwd_tiles(p->N), (unsigned)p->c_nchunk);
    stage_begin(p, kStageFwdMain, s);
    k_split_df<<<grid_for(p->M, 256), 256, 0, s>>>(m, p->M, p->m_df);
    k_gemv_cached<<<grid, 256, 0, s>>>(p->Gc, p->N, p->M, per, p->m_df, p->part);
    stage_end(p, kStageFwdMain, s);
    note_launches(2);
    launch_reduce_rows(p->part, p->c_nchunk, p->N, 1.0, add, add_scale, nullptr, d, s);
}

void launch_cached_diag(const grav_plan *p, double *diag, cudaStream_t s) {
    const int64_t per = (p->M + p->c_nchunk - 1) / p->c_nchunk;
    dim3 grid((unsigned)((p->N + 127) / 128), (unsigned)p->c_nchunk);
    k_gemv_cached_sq<<<grid, 128, 0, s>>>(p->Gc, p->N, p->M, (int64_t)p->nx * p->ny, per, p->d_w2, p->part);
    note_launches(1);
    launch_reduce_rows(p->part, p->c_nchunk, p->N, 1.0, nullptr, 0.0, nullptr, diag, s);
}

void launch_cached_adj(const grav_plan *p, const double *r, int depth_weighted, const double *add, double *out,
                       cudaStream_t s) {
    const int64_t threads = p->M * 32;
    stage_begin(p, kStageAdjMain, s);
    k_split_df<<<grid_for(p->N, 256), 256, 0, s>>>(r, p->N, p->r_df);
    k_gemvt_cached<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(p->Gc, p->N, p->M, p->nx, p->ny, p->r_df,
                                                                    depth_weighted ? p->d_w2 : nullptr, add, out);
    stage_end(p, kStageAdjMain, s);
    note_launches(2);
}

size_t fwd64_smem_bytes(const grav_plan *p) {
    return 128 + (size_t)p->ldw * 8 + 2ull * fwd_rows_per_stage(p) * p->ldw * 8;
}

void launch_node_weights(const grav_plan *p, const double *m, cudaStream_t s) {
    const int64_t total = (int64_t)(p->ny + 1) * (p->nz + 1) * p->ldw;
    k_node_weights<<<grid_for(total, 256), 256, 0, s>>>(p->nx, p->ny, p->nz, p->ldw, m, p->w);
    note_launches(1);
}

void fp64_setup(grav_plan *p, cudaStream_t s) {
    k_init_st4<<<grid_for(p->N, 256), 256, 0, s>>>(p->st4, p->sx, p->sy, p->sz, p->N);
    cudaFuncSetAttribute(k_fwd64<kFwdT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmemLimit);
}

void launch_fwd64(const grav_plan *p, cudaStream_t s) {
    const int tiles = (int)((p->N + kFwdThreads * kFwdT - 1) / (kFwdThreads * kFwdT));
    dim3 grid(tiles, p->f64_nchunk);
    const size_t smem = fwd64_smem_bytes(p);
    stage_begin(p, kStageFwdMain, s);
    k_fwd64<kFwdT><<<grid, kFwdThreads, smem, s>>>(make_geo(p), p->ldw, p->w, p->f64_rows_per_chunk,
                                                   fwd_rows_per_stage(p), p->sx, p->sy, p->sz, p->part,
                                                   p->ctx->d_status);
    stage_end(p, kStageFwdMain, s);
    note_launches(1);
}

void launch_reduce_rows(const double *part, int nchunk, int64_t n, double scale, const double *add,
                        double add_scale, const double *add2, double *out, cudaStream_t s,
                        const unsigned long long *fbits) {
    if (n <= 0) return;
    k_reduce_rows<<<(unsigned)((n + 31) / 32), kRedWarps * 32, 0, s>>>(part, nchunk, n, scale, add, add_scale, add2,
                                                                      fbits, out);
    note_launches(1);
}

void launch_adj64(const grav_plan *p, const double *r, cudaStream_t s) {
    k_set_r<<<grid_for(p->N, 256), 256, 0, s>>>(p->st4, r, p->N);
    dim3 grid((p->a64_groups + kAdjWarps - 1) / kAdjWarps, p->a64_nschunk);
    const size_t smem = 128 + 2ull * kAdjStage * sizeof(double4_16a);
    stage_begin(p, kStageAdjMain, s);
    k_adj64<kAdjTZ><<<grid, kAdjWarps * 32, smem, s>>>(make_geo(p), p->st4, p->a64_schunk_len, p->upart,
                                                       p->Nn, p->ctx->d_status);
    stage_end(p, kStageAdjMain, s);
    note_launches(2);
    launch_reduce_rows(p->upart, p->a64_nschunk, p->Nn, 1.0, nullptr, 0.0, nullptr, p->u, s);
}

void launch_adj_finish(const grav_plan *p, const double *u, double scale, int depth_weighted,
                       const double *add, double *out, cudaStream_t s) {
    k_adj_finish<<<grid_for(p->M, 256), 256, 0, s>>>(p->nx, p->ny, p->nz, u, scale,
                                                     depth_weighted ? p->d_w2 : nullptr, add, out);
    note_launches(1);
}

void launch_diag64(const grav_plan *p, double *diag, cudaStream_t s) {
    if (!p->opt.diag_fp64) {   // double-float corner function, warp per station
        // row chunks only as far as needed for >= 64 warps per SM: each chunk
        // evaluates its first y edge once more
        int64_t nch = std::max<int64_t>(1, (148LL * 64 + p->N - 1) / p->N);
        nch = std::min<int64_t>(nch, p->f64_diag_nchunk);
        const int jrows = (int)((p->ny + nch - 1) / nch);
        nch = (p->ny + jrows - 1) / jrows;
        dim3 grid((unsigned)((p->N + 3) / 4), (unsigned)nch);
        k_diagdf<kDiagDfZC><<<grid, 128, 0, s>>>(make_geo(p), p->d_w2, jrows, p->sx, p->sy, p->sz, p->part);
        note_launches(1);
        launch_reduce_rows(p->part, (int)nch, p->N, 1.0, nullptr, 0.0, nullptr, diag, s);
        return;
    }
    if (p->nx <= 32 * kDiagKMax) {   // warp per station (x nodes across the lanes)
        // row chunks only as far as needed for >= 64 warps per SM: each chunk
        // evaluates its first y edge once more
        int64_t nch = std::max<int64_t>(1, (148LL * 64 + p->N - 1) / p->N);
        nch = std::min<int64_t>(nch, p->f64_diag_nchunk);
        const int jrows = (int)((p->ny + nch - 1) / nch);
        nch = (p->ny + jrows - 1) / jrows;
        dim3 grid((unsigned)((p->N + 3) / 4), (unsigned)nch);
        k_diag64w<kDiagZC, kDiagKMax><<<grid, 128, 0, s>>>(make_geo(p), p->d_w2, jrows, p->sx, p->sy, p->sz, p->part);
        note_launches(1);
        launch_reduce_rows(p->part, (int)nch, p->N, 1.0, nullptr, 0.0, nullptr, diag, s);
        return;
    } else {
        const int tiles = (int)((p->N + 127) / 128);
        dim3 grid(tiles, p->f64_diag_nchunk);
        k_diag64<kDiagZC, false><<<grid, 128, 0, s>>>(make_geo(p), p->d_w2, p->f64_diag_jrows, p->sx, p->sy, p->sz,
                                                      p->part, nullptr);
    }
    note_launches(1);
    launch_reduce_rows(p->part, p->f64_diag_nchunk, p->N, 1.0, nullptr, 0.0, nullptr, diag, s);
}

}  // namespace grav

namespace grav {

// Raw-pointer launchers of the FP64 forward kernels for callers that manage
// their own scratch (no plan): node weights into w, per-chunk partials into
// part.  Returns the number of kernels launched.
int launch_fwd64_raw(Geo g, int ldw, const double *m, double *w, int rows_per_chunk, int nchunk,
                     const double *sx, const double *sy, const double *sz, double *part, int *status,
                     cudaStream_t s) {
    if (cudaFuncSetAttribute(k_fwd64<kFwdT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmemLimit) !=
        cudaSuccess)
        return -1;
    const int64_t total = (int64_t)(g.ny + 1) * (g.nz + 1) * ldw;
    k_node_weights<<<grid_for(total, 256), 256, 0, s>>>(g.nx, g.ny, g.nz, ldw, m, w);
    const int rps = std::max(1, std::min(rows_per_chunk, (16384 / 8) / ldw));
    const size_t smem = 128 + (size_t)ldw * 8 + 2ull * rps * ldw * 8;
    const int tiles = (int)((g.N + kFwdThreads * kFwdT - 1) / (kFwdThreads * kFwdT));
    dim3 grid(tiles, nchunk);
    k_fwd64<kFwdT><<<grid, kFwdThreads, smem, s>>>(g, ldw, w, rows_per_chunk, rps, sx, sy, sz, part, status);
    note_launches(2);
    return 2;
}

int fwd64_stations_per_cta() { return kFwdThreads * kFwdT; }

// 128 bytes of barriers + the x-edge row + two stage buffers of >= 1 row
// (rows of ldw doubles, ldw = nx+1 rounded up to even).
int fwd64_max_nodes_x() { return (kFwdSmemLimit - 128) / 24 / 2 * 2; }

}  // namespace grav

namespace grav {

// The one constructor of a plan's Geo (both kernel files use it): every field,
// the function table included, comes from the plan and its context.
Geo make_geo(const grav_plan *p) {
    Geo g;
    g.nx = p->nx; g.ny = p->ny; g.nz = p->nz;
    g.xe = p->d_xe; g.ye = p->d_ye; g.ze = p->d_ze;
    g.N = p->N;
    g.fn = p->ctx->d_fn;
    return g;
}

__global__ void k_gather_check(const double *__restrict__ sx, const double *__restrict__ sy,
                               const double *__restrict__ sz, const double *__restrict__ d, int64_t n, int n_check,
                               double *ox, double *oy, double *oz, double *od) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_check) return;
    const int64_t i = (int64_t)k * n / n_check;
    ox[k] = sx[i];
    oy[k] = sy[i];
    oz[k] = sz[i];
    od[k] = d[i];
}

void launch_gather_check(const double *sx, const double *sy, const double *sz, const double *d, int64_t n,
                         int n_check, double *ox, double *oy, double *oz, double *od, cudaStream_t s) {
    k_gather_check<<<(n_check + 127) / 128, 128, 0, s>>>(sx, sy, sz, d, n, n_check, ox, oy, oz, od);
    note_launches(1);
}

int fn_table_size() { return kFnTableSize; }

void fill_fn_table(double *t) {
    for (int i = 0; i < kFnTableSize; ++i) t[i] = 0.0;
    const long double grid = 4398046511104.0L;   // 2^42
    auto split42 = [&](long double v, double &hi, double &lo) {
        hi = (double)(nearbyintl(v * grid) / grid);
        lo = (double)(v - (long double)hi);
    };
    for (int j = 0; j <= kFnLogJ; ++j) {
        const long double F = 1.0L + (long double)j / kFnLogJ;
        t[kFnLog + 3 * j] = (double)(1.0L / F);
        split42(logl(F), t[kFnLog + 3 * j + 1], t[kFnLog + 3 * j + 2]);
    }
    split42(logl(2.0L), t[kFnLn2], t[kFnLn2 + 1]);
    const long double half_pi = 2.0L * atanl(1.0L);
    for (int j = 0; j <= kFnAtanJ; ++j) {
        const long double a = atanl((long double)j / kFnAtanJ);
        const long double b = half_pi - a;
        t[kFnAtan + 4 * j] = (double)a;
        t[kFnAtan + 4 * j + 1] = (double)(a - (long double)(double)a);
        t[kFnAtan + 4 * j + 2] = (double)b;
        t[kFnAtan + 4 * j + 3] = (double)(b - (long double)(double)b);
    }
    // double-float tables: each value as a high float and the float nearest
    // to the remainder
    float *f = reinterpret_cast<float *>(t + kFnDf);
    auto split32 = [&](long double v, float *out) {
        out[0] = (float)v;
        out[1] = (float)(v - (long double)out[0]);
    };
    for (int j = 0; j <= kDfLogJ; ++j) {
        const long double c = 1.0L + (long double)j / kDfLogJ;
        split32(logl(c), f + kDfLog + 4 * j);
        split32(1.0L / c, f + kDfLog + 4 * j + 2);
    }
    for (int j = 0; j <= kDfAtanJ; ++j) split32(atanl((long double)j / kDfAtanJ), f + kDfAtan + 2 * j);
    split32(logl(2.0L), f + kDfLn2);
    split32(half_pi, f + kDfPio2);
}

}  // namespace grav
