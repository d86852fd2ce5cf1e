// FP64 vector kernels of the data-space CG (Section 2.2, Eq. 11 solved
// iteratively as in Section 3.1): deterministic dot products (fixed grid,
// fixed per-thread ranges, fixed reduction trees), step lengths computed on
// the device, fused vector updates, and a device-side freeze flag so that
// iterations enqueued past convergence change nothing.
#include "cg.h"
#include "device_common.cuh"
#include "internal.h"

namespace grav {

namespace {

constexpr int kDotThreads = 256;

// partials[block] = sum over the block's fixed index set of a[i]*b[i] (b == nullptr: a[i])
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const double *__restrict__ a, const double *__restrict__ b,
                                                             int64_t n, double *__restrict__ partials) {
    __shared__ double ws[kDotThreads / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads)
        acc = b ? fma(a[i], b[i], acc) : acc + a[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kDotThreads / 32; ++w) s += ws[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_dot_final(const double *__restrict__ partials, int np, double *__restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += 32) s += partials[i];
    s = warp_sum(s);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_cg_alpha(double *__restrict__ sc) {
    const double pAp = sc[kSPAp];
    sc[kSAlpha] = (sc[kSFrozen] != 0.0 || !(pAp > 0.0)) ? 0.0 : sc[kSRR] / pAp;
    if (sc[kSFrozen] == 0.0 && !(pAp > 0.0)) sc[kSFrozen] = 2.0;   // breakdown: stop updating
}

__global__ void k_cg_update_yr(double *__restrict__ y, double *__restrict__ r, const double *__restrict__ p,
                               const double *__restrict__ Ap, int64_t n, const double *__restrict__ sc) {
    const double alpha = sc[kSAlpha];
    if (alpha == 0.0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        y[i] = fma(alpha, p[i], y[i]);
        r[i] = fma(-alpha, Ap[i], r[i]);
    }
}

// beta = rz_new / rz (rz = r.z, z = M^-1 r; z = r without preconditioner);
// convergence on the residual norm held in conv_slot.
__global__ void k_cg_beta(double *__restrict__ sc, int it, int conv_slot, double *__restrict__ hist, int hist_len) {
    if (sc[kSFrozen] != 0.0) {
        sc[kSBeta] = 0.0;
        return;
    }
    const double rz_new = sc[kSRRNew];
    sc[kSBeta] = rz_new / sc[kSRR];
    sc[kSRR] = rz_new;
    sc[kSIters] = (double)(it + 1);
    if (hist && it < hist_len) hist[it] = sqrt(sc[conv_slot] / sc[kSBB]);
    if (sc[conv_slot] <= sc[kSTol2] * sc[kSBB]) sc[kSFrozen] = 1.0;
}

__global__ void k_cg_update_p(double *__restrict__ p, const double *__restrict__ r, int64_t n,
                              const double *__restrict__ sc) {
    if (sc[kSFrozen] != 0.0) return;
    const double beta = sc[kSBeta];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}

// out = a*x + b*y (y may be null)
__global__ void k_axpby(double a, const double *__restrict__ x, double b, const double *__restrict__ y, int64_t n,
                        double *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = y ? fma(a, x[i], b * y[i]) : a * x[i];
}

__global__ void k_fill(double *__restrict__ x, int64_t n, double v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

__global__ void k_set_scalars(double *__restrict__ sc, double tol2, int bb_slot) {
    sc[kSBB] = sc[bb_slot];
    sc[kSTol2] = tol2;
    sc[kSFrozen] = (sc[kSBB] <= 0.0) ? 1.0 : 0.0;
    sc[kSIters] = 0.0;
}

__global__ void k_mul(const double *__restrict__ a, const double *__restrict__ b, int64_t n, double *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

__global__ void k_jacobi_inv(const double *__restrict__ diag, double lam, int64_t n, double *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = 1.0 / (diag[i] + lam);
}

// restart from the true residual whose r.r is in kSTmp: unfreeze unless it is
// already below tol; without preconditioner rz = r.r (copy_rr), with one the
// caller has put r.z in kSRR.
__global__ void k_cg_restart(double *__restrict__ sc, int copy_rr) {
    if (copy_rr) sc[kSRR] = sc[kSTmp];
    sc[kSFrozen] = (sc[kSTmp] <= sc[kSTol2] * sc[kSBB]) ? 1.0 : 0.0;
}

// c[j] = Q[j] . r, one CTA per basis vector, fixed reduction order
__global__ void __launch_bounds__(kDotThreads) k_basis_coef(const double *__restrict__ Q, int64_t n,
                                                            const double *__restrict__ r, double *__restrict__ c,
                                                            const double *__restrict__ sc) {
    if (sc[kSFrozen] != 0.0) return;
    __shared__ double ws[kDotThreads / 32];
    const double *q = Q + (int64_t)blockIdx.x * n;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kDotThreads) acc = fma(q[i], r[i], acc);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kDotThreads / 32; ++w) t += ws[w];
        c[blockIdx.x] = t;
    }
}

// r[i] -= sum_j c[j] Q[j][i]  (coalesced across i; c staged in shared memory)
__global__ void __launch_bounds__(256) k_basis_sub(const double *__restrict__ Q, int k, int64_t n,
                                                   const double *__restrict__ c, double *__restrict__ r,
                                                   const double *__restrict__ sc) {
    if (sc[kSFrozen] != 0.0) return;
    __shared__ double cs[kReorthMaxBasis];
    for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = c[j];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < k; ++j) acc = fma(cs[j], Q[(int64_t)j * n + i], acc);
        r[i] -= acc;
    }
}

__global__ void k_basis_append(double *__restrict__ q, const double *__restrict__ r, int64_t n,
                               const double *__restrict__ sc, int rr_slot) {
    if (sc[kSFrozen] != 0.0 || !(sc[rr_slot] > 0.0)) return;
    const double inv = 1.0 / sqrt(sc[rr_slot]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = r[i] * inv;
}

inline int vgrid(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 148 * 16 ? 148 * 16 : b));
}

}  // namespace

void launch_dot(const double *a, const double *b, int64_t n, double *partials, double *out, cudaStream_t s) {
    k_dot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, n, partials);
    k_dot_final<<<1, 32, 0, s>>>(partials, kDotBlocks, out);
    note_launches(2);
}

void cg_alpha(double *sc, cudaStream_t s) { k_cg_alpha<<<1, 1, 0, s>>>(sc); note_launches(1); }
void cg_update_yr(double *y, double *r, const double *p, const double *Ap, int64_t n, const double *sc,
                  cudaStream_t s) {
    k_cg_update_yr<<<vgrid(n), 256, 0, s>>>(y, r, p, Ap, n, sc); note_launches(1);
}
void cg_beta(double *sc, int it, int conv_slot, cudaStream_t s, double *hist, int hist_len) {
    k_cg_beta<<<1, 1, 0, s>>>(sc, it, conv_slot, hist, hist_len); note_launches(1);
}
void cg_update_p(double *p, const double *r, int64_t n, const double *sc, cudaStream_t s) {
    k_cg_update_p<<<vgrid(n), 256, 0, s>>>(p, r, n, sc); note_launches(1);
}
void vec_axpby(double a, const double *x, double b, const double *y, int64_t n, double *out, cudaStream_t s) {
    k_axpby<<<vgrid(n), 256, 0, s>>>(a, x, b, y, n, out); note_launches(1);
}
void vec_fill(double *x, int64_t n, double v, cudaStream_t s) { k_fill<<<vgrid(n), 256, 0, s>>>(x, n, v); note_launches(1); }
void cg_restart(double *sc, int copy_rr, cudaStream_t s) { k_cg_restart<<<1, 1, 0, s>>>(sc, copy_rr); note_launches(1); }
void cg_set_scalars(double *sc, double tol2, int bb_slot, cudaStream_t s) {
    k_set_scalars<<<1, 1, 0, s>>>(sc, tol2, bb_slot); note_launches(1);
}
void vec_mul(const double *a, const double *b, int64_t n, double *out, cudaStream_t s) {
    k_mul<<<vgrid(n), 256, 0, s>>>(a, b, n, out); note_launches(1);
}
void vec_jacobi_inv(const double *diag, double lam, int64_t n, double *out, cudaStream_t s) {
    k_jacobi_inv<<<vgrid(n), 256, 0, s>>>(diag, lam, n, out); note_launches(1);
}
void cg_reorth(const double *Q, int k, int64_t n, double *r, double *c, const double *sc, cudaStream_t s) {
    if (k <= 0) return;
    for (int pass = 0; pass < 2; ++pass) {   // "twice is enough"
        k_basis_coef<<<k, kDotThreads, 0, s>>>(Q, n, r, c, sc);
        k_basis_sub<<<vgrid(n), 256, 0, s>>>(Q, k, n, c, r, sc);
    }
    note_launches(4);
}
void cg_reorth2(const double *W, const double *V, int k, int64_t n, double *r, double *c, const double *sc,
                cudaStream_t s) {
    if (k <= 0) return;
    for (int pass = 0; pass < 2; ++pass) {
        k_basis_coef<<<k, kDotThreads, 0, s>>>(W, n, r, c, sc);
        k_basis_sub<<<vgrid(n), 256, 0, s>>>(V, k, n, c, r, sc);
    }
    note_launches(4);
}
void cg_basis_append(double *q_k, const double *r, int64_t n, const double *sc, int rr_slot, cudaStream_t s) {
    k_basis_append<<<vgrid(n), 256, 0, s>>>(q_k, r, n, sc, rr_slot); note_launches(1);
}

}  // namespace grav
