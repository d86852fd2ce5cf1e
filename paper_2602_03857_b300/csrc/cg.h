// Device-resident CG state: slots of the scalar array and vector launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace grav {

enum CgScalar : int {
    kSRR = 0,      // r.r of the current iterate
    kSPAp = 1,     // p.(A p)
    kSAlpha = 2,
    kSBeta = 3,
    kSRRNew = 4,
    kSBB = 5,      // dd.dd
    kSTol2 = 6,    // tol^2
    kSFrozen = 7,  // 0 running, 1 converged, 2 breakdown (p.Ap <= 0)
    kSIters = 8,   // iterations completed before freezing
    kSTrace = 9,
    kSTmp = 10,
    kSResNew = 11, // r.r after the update (convergence test of the preconditioned CG)
    kSPhi = 12,    // 7 slots: dot products of the outer loop's line search
    kSBB0 = 19,    // dd.dd when CG starts from a given y0
    kSCount = 24
};

void cg_alpha(double *sc, cudaStream_t s);
void cg_update_yr(double *y, double *r, const double *p, const double *Ap, int64_t n, const double *sc,
                  cudaStream_t s);
// hist (may be null): hist[it] = sqrt(sc[conv_slot] / sc[kSBB]) for it < hist_len
void cg_beta(double *sc, int it, int conv_slot, cudaStream_t s, double *hist = nullptr, int hist_len = 0);
void cg_update_p(double *p, const double *r, int64_t n, const double *sc, cudaStream_t s);
void vec_axpby(double a, const double *x, double b, const double *y, int64_t n, double *out, cudaStream_t s);
void vec_fill(double *x, int64_t n, double v, cudaStream_t s);
void cg_set_scalars(double *sc, double tol2, int bb_slot, cudaStream_t s);
void cg_restart(double *sc, int copy_rr, cudaStream_t s);
void vec_mul(const double *a, const double *b, int64_t n, double *out, cudaStream_t s);
void vec_jacobi_inv(const double *diag, double lam, int64_t n, double *out, cudaStream_t s);
// Full reorthogonalisation of the CG residual against the stored basis Q
// ([k][n], orthonormal rows): r -= Q^T (Q r), done twice; then
// cg_basis_append: Q[k] = r / |r| with |r|^2 from sc[rr_slot].  Both are
// no-ops once the CG state is frozen.  c: k doubles of scratch.
constexpr int kReorthMaxBasis = 4096;
void cg_reorth(const double *Q, int k, int64_t n, double *r, double *c, const double *sc, cudaStream_t s);
void cg_basis_append(double *q_k, const double *r, int64_t n, const double *sc, int rr_slot, cudaStream_t s);
// Preconditioned variant: r -= V^T (W r), twice, with V[j] = r_j / sqrt(r_j.z_j)
// and W[j] = z_j / sqrt(r_j.z_j) (z = M^-1 r): makes r orthogonal to the earlier
// residuals in the M^-1 inner product.
void cg_reorth2(const double *W, const double *V, int k, int64_t n, double *r, double *c, const double *sc,
                cudaStream_t s);

}  // namespace grav
