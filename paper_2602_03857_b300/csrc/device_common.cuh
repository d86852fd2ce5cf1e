// Device helpers shared by the libgrav kernels: physical constants, the
// FP64 corner function of Eq. 2-3, the FP32 far-field point-mass term,
// bounded mbarrier waits, 1D TMA bulk copies and the device status word.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace grav {

// gamma (CODATA 2018, m^3 kg^-1 s^-2) times 1e5 (m/s^2 -> mGal).
constexpr double kGammaMgal = 6.67430e-11 * 1.0e5;

// Device status word bits (OR-ed into ctx->d_status; never a trap).
constexpr int kStatusMbarTimeout = 1;
constexpr int kStatusBadLaunch = 2;

// Bound on every device-side wait, in nanoseconds of %globaltimer.
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Non-blocking probe of phase completion.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Waits for `phase` of `bar` for at most limit_ns (default kWaitLimitNs);
// returns false on timeout (the caller records the status and leaves the
// kernel).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_test(bar, phase)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_test(bar, phase)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
}

// As mbar_wait_bounded, but polling with mbarrier.try_wait (the hardware
// suspends the thread until the phase completes or a short system time limit
// passes) instead of test_wait + __nanosleep: for pipelines whose consumer
// spends little time per stage, where a sleep quantum would dominate.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_spin_bounded(uint64_t *bar, uint32_t phase,
                                                       uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, phase)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// 1D bulk copy global -> shared, completing on `bar` (TMA, no tensor map).
// dst and src must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2 (no shared memory, no
// completion): src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void set_status(int *status, int bit) {
    if (status) atomicOr(status, bit);
}

// ---------------------------------------------------------------------------
// FP64 elementary functions of Eq. 2-3, table-driven (the tables live in the
// context, built on the host from long-double logl/atanl; layout below).
//
// log64: P. T. P. Tang, "Table-driven implementation of the logarithm
// function in IEEE floating-point arithmetic", ACM TOMS 16 (1990) 378-400.
// x = 2^k m, m in [1, 2); F = 1 + j/256 nearest to m; f = m - F (exact);
// ln x = k ln2 + ln F + ln(1 + u), u = f / F, |u| <= 2^-9, with ln 2 and ln F
// split into a high part on the 2^-42 grid (so k ln2_hi + lnF_hi is exact)
// and a low part, and ln(1 + u) - u by its Taylor series to u^6 (truncation
// below 2^-65).  u is carried as uh + ul (ul from the exact residual
// f - uh F).  Zero, negative, subnormal, infinite and NaN arguments go to
// CUDA's log.
//
// atan_ratio64(a, b) = atan(a / b) for b > 0: with v = min(|a|, b) /
// max(|a|, b) in [0, 1] and c = j/64 nearest to v, atan(v) = atan(c) +
// atan(w), w = (v - c) / (1 + v c) = (p - c q) / (q + c p) for v = p / q —
// one division for the ratio and the reduction together, |w| <= 2^-7 — and
// atan(w) by its Taylor series to w^7 (truncation below 2^-65); for |a| > b,
// atan(a/b) = sign(a) (pi/2 - atan(b/|a|)).  The table holds atan(c) and
// pi/2 - atan(c) as high + low doubles.  Error: log64 <= 1 ulp; atan_ratio64
// (the ratio's three roundings included) about 1.1 ulp at worst, below CUDA's
// atan of a rounded quotient.
// ---------------------------------------------------------------------------
constexpr int kFnLogJ = 256;                            // log table: F = 1 + j/256, j = 0..256
constexpr int kFnLog = 0;                               // [3 j + 0..2] = 1/F, ln F hi, ln F lo
constexpr int kFnLn2 = kFnLog + 3 * (kFnLogJ + 1);      // ln 2 hi, ln 2 lo
constexpr int kFnAtanJ = 64;                            // atan table: c = j/64, j = 0..64
constexpr int kFnAtan = kFnLn2 + 2;                     // [4 j + 0..3] = atan c hi, lo, pi/2 - atan c hi, lo
constexpr int kFnDf = kFnAtan + 4 * (kFnAtanJ + 1);     // start of the FP32 table of the double-float functions
// double-float tables (FP32 offsets from T + kFnDf): ln c and 1/c for
// c = 1 + j/256, atan(j/256), ln 2, pi/2, each as a high + low float
constexpr int kDfLogJ = 256;
constexpr int kDfLog = 0;                               // [4 j + 0..3] = ln c hi, lo, 1/c hi, lo
constexpr int kDfAtanJ = 256;
constexpr int kDfAtan = kDfLog + 4 * (kDfLogJ + 1);     // [2 j + 0..1] = atan(j/256) hi, lo
constexpr int kDfLn2 = kDfAtan + 2 * (kDfAtanJ + 1);    // ln 2 hi, lo
constexpr int kDfPio2 = kDfLn2 + 2;                     // pi/2 hi, lo
constexpr int kDfTableFloats = kDfPio2 + 2;
constexpr int kFnTableSize = kFnDf + (kDfTableFloats + 1) / 2;

__device__ __forceinline__ double log64(double x, const double *__restrict__ T) {
    const long long b = __double_as_longlong(x);
    const int e = (int)(b >> 52);
    if (e <= 0 || e >= 0x7ff) return log(x);
    const long long mb = b & 0x000fffffffffffffLL;
    const int j = (int)((mb + (1LL << 43)) >> 44);
    const double m = __longlong_as_double(mb | 0x3ff0000000000000LL);
    const double F = fma((double)j, 1.0 / kFnLogJ, 1.0);
    const double f = m - F;
    const double inv = __ldg(T + kFnLog + 3 * j);
    const double uh = f * inv;
    const double ul = fma(-uh, F, f) * inv;
    const double u2 = uh * uh;
    double p = fma(uh, -1.0 / 6.0, 1.0 / 5.0);
    p = fma(p, uh, -0.25);
    p = fma(p, uh, 1.0 / 3.0);
    p = fma(p, uh, -0.5);
    const double k = (double)(e - 1023);
    const double hi = fma(k, __ldg(T + kFnLn2), __ldg(T + kFnLog + 3 * j + 1));
    const double lo = fma(k, __ldg(T + kFnLn2 + 1), __ldg(T + kFnLog + 3 * j + 2));
    return hi + (uh + fma(u2, p, ul + lo));
}

__device__ __forceinline__ double atan_ratio64(double a, double b, const double *__restrict__ T) {
    const double pa = fabs(a);
    const bool big = pa > b;
    const double p = big ? b : pa, q = big ? pa : b;   // v = p / q in [0, 1]
    const float vf = __fdividef((float)p, (float)q);
    int j = __float2int_rn(vf * (float)kFnAtanJ);
    j = min(max(j, 0), kFnAtanJ);
    const double c = (double)j * (1.0 / kFnAtanJ);
    const double w = fma(-c, q, p) / fma(c, p, q);
    const double w2 = w * w;
    double r = fma(w2, -1.0 / 7.0, 1.0 / 5.0);
    r = fma(r, w2, -1.0 / 3.0);
    r = fma(w2 * w, r, w);
    // base + r with base = table high + low; |base_hi| >= |r| for j >= 1 (and
    // base = 0 for j = 0), so Fast2Sum gives the rounding error of base_hi + r
    const double *t = T + kFnAtan + 4 * j + (big ? 2 : 0);
    const double th = __ldg(t), rr = big ? -r : r;
    const double sh = th + rr;
    const double er = rr - (sh - th);
    const double res = sh + (er + __ldg(t + 1));
    return a < 0.0 ? -res : res;
}

// ---------------------------------------------------------------------------
// Eq. 2-3 in FP64.  Arguments are the vertex coordinates relative to the
// station (z > 0: the vertex lies below the station) and their squares; T is
// the function table above.  ln(R + a) for a < 0 is taken as
// ln((R^2 - a^2) / (R - a)), an exact identity that avoids the cancellation
// of R + a (the reading adopted for the paper's unspecified
// "singularity-robust formulation", Section 2.3).  With z > 0, R > 0 and
// R^2 - a^2 > 0, so every logarithm argument is positive; at x = 0 (y = 0)
// the x ln (y ln) term is exactly 0 * finite = 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double psi64(double x, double y, double z, double x2, double y2, double z2,
                                        const double *__restrict__ T) {
    const double R2 = x2 + y2 + z2;
    const double R = sqrt(R2);
    const double t_atan = z * atan_ratio64(x * y, z * R, T);
    double ry, rx;
    if (y >= 0.0) ry = R + y; else ry = (x2 + z2) / (R - y);
    if (x >= 0.0) rx = R + x; else rx = (y2 + z2) / (R - x);
    return t_atan - x * log64(ry, T) - y * log64(rx, T);
}

// Eq. 2-3 evaluated entirely in FP32 (CUDA's IEEE sqrtf/logf/atanf and
// divisions), with the same cancellation-free logarithm forms as psi64.  Used
// only by the GRAV_MIXED_CORNER variant, the literal "FP32 corner terms"
// reading, whose far-field error this library reports.
__device__ __forceinline__ float psi32(float x, float y, float z) {
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    const float R = sqrtf(x2 + y2 + z2);
    const float t_atan = z * atanf((x * y) / (z * R));
    float ry, rx;
    if (y >= 0.0f) ry = R + y; else ry = (x2 + z2) / (R - y);
    if (x >= 0.0f) rx = R + x; else rx = (y2 + z2) / (R - x);
    return t_atan - x * logf(ry) - y * logf(rx);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (T. J. Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18 (1971) 224-242; Knuth's
// TwoSum): a value is the unevaluated sum hi + lo of two FP32 numbers,
// |lo| <= ulp(hi)/2, about 44-48 significant bits, computed on the FP32 pipe
// (64x the FP64 rate on this GPU).  The rounded intrinsics keep the compiler
// from contracting the error-free transformations into FMAs.
// ---------------------------------------------------------------------------
struct df32 {
    float hi, lo;
};
__device__ __forceinline__ df32 df_make(float hi, float lo) {
    df32 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}
// |a| >= |b| or a = 0: s + e = a + b exactly
__device__ __forceinline__ df32 df_fast2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df32 df_2sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df_make(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ df32 df_2prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return df_make(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    const df32 s = df_2sum(a.hi, b.hi);
    return df_fast2sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df32 df_neg(df32 a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df32 df_sub(df32 a, df32 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
    const df32 p = df_2prod(a.hi, b.hi);
    return df_fast2sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ df32 df_mulf(df32 a, float b) {
    const df32 p = df_2prod(a.hi, b);
    return df_fast2sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ df32 df_sqr(df32 a) {
    const df32 p = df_2prod(a.hi, a.hi);
    return df_fast2sum(p.hi, __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, p.lo));
}
// a / b: the FP32 quotient, then two corrections from the residual a - b q
__device__ __forceinline__ df32 df_div(df32 a, df32 b) {
    const float r = __frcp_rn(b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    const float q2 = __fmul_rn(df_sub(a, df_mulf(b, q1)).hi, r);
    const df32 q = df_fast2sum(q1, q2);
    const float q3 = __fmul_rn(df_sub(a, df_mul(b, q)).hi, r);
    return df_add(q, df_make(q3, 0.0f));
}
// sqrt(a), a >= 0: the FP32 root and one correction from the residual
__device__ __forceinline__ df32 df_sqrt(df32 a) {
    if (!(a.hi > 0.0f)) return df_make(0.0f, 0.0f);
    const float s = __fsqrt_rn(a.hi);
    const df32 p = df_2prod(s, s);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
    return df_fast2sum(s, __fmul_rn(d, __fmul_rn(0.5f, __frcp_rn(s))));
}
__device__ __forceinline__ df32 df_from_double(double x) {
    const float h = __double2float_rn(x);
    return df_make(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

// ln a for a double-float a > 0 (a.hi normal): the table method of log64
// (Tang, 1990) in double-float.  a = 2^e m, c = 1 + j/256 nearest to m,
// f = (m - c + a.lo 2^-e) / c with |f| <= 2^-9, ln a = e ln 2 + ln c +
// ln(1 + f), ln(1 + f) = f - f^2/2 (double-float) + f^3 (1/3 - f/4 + f^2/5 -
// f^3/6 + f^4/7) (FP32, ~2^-53 absolute; f^8/8 is below 2^-74).
// D = T + kFnDf as floats.
__device__ __forceinline__ df32 df_log(df32 a, const float *__restrict__ D) {
    const int b = __float_as_int(a.hi);
    const int e = ((b >> 23) & 0xff) - 127;
    const int mb = b & 0x7fffff;
    const float m = __int_as_float(mb | 0x3f800000);            // [1, 2)
    const int j = (mb + (1 << 14)) >> 15;                        // 0 .. 256
    const float c = __fmaf_rn((float)j, 1.0f / kDfLogJ, 1.0f);   // exact
    const df32 u = df_2sum(__fsub_rn(m, c), ldexpf(a.lo, -e));   // m - c exact
    const df32 f = df_mul(u, df_make(__ldg(D + kDfLog + 4 * j + 2), __ldg(D + kDfLog + 4 * j + 3)));
    const float fh = f.hi;
    float p = __fmaf_rn(1.0f / 7.0f, fh, -1.0f / 6.0f);
    p = __fmaf_rn(p, fh, 1.0f / 5.0f);
    p = __fmaf_rn(p, fh, -0.25f);
    p = __fmaf_rn(p, fh, 1.0f / 3.0f);
    const float f3 = __fmul_rn(__fmul_rn(__fmul_rn(fh, fh), fh), p);
    const df32 f2 = df_sqr(f);
    df32 r = df_add(f, df_make(-0.5f * f2.hi, -0.5f * f2.lo));
    r = df_add(r, df_make(f3, 0.0f));
    const df32 t = df_add(df_mulf(df_make(__ldg(D + kDfLn2), __ldg(D + kDfLn2 + 1)), (float)e),
                          df_make(__ldg(D + kDfLog + 4 * j), __ldg(D + kDfLog + 4 * j + 1)));
    return df_add(t, r);
}

// atan(a / b) for b > 0 in double-float: the reduction of atan_ratio64 —
// v = min(|a|, b) / max(|a|, b), c = j/256 nearest, atan v = atan c + atan w,
// w = (p - c q) / (q + c p), |w| <= 2^-9, atan w = w + w^3 (-1/3 + w^2/5 -
// w^4/7) (the cubic part in FP32 at w.hi, with its first-order term in w.lo;
// w^9/9 is below 2^-65); for |a| > b,
// atan(a/b) = sign(a) (pi/2 - atan(b/|a|)).
__device__ __forceinline__ df32 df_atan_ratio(df32 a, df32 b, const float *__restrict__ D) {
    const bool neg = a.hi < 0.0f;
    const df32 pa = neg ? df_neg(a) : a;
    const bool big = pa.hi > b.hi;
    const df32 p = big ? b : pa, q = big ? pa : b;
    int j = __float2int_rn(__fmul_rn(__fdividef(p.hi, q.hi), (float)kDfAtanJ));
    j = min(max(j, 0), kDfAtanJ);
    const float c = (float)j * (1.0f / kDfAtanJ);   // exact
    const df32 w = df_div(df_sub(p, df_mulf(q, c)), df_add(q, df_mulf(p, c)));
    const float wh = w.hi, w2 = __fmul_rn(wh, wh);
    float r = __fmaf_rn(w2, -1.0f / 7.0f, 1.0f / 5.0f);
    r = __fmaf_rn(r, w2, -1.0f / 3.0f);
    // cubic part at wh (its FP32 rounding: ~2^-43 of w at |w| = 2^-9, the
    // reason for the 256-entry table), plus its first-order change with w.lo
    df32 s = df_add(w, df_make(__fmaf_rn(__fmul_rn(wh, w2), r, -__fmul_rn(w2, w.lo)), 0.0f));
    s = df_add(df_make(__ldg(D + kDfAtan + 2 * j), __ldg(D + kDfAtan + 2 * j + 1)), s);
    if (big) s = df_sub(df_make(__ldg(D + kDfPio2), __ldg(D + kDfPio2 + 1)), s);
    return neg ? df_neg(s) : s;
}

// Eq. 2-3 in double-float, with the same cancellation-free logarithm forms
// and limits as psi64 (z > 0).  Error about 2^-45 of R (|ln R| + 1); the
// near-field set-up needs about 2^-39 for the FP32 entries of its table.
__device__ __forceinline__ df32 psi_df(df32 x, df32 y, df32 z, const float *__restrict__ D) {
    const df32 x2 = df_sqr(x), y2 = df_sqr(y), z2 = df_sqr(z);
    const df32 R = df_sqrt(df_add(df_add(x2, y2), z2));
    const df32 ta = df_mul(z, df_atan_ratio(df_mul(x, y), df_mul(z, R), D));
    const df32 ry = (y.hi >= 0.0f) ? df_add(R, y) : df_div(df_add(x2, z2), df_sub(R, y));
    const df32 rx = (x.hi >= 0.0f) ? df_add(R, x) : df_div(df_add(y2, z2), df_sub(R, x));
    return df_sub(df_sub(ta, df_mul(x, df_log(ry, D))), df_mul(y, df_log(rx, D)));
}

// ---------------------------------------------------------------------------
// FP32 far-field term of a cubic prism: dz / R^3 (point mass at the cell
// centre).  dz, R2 in metres; one MUFU reciprocal square root.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float far_kernel(float dz, float R2) {
    const float rs = rsqrt_approx(R2);
    const float rs2 = rs * rs;
    return (dz * rs) * rs2;
}

// Two FP32 values packed in one 64-bit register pair (.lo = first), operated on
// by the sm_100-family packed instructions add/mul/fma.rn.f32x2: two IEEE
// round-to-nearest FP32 results per instruction, bit-identical to the scalar
// operations on each half.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f2_t rsqrt2(f2_t R2) {
    float r0, r1;
    f2_unpack(R2, r0, r1);
    return f2_pack(rsqrt_approx(r0), rsqrt_approx(r1));
}

// The far-field term for two pairs at once: acc += w * dz / R^3 with
// dz = zc + nzs (nzs = -station depth), R^2 = dz^2 + h2.  Same operations, in
// the same order, as far_kernel() on each half.
__device__ __forceinline__ f2_t far_pair_acc(f2_t zc, f2_t nzs, f2_t h2, f2_t w, f2_t acc) {
    const f2_t dz = f2_add(zc, nzs);
    const f2_t R2 = f2_fma(dz, dz, h2);
    const f2_t rs = rsqrt2(R2);
    const f2_t rs2 = f2_mul(rs, rs);
    const f2_t k = f2_mul(f2_mul(dz, rs), rs2);
    return f2_fma(w, k, acc);
}

// Far-field term of a uniform a x b x c box to second order.  Averaging
// K = dz / R^3 over the box adds (a^2 Kxx + b^2 Kyy + c^2 Kzz) / 24 (the
// second moments a^2/12, b^2/12, c^2/12; K is harmonic, so the box's
// quadrupole is all there is to this order), i.e. K times
//   1 + (A dx^2 + B dy^2 + C dz^2) / R^4,
//   A = (12a^2 - 3b^2 - 9c^2) / 24, B = (12b^2 - 3a^2 - 9c^2) / 24,
//   C = (6c^2 - 3a^2 - 3b^2) / 24
// (all three vanish for a cube).  ph = A dx^2 + B dy^2 is formed once per
// (station, column) by far_ph(); qg = C.
__device__ __forceinline__ float far_ph(float2 X, float2 Y, float xh, float xl, float yh, float yl, float qa,
                                        float qb) {
    const float dx = (X.x - xh) + (X.y - xl);
    const float dy = (Y.x - yh) + (Y.y - yl);
    return fmaf(qa * dx, dx, (qb * dy) * dy);
}

__device__ __forceinline__ float far_kernel_q(float dz, float R2, float qg, float ph) {
    const float rs = rsqrt_approx(R2);
    const float rs2 = rs * rs;
    const float k = (dz * rs) * rs2;
    const float n = fmaf(qg, dz * dz, ph);
    const float f = fmaf(n, rs2 * rs2, 1.0f);
    return k * f;
}

// The same for two pairs at once (same operations per half).
__device__ __forceinline__ f2_t far_pair_acc_q(f2_t zc, f2_t nzs, f2_t h2, f2_t w, f2_t acc, f2_t qg, f2_t ph) {
    const f2_t dz = f2_add(zc, nzs);
    const f2_t R2 = f2_fma(dz, dz, h2);
    const f2_t rs = rsqrt2(R2);
    const f2_t rs2 = f2_mul(rs, rs);
    const f2_t k = f2_mul(f2_mul(dz, rs), rs2);
    const f2_t n = f2_fma(qg, f2_mul(dz, dz), ph);
    const f2_t f = f2_fma(n, f2_mul(rs2, rs2), f2_pack(1.0f, 1.0f));
    return f2_fma(w, f2_mul(k, f), acc);
}

template <bool QUAD>
__device__ __forceinline__ f2_t far_pair(f2_t zc, f2_t nzs, f2_t h2, f2_t w, f2_t acc, f2_t qg, f2_t ph) {
    return QUAD ? far_pair_acc_q(zc, nzs, h2, w, acc, qg, ph) : far_pair_acc(zc, nzs, h2, w, acc);
}

template <bool QUAD>
__device__ __forceinline__ float far_k(float dz, float R2, float qg, float ph) {
    return QUAD ? far_kernel_q(dz, R2, qg, ph) : far_kernel(dz, R2);
}

// Knuth two-sum: (s, e) with s = fl(a + b), a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Warp-wide sum with a fixed xor butterfly (deterministic, every lane gets it).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace grav
