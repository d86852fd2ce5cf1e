// Pipe-rate microbenchmarks: throughput of the MUFU reciprocal square root
// and base-2 logarithm, FP32 FMA and FP64 FMA on this device, plus the SM
// clock seen while they run.  They give the per-clock unit rates behind the
// ALU rooflines of the operator kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace grav {
namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_v(float x) {
    float r;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_v(float x) {
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_v(float x) {
    float r;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// op: 0 rsqrt, 1 lg2, 2 ffma, 3 dfma, 4 packed fma.rn.f32x2 (counted as 2 FP32 FMAs),
//     5 FP64 log, 6 FP64 atan, 7 FP64 sqrt, 8 FP64 division (CUDA's implementations),
//     9 this library's table-driven log64, 10 its atan_ratio64 (tables in fn),
//     11 MUFU rcp, 12 MUFU ex2
template <int OP>
__global__ void k_pipe(int iters, float seed, float *out, unsigned long long *clk, const double *fn) {
    const uint64_t t0 = globaltimer_ns();
    const long long c0 = clock64();
    if (OP == 4) {
        f2_t a[kChains];
        const f2_t m = f2_pack(0.999999f, 0.999998f), c = f2_pack(1e-7f, 2e-7f);
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = f2_pack(seed + 0.001f * (threadIdx.x + k), seed);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = f2_fma(a[k], m, c);
        }
        float s = 0, lo, hi;
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            f2_unpack(a[k], lo, hi);
            s += lo + hi;
        }
        if (s == 12345.678f) out[0] = s;
    } else if (OP >= 5 && OP <= 10) {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 1.5 + seed + 0.001 * (threadIdx.x + k);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if (OP == 5) a[k] = log(a[k]) + 2.5;
                else if (OP == 6) a[k] = atan(a[k]) + 1.25;
                else if (OP == 9) a[k] = log64(a[k], fn) + 2.5;
                else if (OP == 10) a[k] = atan_ratio64(a[k], 1.0, fn) + 1.25;
                else if (OP == 7) a[k] = sqrt(a[k]) + 1.5;
                else a[k] = 3.0 / a[k] + 1.0;
            }
        }
        double s = 0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == 12345.678) out[0] = (float)s;
    } else if (OP == 3) {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = seed + 0.001 * (threadIdx.x + k);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], 0.999999, 1e-7);
        }
        double s = 0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == 12345.678) out[0] = (float)s;
    } else {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = seed + 0.001f * (threadIdx.x + k);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if (OP == 0) a[k] = rsqrt_v(a[k]);
                else if (OP == 1) a[k] = lg2_approx(a[k] + 2.0f);
                else if (OP == 11) a[k] = rcp_v(a[k] + 1.0f);
                else if (OP == 12) a[k] = ex2_v(a[k] * -0.5f);
                else a[k] = fmaf(a[k], 0.999999f, 1e-7f);
            }
        }
        float s = 0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == 12345.678f) out[0] = s;
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const long long c1 = clock64();
        const uint64_t t1 = globaltimer_ns();
        clk[0] = (unsigned long long)(c1 - c0);
        clk[1] = (unsigned long long)(t1 - t0);
    }
}

template <int OP>
int run_one(int sms, double *ops_per_s, double *clk_mhz, const double *fn = nullptr) {
    float *out = nullptr;
    unsigned long long *clk = nullptr;
    if (cudaMalloc(&out, 16) != cudaSuccess) return -1;
    if (cudaMalloc(&clk, 16) != cudaSuccess) return -1;
    const int blocks = sms * 8, threads = 256;
    const int iters = (OP == 3) ? 256 : (OP >= 5 && OP <= 10 ? 16 : 4096);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_pipe<OP><<<blocks, threads>>>(iters / 16, 1.5f, out, clk, fn);   // warm-up
    cudaEventRecord(e0);
    k_pipe<OP><<<blocks, threads>>>(iters, 1.5f, out, clk, fn);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long h[2] = {0, 0};
    cudaMemcpy(h, clk, 16, cudaMemcpyDeviceToHost);
    *ops_per_s = (double)blocks * threads * iters * kChains * (OP == 4 ? 2 : 1) / (ms * 1e-3);
    *clk_mhz = h[1] ? (double)h[0] / (double)h[1] * 1e3 : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(clk);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// out[i] = f(a[i], b[i]) for the self-check of the FP64 functions
__global__ void k_eval_fn(int fn, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out,
                          int64_t n, const double *__restrict__ T) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (fn == 0) v = log64(a[i], T);
        else if (fn == 1) v = atan_ratio64(a[i], b[i], T);
        else if (fn == 2) v = log(a[i]);
        else if (fn == 3) v = atan(a[i] / b[i]);
        else {
            const float *D = reinterpret_cast<const float *>(T + kFnDf);
            if (fn == 4) v = df_to_double(df_log(df_from_double(a[i]), D));
            else if (fn == 5) v = df_to_double(df_atan_ratio(df_from_double(a[i]), df_from_double(b[i]), D));
            else v = df_to_double(psi_df(df_from_double(a[i]), df_from_double(b[i]), df_from_double(a[n + i]), D));
        }
        out[i] = v;
    }
}

// The failure path of every bounded mbarrier wait, exercised on purpose: an
// mbarrier that expects one arrival which nothing makes; the wait gives up
// after limit_ns, records kStatusMbarTimeout and the kernel returns.  No
// asynchronous copy is in flight, so nothing outlives the kernel.
__global__ void k_selftest_wait(int *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) set_status(status, kStatusMbarTimeout);
}

}  // namespace
}  // namespace grav

extern "C" int grav_selftest_wait(grav_ctx *ctx, double limit_ms, grav_stream_t stream) {
    using namespace grav;
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    if (!(limit_ms > 0.0) || limit_ms > 1000.0) return set_error(ctx, GRAV_EINVAL, "limit_ms must lie in (0, 1000]");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    k_selftest_wait<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->d_status, (uint64_t)(limit_ms * 1e6));
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    int rc = e == cudaSuccess ? read_status(ctx, (cudaStream_t)stream, 60.0) : cuda_error(ctx, e, "selftest launch");
    cudaSetDevice(prev);
    return rc;
}

extern "C" int grav_eval_fn64(grav_ctx *ctx, int fn, const double *a, const double *b, double *out, int64_t n,
                              grav_stream_t stream) {
    using namespace grav;
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    if (fn < 0 || fn > 6) return set_error(ctx, GRAV_EINVAL, "fn must be 0..6");
    if (n < 0) return set_error(ctx, GRAV_EINVAL, "n must be >= 0");
    if (n == 0) return GRAV_OK;
    if (!a || !out || ((fn == 1 || fn == 3 || fn == 5 || fn == 6) && !b)) return set_error(ctx, GRAV_EINVAL, "NULL argument");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 148LL * 16);
    k_eval_fn<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(fn, a, b, out, n, ctx->d_fn);
    note_launches(1);
    const cudaError_t e = cudaGetLastError();
    cudaSetDevice(prev);
    return e == cudaSuccess ? GRAV_OK : cuda_error(ctx, e, "eval_fn64 launch");
}

extern "C" int grav_bench_pipes(int device, double *out) {
    using namespace grav;
    if (!out) return set_error(nullptr, GRAV_EINVAL, "out is NULL");
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n)
        return set_error(nullptr, GRAV_EINVAL, "bad device");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int rc = 0;
    rc |= run_one<0>(sms, &out[0], &out[1]);
    rc |= run_one<1>(sms, &out[2], &out[3]);
    rc |= run_one<2>(sms, &out[4], &out[5]);
    rc |= run_one<3>(sms, &out[6], &out[7]);
    rc |= run_one<4>(sms, &out[8], &out[9]);
    out[10] = sms;
    rc |= run_one<5>(sms, &out[11], &out[12]);
    rc |= run_one<6>(sms, &out[13], &out[14]);
    rc |= run_one<7>(sms, &out[15], &out[16]);
    rc |= run_one<8>(sms, &out[17], &out[18]);
    std::vector<double> fh(fn_table_size());
    fill_fn_table(fh.data());
    double *fn = nullptr;
    if (cudaMalloc(&fn, 8 * fh.size()) != cudaSuccess ||
        cudaMemcpy(fn, fh.data(), 8 * fh.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        rc = -1;
    } else {
        rc |= run_one<9>(sms, &out[19], &out[20], fn);
        rc |= run_one<10>(sms, &out[21], &out[22], fn);
    }
    rc |= run_one<11>(sms, &out[23], &out[24]);
    rc |= run_one<12>(sms, &out[25], &out[26]);
    if (fn) cudaFree(fn);
    cudaSetDevice(prev);
    return rc ? set_error(nullptr, GRAV_EDEVICE, "pipe microbenchmark failed") : GRAV_OK;
}
