// grav_forward_fp64_noalloc: the FP64 forward product d = G m for callers
// that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc or any allocating routine
// while it runs -- e.g. a host framework whose caching allocator owns all
// device memory and forbids foreign allocations, a service with a fixed,
// pre-reserved memory budget, or a caller that cannot afford the implicit
// device synchronisation an allocation may cause.  Such callers cannot create
// a grav_ctx (whose plans draw their scratch from a memory pool).
//
// How: the scratch (mesh edges, node weights, per-chunk partial sums and the
// device status word) lives in one file-scope static __device__ array of
// kStaticScratchBytes.  Every GPU that loads libgrav holds this array until
// the process exits.  Host code only knows the array's host-side stand-in,
// so the first call on each device looks its device address up with
// cudaGetSymbolAddress (with that device current) and caches it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "device_common.cuh"
#include "internal.h"

namespace grav {
namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;     // 64 MiB per device
constexpr size_t kStaticScratchDoubles = kStaticScratchBytes / sizeof(double);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_static_mu;
double *g_static_ptr[kMaxDevices] = {nullptr};

// Once per device, with that device current: the device address of the array.
int static_scratch_address(int device, double **out) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[device]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return cuda_error(nullptr, e, "cudaGetSymbolAddress(static scratch)");
        g_static_ptr[device] = static_cast<double *>(ptr);
    }
    *out = g_static_ptr[device];
    return GRAV_OK;
}

bool dev_ptr_on(const void *p, int device) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

bool edges_ok(const double *e, int n) {
    for (int i = 0; i <= n; ++i)
        if (!std::isfinite(e[i])) return false;
    for (int i = 0; i < n; ++i)
        if (!(e[i + 1] > e[i])) return false;
    return true;
}

inline size_t round32(size_t v) { return (v + 31) / 32 * 32; }   // 256-byte granularity in doubles

// A bounded wait in k_fwd64 that ran out leaves its CTA's partial sums
// unwritten (the array keeps an earlier call's values there), so the whole
// product is void: every d_i becomes NaN.  The status word was cleared at the
// start of this call on the same stream.
__global__ void k_void_on_status(const int *__restrict__ status, double *__restrict__ d, int64_t n) {
    if (*status == 0) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = nan;
}

}  // namespace
}  // namespace grav

using namespace grav;

extern "C" int grav_forward_fp64_noalloc(const grav_mesh *mesh, const grav_survey *survey, const double *m,
                                         double *d, grav_stream_t stream) {
    if (!mesh || !survey) return set_error(nullptr, GRAV_EINVAL, "mesh or survey is NULL");
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || mesh->nx > (1 << 20) || mesh->ny > (1 << 20) ||
        mesh->nz > (1 << 16))
        return set_error(nullptr, GRAV_EINVAL, "mesh sizes must lie in [1, 2^20] x [1, 2^20] x [1, 2^16]");
    if ((int64_t)mesh->nx * mesh->ny * mesh->nz > ((int64_t)1 << 30) ||
        (int64_t)(mesh->nx + 1) * (mesh->ny + 1) * (mesh->nz + 1) > ((int64_t)1 << 30))
        return set_error(nullptr, GRAV_EINVAL, "mesh too large: at most 2^30 cells and 2^30 nodes");
    if (mesh->nx + 1 > fwd64_max_nodes_x())
        return set_error(nullptr, GRAV_EINVAL,
                         "nx+1 must be <= %d (one row of node weights is staged in shared memory; got %d)",
                         fwd64_max_nodes_x(), mesh->nx + 1);
    if (!mesh->xe || !mesh->ye || !mesh->ze || !edges_ok(mesh->xe, mesh->nx) || !edges_ok(mesh->ye, mesh->ny) ||
        !edges_ok(mesh->ze, mesh->nz))
        return set_error(nullptr, GRAV_EINVAL, "mesh edges must be finite and strictly increasing");
    if (survey->n < 1 || survey->n > ((int64_t)1 << 30))
        return set_error(nullptr, GRAV_EINVAL, "survey size must lie in [1, 2^30]");
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "cudaGetDevice");
    if (device < 0 || device >= kMaxDevices) return set_error(nullptr, GRAV_EINVAL, "device index out of range");
    if (!dev_ptr_on(survey->x, device) || !dev_ptr_on(survey->y, device) || !dev_ptr_on(survey->z, device) ||
        !dev_ptr_on(m, device) || !dev_ptr_on(d, device))
        return set_error(nullptr, GRAV_EINVAL, "survey arrays, m and d must be device pointers on the current device");

    const int nx = mesh->nx, ny = mesh->ny, nz = mesh->nz;
    const int64_t N = survey->n;
    const int ldw = (nx + 2) / 2 * 2;
    // (ny+1)(nz+1) <= 2^30 by the node cap above; the products below are size_t
    const int64_t nrows64 = (int64_t)(ny + 1) * (nz + 1);
    // scratch layout (in doubles): status | FP64 log/atan table | xe | ye | ze | w | partials
    const size_t o_fn = 32;
    const size_t o_xe = o_fn + round32((size_t)fn_table_size());
    const size_t o_ye = o_xe + round32((size_t)nx + 1);
    const size_t o_ze = o_ye + round32((size_t)ny + 1);
    const size_t o_w = o_ze + round32((size_t)nz + 1);
    const size_t w_doubles = (size_t)nrows64 * (size_t)ldw;
    if (w_doubles > kStaticScratchDoubles || o_w + round32(w_doubles) + (size_t)N > kStaticScratchDoubles)
        return set_error(nullptr, GRAV_EINVAL,
                         "problem too large for the %zu MiB static scratch: node weights need %.1f MiB and the "
                         "partial sums at least %.1f MiB",
                         kStaticScratchBytes >> 20, (double)w_doubles * 8 / 1048576.0, (double)N * 8 / 1048576.0);
    const size_t o_part = o_w + round32(w_doubles);
    const int nrows = (int)nrows64;   // fits: the node weights fit 64 MiB
    // chunking: as many node-row chunks as fill the GPU, capped by what fits
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int64_t tiles = (N + fwd64_stations_per_cta() - 1) / fwd64_stations_per_cta();
    const int64_t target = (int64_t)sms * 40;
    int64_t nch = std::min<int64_t>(std::max<int64_t>(1, (target + tiles - 1) / tiles), nrows);
    nch = std::min<int64_t>(nch, (int64_t)((kStaticScratchDoubles - o_part) / (size_t)N));
    const int rows_per_chunk = (int)((nrows + nch - 1) / nch);
    const int nchunk = (nrows + rows_per_chunk - 1) / rows_per_chunk;

    double *base = nullptr;
    int rc = static_scratch_address(device, &base);
    if (rc) return rc;
    const cudaStream_t s = (cudaStream_t)stream;
    // the status word must start at zero; every other region is fully rewritten
    if ((e = cudaMemsetAsync(base, 0, 256, s)) != cudaSuccess) return cuda_error(nullptr, e, "status reset");
    // the function table is built once per process on the host and uploaded each call
    static const std::vector<double> fn_host = [] {
        std::vector<double> t(fn_table_size());
        fill_fn_table(t.data());
        return t;
    }();
    if ((e = cudaMemcpyAsync(base + o_fn, fn_host.data(), 8 * fn_host.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_xe, mesh->xe, 8ull * (nx + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_ye, mesh->ye, 8ull * (ny + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_ze, mesh->ze, 8ull * (nz + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_error(nullptr, e, "edge upload");
    Geo g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.xe = base + o_xe; g.ye = base + o_ye; g.ze = base + o_ze;
    g.N = N;
    g.fn = base + o_fn;
    int *status = reinterpret_cast<int *>(base);
    if (launch_fwd64_raw(g, ldw, m, base + o_w, rows_per_chunk, nchunk, survey->x, survey->y, survey->z,
                         base + o_part, status, s) < 0)
        return cuda_error(nullptr, cudaGetLastError(), "noalloc forward: shared-memory limit of k_fwd64");
    launch_reduce_rows(base + o_part, nchunk, N, kGammaMgal, nullptr, 0.0, nullptr, d, s);
    k_void_on_status<<<(unsigned)std::min<int64_t>((N + 255) / 256, (int64_t)sms * 8), 256, 0, s>>>(status, d, N);
    note_launches(1);
    e = cudaGetLastError();
    return e == cudaSuccess ? GRAV_OK : cuda_error(nullptr, e, "noalloc forward launch");
}
