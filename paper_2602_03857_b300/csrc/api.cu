// C ABI of libgrav: context, argument validation, plans, one-shot operator
// calls and the data-space CG solve (Section 2.2, Eq. 10-11).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>

#include "cg.h"
#include "device_common.cuh"
#include "internal.h"

using grav::kSCount;

namespace grav {

namespace {
std::atomic<uint64_t> g_launches{0};
std::mutex g_err_mu;
std::string g_last_error = "";

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Polls the event until it completes or timeout_s passes.  The sleep between
// polls is 1/16 of the time already waited (5 us .. 2 ms), so a wait ends at
// most ~6 % (2 ms) after the event while long waits do not spin; a doubling
// backoff instead overshot a 5.7 ms CG iteration by up to 2 ms.
int wait_event(grav_ctx *ctx, cudaEvent_t ev, double timeout_s, const char *what) {
    const double t0 = now_s();
    while (true) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return GRAV_OK;
        if (e != cudaErrorNotReady) return cuda_error(ctx, e, what);
        const double el = now_s() - t0;
        if (el > timeout_s) return set_error(ctx, GRAV_ETIMEDOUT, "%s: timed out after %.1f s", what, timeout_s);
        const double us = std::min(2000.0, std::max(5.0, el * 1e6 / 16.0));
        std::this_thread::sleep_for(std::chrono::microseconds((int64_t)us));
    }
}

bool is_device_ptr(const void *p, int device) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

bool finite_increasing(const double *e, int n) {
    for (int i = 0; i <= n; ++i)
        if (!std::isfinite(e[i])) return false;
    for (int i = 0; i < n; ++i)
        if (!(e[i + 1] > e[i])) return false;
    return true;
}

int check_mesh(grav_ctx *ctx, const grav_mesh *mesh) {
    if (!mesh) return set_error(ctx, GRAV_EINVAL, "mesh is NULL");
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1)
        return set_error(ctx, GRAV_EINVAL, "mesh sizes must be >= 1 (got %d x %d x %d)", mesh->nx, mesh->ny, mesh->nz);
    if ((int64_t)mesh->nx * mesh->ny * mesh->nz > (int64_t)1 << 30 ||
        (int64_t)(mesh->nx + 1) * (mesh->ny + 1) * (mesh->nz + 1) > (int64_t)1 << 30 || mesh->nx > 1 << 20 ||
        mesh->ny > 1 << 20 || mesh->nz > 1 << 16)
        return set_error(ctx, GRAV_EINVAL, "mesh too large");
    if (!mesh->xe || !mesh->ye || !mesh->ze) return set_error(ctx, GRAV_EINVAL, "mesh edge array is NULL");
    if (!finite_increasing(mesh->xe, mesh->nx) || !finite_increasing(mesh->ye, mesh->ny) ||
        !finite_increasing(mesh->ze, mesh->nz))
        return set_error(ctx, GRAV_EINVAL, "mesh edges must be finite and strictly increasing");
    return GRAV_OK;
}

int check_options(grav_ctx *ctx, const grav_options &o) {
    if (o.precision != GRAV_FP64 && o.precision != GRAV_MIXED && o.precision != GRAV_MIXED_CORNER)
        return set_error(ctx, GRAV_EINVAL, "precision must be GRAV_FP64, GRAV_MIXED or GRAV_MIXED_CORNER (got %d)",
                         o.precision);
    if (!std::isfinite(o.z0) || o.z0 < 0) return set_error(ctx, GRAV_EINVAL, "z0 must be finite and >= 0");
    if (!(o.lambda_scale > 0) || !std::isfinite(o.lambda_scale))
        return set_error(ctx, GRAV_EINVAL, "lambda_scale must be > 0");
    if (!std::isfinite(o.lambda) || o.lambda < 0) return set_error(ctx, GRAV_EINVAL, "lambda must be >= 0");
    if (!(o.tol > 0) || !(o.tol < 1)) return set_error(ctx, GRAV_EINVAL, "tol must lie in (0, 1)");
    if (o.max_iter < 1) return set_error(ctx, GRAV_EINVAL, "max_iter must be >= 1");
    if (o.check_every < 0) return set_error(ctx, GRAV_EINVAL, "check_every must be >= 0");
    if (!(o.near_cells >= 1.0 && o.near_cells <= 16.0))
        return set_error(ctx, GRAV_EINVAL, "near_cells must lie in [1, 16]");
    if (!(o.timeout_s > 0)) return set_error(ctx, GRAV_EINVAL, "timeout_s must be > 0");
    if (o.precond < 0 || o.precond > 2)
        return set_error(ctx, GRAV_EINVAL, "precond must be 0 (none), 1 (Jacobi) or 2 (Nystrom)");
    if (o.precond == 2 && (o.nys_rank < 0 || o.nys_rank > 8192))
        return set_error(ctx, GRAV_EINVAL, "nys_rank must lie in [0 (automatic), 8192]");
    if (o.precond == 2 && (o.nys_coarsen < 0 || o.nys_coarsen > 8))
        return set_error(ctx, GRAV_EINVAL, "nys_coarsen must lie in [0 (automatic), 8]");
    if (o.cache_g != 0 && o.cache_g != 1) return set_error(ctx, GRAV_EINVAL, "cache_g must be 0 or 1");
    if (o.outer_max < 0 || o.outer_max > 100000) return set_error(ctx, GRAV_EINVAL, "outer_max must lie in [0, 1e5]");
    if (o.outer_max > 0 && o.inner_max < 1) return set_error(ctx, GRAV_EINVAL, "inner_max must be >= 1");
    if (o.check_stations < 0) return set_error(ctx, GRAV_EINVAL, "check_stations must be >= 0");
    if (o.reorth < 0 || o.reorth > kReorthMaxBasis)
        return set_error(ctx, GRAV_EINVAL, "reorth must lie in [0, %d]", kReorthMaxBasis);
    if (o.refine < 0 || o.refine > 64) return set_error(ctx, GRAV_EINVAL, "refine must lie in [0, 64]");
    if (o.near_fp64 != 0 && o.near_fp64 != 1) return set_error(ctx, GRAV_EINVAL, "near_fp64 must be 0 or 1");
    if (o.diag_fp64 != 0 && o.diag_fp64 != 1) return set_error(ctx, GRAV_EINVAL, "diag_fp64 must be 0 or 1");
    if (o.refine > 0 && (o.precision != GRAV_FP64 || o.outer_max > 0))
        return set_error(ctx, GRAV_EINVAL, "refine needs precision GRAV_FP64 and outer_max = 0");
    return GRAV_OK;
}

grav_options resolve(const grav_options *opt) {
    grav_options o;
    grav_options_default(&o);
    if (opt) o = *opt;
    return o;
}

// An empty survey (n == 0) is a valid no-op for the one-shot calls; this
// validates the rest of the arguments for that case.  Returns 1 when the
// survey is empty and everything else is valid, 0 when it is not empty, or a
// negative status.
int empty_survey(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const grav_options *opt) {
    if (!survey) return set_error(ctx, GRAV_EINVAL, "survey is NULL");
    if (survey->n != 0) return 0;
    int rc = check_options(ctx, resolve(opt));
    if (rc) return rc;
    if ((rc = check_mesh(ctx, mesh))) return rc;
    return 1;
}

}  // namespace

int host_wait(grav_ctx *ctx, cudaEvent_t ev, double timeout_s, const char *what) {
    return wait_event(ctx, ev, timeout_s, what);
}

void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

void stage_begin(const grav_plan *p, int stage, cudaStream_t s) {
    StageTimer &t = p->timer;
    if (!t.enabled) return;
    if (2 * (t.used + 1) > (int)t.pool.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            t.pool.push_back(e);
        }
    }
    t.stage_of.resize(t.used + 1);
    t.stage_of[t.used] = stage;
    cudaEventRecord(t.pool[2 * t.used], s);
}

void stage_end(const grav_plan *p, int stage, cudaStream_t s) {
    StageTimer &t = p->timer;
    if (!t.enabled) return;
    (void)stage;
    cudaEventRecord(t.pool[2 * t.used + 1], s);
    ++t.used;
}

int set_error(grav_ctx *ctx, int code, const char *fmt, ...) {
    char buf[768];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->last_error = buf;
    } else {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_last_error = buf;
    }
    return code;
}

int cuda_error(grav_ctx *ctx, cudaError_t e, const char *what) {
    return set_error(ctx, e == cudaErrorMemoryAllocation ? GRAV_ENOMEM : GRAV_EDEVICE, "%s: %s (%s)", what,
                     cudaGetErrorString(e), cudaGetErrorName(e));
}

// ---------------------------------------------------------------------------
// plan internals shared with the solver and the serving scheduler
// ---------------------------------------------------------------------------
namespace {

void fp64_sizes(grav_plan *p, int sm) {
    const int64_t target = (int64_t)sm * 5 * 8;
    p->ldw = (p->nx + 1 + 1) / 2 * 2;
    const int nrows = (p->ny + 1) * (p->nz + 1);
    const int64_t tiles = (p->N + 255) / 256;
    int nch = (int)std::min<int64_t>(std::max<int64_t>(1, (target + tiles - 1) / tiles), nrows);
    p->f64_rows_per_chunk = (nrows + nch - 1) / nch;
    p->f64_nchunk = (nrows + p->f64_rows_per_chunk - 1) / p->f64_rows_per_chunk;
    const int ngz = (p->nz + 1 + 7) / 8;
    p->a64_groups = (int)((int64_t)(p->nx + 1) * (p->ny + 1) * ngz);
    const int64_t ctas = (p->a64_groups + 7) / 8;
    int64_t nsch = std::max<int64_t>(1, (target + ctas - 1) / ctas);
    nsch = std::min<int64_t>(nsch, (p->N + 255) / 256);
    int64_t len = (p->N + nsch - 1) / nsch;
    len = (len + 255) / 256 * 256;
    p->a64_schunk_len = (int)len;
    p->a64_nschunk = (int)((p->N + len - 1) / len);
    const int64_t dt = (p->N + 127) / 128;
    int dch = (int)std::min<int64_t>(std::max<int64_t>(1, (target + dt - 1) / dt), p->ny);
    p->f64_diag_jrows = (p->ny + dch - 1) / dch;
    p->f64_diag_nchunk = (p->ny + p->f64_diag_jrows - 1) / p->f64_diag_jrows;
}

size_t fp64_bytes(const grav_plan *p) {
    const size_t nrows = (size_t)(p->ny + 1) * (p->nz + 1);
    size_t b = 0;
    auto add = [&](size_t v) { b += (v + 255) / 256 * 256 + 256; };
    add(nrows * p->ldw * 8);                                                   // w
    add((size_t)std::max(p->f64_nchunk, p->f64_diag_nchunk) * p->N * 8);       // part
    add((size_t)p->N * 32);                                                    // st4
    add((size_t)p->a64_nschunk * p->Nn * 8);                                   // upart
    add((size_t)p->Nn * 8);                                                    // u
    return b;
}

}  // namespace

int plan_forward_ex(grav_plan *p, const double *m, double *d, const double *add, double add_scale,
                    cudaStream_t s) {
    NvtxRange nv("grav::forward");
    if (p->cached) {
        launch_cached_fwd(p, m, add, add_scale, d, s);
    } else if (p->opt.precision == GRAV_FP64) {
        launch_node_weights(p, m, s);
        launch_fwd64(p, s);
        launch_reduce_rows(p->part, p->f64_nchunk, p->N, kGammaMgal, add, add_scale, nullptr, d, s);
    } else if (p->opt.precision == GRAV_MIXED_CORNER) {
        launch_corner_fwd(p, m, s);
        launch_mixed_prep_q(p, m, s, false);   // the near field reads q
        launch_mixed_near_fwd(p, m, s);
        launch_reduce_rows(p->cr_part, p->cr_nchunk, p->N, kGammaMgal, add, add_scale, p->near_corr, d, s);
    } else {
        launch_mixed_prep_q(p, m, s, true);
        launch_mixed_fwd(p, s);
        launch_mixed_near_fwd(p, m, s);
        launch_reduce_rows(p->m_part, p->m_fwd_nchunk, p->N, 1.0, add, add_scale, p->near_corr, d, s, p->mmax_bits);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRAV_OK : cuda_error(p->ctx, e, "forward launch");
}

int plan_adjoint_ex(grav_plan *p, const double *r, double *out, int depth_weighted, const double *add,
                    cudaStream_t s) {
    NvtxRange nv("grav::adjoint");
    if (p->opt.precision == GRAV_MIXED_CORNER)
        return set_error(p->ctx, GRAV_EINVAL, "GRAV_MIXED_CORNER provides the forward product only");
    if (p->cached) {
        launch_cached_adj(p, r, depth_weighted, add, out, s);
    } else if (p->opt.precision == GRAV_FP64) {
        launch_adj64(p, r, s);
        launch_adj_finish(p, p->u, kGammaMgal, depth_weighted, add, out, s);
    } else {
        launch_mixed_adj(p, r, s);
        launch_mixed_adj_finish(p, r, depth_weighted, add, out, s);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRAV_OK : cuda_error(p->ctx, e, "adjoint launch");
}

int plan_diag(grav_plan *p, double *diag, cudaStream_t s) {
    NvtxRange nv("grav::diag");
    if (p->opt.precision == GRAV_MIXED_CORNER)
        return set_error(p->ctx, GRAV_EINVAL, "GRAV_MIXED_CORNER provides the forward product only");
    if (p->cached) launch_cached_diag(p, diag, s);
    else if (p->opt.precision == GRAV_FP64) launch_diag64(p, diag, s);
    else launch_mixed_diag(p, diag, s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRAV_OK : cuda_error(p->ctx, e, "diag launch");
}

int plan_prepare(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const grav_options &o,
                 grav_plan **out) {
    if (!out) return set_error(ctx, GRAV_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh || !survey) return set_error(ctx, GRAV_EINVAL, "mesh or survey is NULL");
    int rc = check_options(ctx, o);
    if (rc) return rc;
    if ((rc = check_mesh(ctx, mesh))) return rc;
    if (survey->n < 1 || survey->n > ((int64_t)1 << 30))
        return set_error(ctx, GRAV_EINVAL, "survey size must lie in [1, 2^30] (got %lld)", (long long)survey->n);
    if (!is_device_ptr(survey->x, ctx->device) || !is_device_ptr(survey->y, ctx->device) ||
        !is_device_ptr(survey->z, ctx->device))
        return set_error(ctx, GRAV_EINVAL, "survey x/y/z must be device pointers on device %d", ctx->device);

    grav_plan *p = new grav_plan();
    p->ctx = ctx;
    p->opt = o;
    p->nx = mesh->nx; p->ny = mesh->ny; p->nz = mesh->nz;
    p->N = survey->n;
    p->M = (int64_t)p->nx * p->ny * p->nz;
    p->Nn = (int64_t)(p->nx + 1) * (p->ny + 1) * (p->nz + 1);
    p->xe.assign(mesh->xe, mesh->xe + p->nx + 1);
    p->ye.assign(mesh->ye, mesh->ye + p->ny + 1);
    p->ze.assign(mesh->ze, mesh->ze + p->nz + 1);
    p->sx = survey->x; p->sy = survey->y; p->sz = survey->z;
    {
        const double a = p->xe[1] - p->xe[0];
        const double b = p->ye[1] - p->ye[0];
        const double c = p->ze[1] - p->ze[0];
        auto uni = [&](const std::vector<double> &e, double h) {
            for (size_t i = 0; i + 1 < e.size(); ++i)
                if (std::fabs((e[i + 1] - e[i]) - h) > 1e-9 * h) return false;
            return true;
        };
        p->uniform = uni(p->xe, a) && uni(p->ye, b) && uni(p->ze, c);
        p->cubic = p->uniform && std::fabs(a - b) <= 1e-9 * a && std::fabs(a - c) <= 1e-9 * a;
        p->cell_a = a;
        p->cell_b = b;
        p->cell_c = c;
    }
    if (o.precision == GRAV_FP64 && p->nx + 1 > fwd64_max_nodes_x()) {
        delete p;
        return set_error(ctx, GRAV_EINVAL,
                         "GRAV_FP64 stages one row of nx+1 node weights in shared memory: nx+1 must be <= %d "
                         "(got %d)",
                         fwd64_max_nodes_x(), mesh->nx + 1);
    }
    if (o.precision != GRAV_FP64 && !p->uniform) {
        delete p;
        return set_error(ctx, GRAV_EINVAL,
                         "GRAV_MIXED needs a uniform mesh (constant dx, dy and dz; they may differ from each other)");
    }
    size_t bytes = 0;
    auto add = [&](size_t v) { bytes += (v + 255) / 256 * 256 + 256; };
    add(8ull * (p->nx + 1)); add(8ull * (p->ny + 1)); add(8ull * (p->nz + 1)); add(8ull * p->nz);
    if (o.precision == GRAV_FP64) {
        fp64_sizes(p, ctx->sm_count);
        bytes += fp64_bytes(p);
        // stored G when asked for and it fits next to what is already in use
        const double gbytes = 8.0 * (double)p->N * (double)p->M;
        // forward: tiles of 4,096 stations x cell chunks, four full waves of
        // resident CTAs (a wave that is only partly filled costs as much as a
        // full one: 2 tiles x 256 chunks at 3 CTAs per SM ran 1.15 waves and
        // 34 % slower), at most 1,024 chunks of partials
        const int64_t tiles = cached_fwd_tiles(p->N);
        const int64_t resident = (int64_t)ctx->sm_count * cached_fwd_ctas_per_sm();
        const int cnch = (int)std::min<int64_t>(
            std::min<int64_t>(std::max<int64_t>(1, (4 * resident + tiles - 1) / tiles), 1024), p->M);
        if (o.cache_g && (double)ctx->hbm_used.load() + (double)bytes + gbytes + 8.0 * p->N * cnch <= (double)ctx->hbm_budget) {
            p->cached = 1;
            p->c_nchunk = cnch;
            bytes += (size_t)gbytes + 256 + 8ull * (p->M + p->N) + 512;   // G, m and r as pairs
            // the forward partials reuse `part`; make sure it has c_nchunk rows
            const int rows = std::max(p->f64_nchunk, p->f64_diag_nchunk);
            if (p->c_nchunk > rows) bytes += (size_t)(p->c_nchunk - rows) * p->N * 8 + 256;
        }
    } else {
        // the window radius is k cell widths, width = the largest cell edge
        const double L = std::max(p->cell_a, std::max(p->cell_b, p->cell_c));
        const double k = o.near_cells;
        p->ng.radius_cells = k;
        p->ng.width = L;
        p->ng.bx = (int)std::ceil(2.0 * k * L / p->cell_a) + 1;
        p->ng.by = (int)std::ceil(2.0 * k * L / p->cell_b) + 1;
        int bz = 0;
        for (int l = 0; l < p->nz; ++l)
            if (0.5 * (p->ze[l] + p->ze[l + 1]) - p->ze[0] < k * L) bz = l + 1;
        p->ng.bz = std::max(1, bz);
        p->ng.slots = p->ng.bx * p->ng.by * p->ng.bz;
        p->ng.ld = (p->ng.slots + 3) / 4 * 4;
        p->ng.nbx = p->nx + p->ng.bx - 1;
        p->ng.nby = p->ny + p->ng.by - 1;
        bytes += mixed_scratch_bytes(p);
        if (near_setup_warps(p) < 1) {
            delete p;
            return set_error(ctx, GRAV_EINVAL, "near_cells window too large for this mesh (shared-memory limit)");
        }
    }
    p->bytes = bytes;
    *out = p;
    return GRAV_OK;
}

// Allocates the prepared plan's arena from the context pool (stream-ordered)
// and enqueues its set-up.  On failure the plan is deleted.
int plan_allocate(grav_plan *p, cudaStream_t s) {
    grav_ctx *ctx = p->ctx;
    const grav_options &o = p->opt;
    const size_t bytes = p->bytes;
    int rc = GRAV_OK;
    if (ctx->hbm_used.load() + bytes > ctx->hbm_budget) {
        delete p;
        return set_error(ctx, GRAV_ENOMEM, "plan needs %.3f GB; context budget %.3f GB, %.3f GB in use", bytes / 1e9,
                         ctx->hbm_budget / 1e9, ctx->hbm_used.load() / 1e9);
    }
    void *base = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&base, bytes, ctx->pool, s);
    if (e != cudaSuccess) {
        delete p;
        return cuda_error(ctx, e, "plan allocation");
    }
    ctx->hbm_used += bytes;
    p->arena.base = (char *)base;
    p->arena.size = bytes;
    p->d_xe = (double *)p->arena.take(8ull * (p->nx + 1));
    p->d_ye = (double *)p->arena.take(8ull * (p->ny + 1));
    p->d_ze = (double *)p->arena.take(8ull * (p->nz + 1));
    p->d_w2 = (double *)p->arena.take(8ull * p->nz);
    std::vector<double> w2(p->nz);
    for (int l = 0; l < p->nz; ++l) {
        const double zc = 0.5 * (p->ze[l] + p->ze[l + 1]) - p->ze[0];
        w2[l] = (zc + o.z0) * (zc + o.z0);
    }
    cudaMemcpyAsync(p->d_xe, p->xe.data(), 8ull * (p->nx + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->d_ye, p->ye.data(), 8ull * (p->ny + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->d_ze, p->ze.data(), 8ull * (p->nz + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->d_w2, w2.data(), 8ull * p->nz, cudaMemcpyHostToDevice, s);
    if (o.precision == GRAV_FP64) {
        const size_t nrows = (size_t)(p->ny + 1) * (p->nz + 1);
        p->w = (double *)p->arena.take(nrows * p->ldw * 8);
        p->part = (double *)p->arena.take((size_t)std::max(std::max(p->f64_nchunk, p->f64_diag_nchunk), p->c_nchunk) *
                                          p->N * 8);
        p->st4 = (double4_16a *)p->arena.take((size_t)p->N * 32);
        p->upart = (double *)p->arena.take((size_t)p->a64_nschunk * p->Nn * 8);
        p->u = (double *)p->arena.take((size_t)p->Nn * 8);
        if (p->cached) {
            p->Gc = (float2 *)p->arena.take((size_t)p->N * p->M * 8);
            p->m_df = (float2 *)p->arena.take((size_t)p->M * 8);
            p->r_df = (float2 *)p->arena.take((size_t)p->N * 8);
        }
        if (!p->arena.overflow) {
            fp64_setup(p, s);
            if (p->cached) launch_build_g64(p, p->Gc, nullptr, s);
        }
    } else {
        rc = mixed_setup(p, s);
    }
    if (rc || p->arena.overflow) {
        cudaFreeAsync(base, s);
        ctx->hbm_used -= bytes;
        delete p;
        return set_error(ctx, GRAV_EDEVICE, "internal: plan set-up failed (arena overflow or bad window)");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(base, s);
        ctx->hbm_used -= bytes;
        delete p;
        return cuda_error(ctx, e, "plan set-up");
    }
    return GRAV_OK;
}

// FP64 check of a product d = G m of plan p at n_check evenly spaced stations:
// a transient FP64 plan over those stations evaluates G m exactly (Eq. 1-3).
int check_fp64(grav_plan *p, const double *m, const double *d, int n_check, double *max_abs, double *rel,
               cudaStream_t s) {
    grav_ctx *ctx = p->ctx;
    if (n_check < 1 || n_check > p->N) return set_error(ctx, GRAV_EINVAL, "n_check must lie in [1, n]");
    double *buf = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&buf, 40ull * n_check + 8, ctx->pool, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "check scratch");
    double *sx = buf, *sy = buf + n_check, *sz = buf + 2 * n_check, *dg = buf + 3 * n_check, *d64 = buf + 4 * n_check;
    unsigned long long *dmax = reinterpret_cast<unsigned long long *>(buf + 5 * n_check);
    launch_gather_check(p->sx, p->sy, p->sz, d, p->N, n_check, sx, sy, sz, dg, s);
    launch_absmax(d, p->N, dmax, s);   // max |d| over every station: the scale of the tolerance
    grav_mesh mesh{p->nx, p->ny, p->nz, p->xe.data(), p->ye.data(), p->ze.data()};
    grav_survey sub{n_check, sx, sy, sz};
    grav_options o;
    grav_options_default(&o);
    o.z0 = p->opt.z0;
    o.timeout_s = p->opt.timeout_s;
    grav_plan *q = nullptr;
    int rc = plan_create(ctx, &mesh, &sub, o, &q, s);
    if (!rc) {
        rc = plan_forward_ex(q, m, d64, nullptr, 0.0, s);
        plan_destroy(q, s);
    }
    std::vector<double> h(2ull * n_check + 1);
    if (!rc) {
        cudaMemcpyAsync(h.data(), dg, 16ull * n_check + 8, cudaMemcpyDeviceToHost, s);
        rc = read_status(ctx, s, p->opt.timeout_s);
    }
    cudaFreeAsync(buf, s);
    if (rc) return rc;
    // the error is stated relative to max |g| over the whole survey: the
    // checked stations' FP64 values, or the largest |d_i| anywhere (d agrees
    // with the FP64 operator to the error being stated), whichever is larger;
    // a sample that misses the anomaly would otherwise inflate it
    double ea = 0.0, ma = 0.0;
    for (int k = 0; k < n_check; ++k) {
        ea = std::max(ea, std::fabs(h[k] - h[n_check + k]));
        ma = std::max(ma, std::fabs(h[n_check + k]));
    }
    unsigned long long bits = 0;
    std::memcpy(&bits, &h[2ull * n_check], 8);
    double dall = 0.0;
    std::memcpy(&dall, &bits, 8);
    if (std::isfinite(dall)) ma = std::max(ma, dall);
    if (max_abs) *max_abs = ea;
    if (rel) *rel = ma > 0 ? ea / ma : ea;
    return GRAV_OK;
}

int plan_create(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const grav_options &o,
                grav_plan **out, cudaStream_t s) {
    NvtxRange nv("grav::plan_create");
    grav_plan *p = nullptr;
    int rc = plan_prepare(ctx, mesh, survey, o, &p);
    if (rc) return rc;
    rc = plan_allocate(p, s);
    if (rc) return rc;
    *out = p;
    return GRAV_OK;
}

// Basis vectors kept by the reorthogonalised CG (0: plain CG).
int reorth_cap(const grav_plan *p) {
    const grav_options &o = p->opt;
    if (o.reorth <= 0 || o.precond == 1 || o.outer_max > 0) return 0;
    return (int)std::min<int64_t>(o.reorth, (int64_t)o.max_iter + 1);
}

size_t solve_bytes(const grav_plan *p) {
    const int cap = reorth_cap(p);
    // reorthogonalisation: one basis, two (residuals and preconditioned residuals) with precond = 2
    const size_t bases = (p->opt.precond == 2 ? 2ull : 1ull) * cap * p->N;
    return 8ull * (12 * p->N + p->M + kDotBlocks + kSCount) + 16 * 256 + 8ull * (bases + cap) + 3 * 256;
}

size_t plan_resident_bytes(const grav_plan *p) {
    return p->bytes + (p->nys_kept ? static_cast<const NysState *>(p->nys_kept)->bytes : 0);
}

void plan_destroy(grav_plan *p, cudaStream_t s) {
    if (!p) return;
    if (p->nys_kept) {
        NysState *k = static_cast<NysState *>(p->nys_kept);
        nys_free(p, k, s);
        delete k;
        p->nys_kept = nullptr;
    }
    for (cudaEvent_t e : p->timer.pool) cudaEventDestroy(e);
    if (p->arena.base) cudaFreeAsync(p->arena.base, s);
    p->ctx->hbm_used -= p->bytes;
    delete p;
}

int read_status(grav_ctx *ctx, cudaStream_t s, double timeout_s) {
    // one pinned host mirror per host thread (serving slots read concurrently)
    thread_local int *h_status = nullptr;
    if (!h_status && cudaMallocHost((void **)&h_status, 64) != cudaSuccess) return cuda_error(ctx, cudaGetLastError(), "pinned status");
    *h_status = 0;
    cudaMemcpyAsync(h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, s);
    int rc = wait_event(ctx, ev, timeout_s, "stream synchronisation");
    cudaEventDestroy(ev);
    if (rc) return rc;
    if (*h_status != 0) {
        const int st = *h_status;
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
        return set_error(ctx, GRAV_EDEVICE, "device status word 0x%x (bounded device wait expired)", st);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRAV_OK : cuda_error(ctx, e, "device");
}

// ---------------------------------------------------------------------------
// Data-space CG: A = G W^-2 G^T + lambda I, y0 = 0, r0 = dd.
// ---------------------------------------------------------------------------
int solve_on_plan(grav_plan *p, const double *d, const double *m_ref, double *m_out, double *y_out,
                  grav_solve_info *info, cudaStream_t s, const std::atomic<int> *cancel, const double *y0,
                  double *hist, int hist_len) {
    NvtxRange nv("grav::solve");
    grav_ctx *ctx = p->ctx;
    const grav_options &o = p->opt;
    const double t0 = now_s();
    const int64_t N = p->N, M = p->M;
    if (o.precision == GRAV_MIXED_CORNER)
        return set_error(ctx, GRAV_EINVAL, "GRAV_MIXED_CORNER provides the forward product only (no inversion)");
    const size_t bytes = solve_bytes(p);
    if (ctx->hbm_used.load() + bytes > ctx->hbm_budget) return set_error(ctx, GRAV_ENOMEM, "solve vectors exceed budget");
    char *base = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&base, bytes, ctx->pool, s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "solve allocation");
    ctx->hbm_used += bytes;
    Arena ar;
    ar.base = base; ar.size = bytes;
    double *dd = (double *)ar.take(8ull * N);
    double *r = (double *)ar.take(8ull * N);
    double *y = (double *)ar.take(8ull * N);
    double *pv = (double *)ar.take(8ull * N);
    double *Ap = (double *)ar.take(8ull * N);
    double *q = (double *)ar.take(8ull * M);
    double *zv = (double *)ar.take(8ull * N);     // z = M^-1 r (preconditioned CG)
    double *dinv = (double *)ar.take(8ull * N);   // diag(A)^-1 (preconditioned CG)
    double *yo = (double *)ar.take(8ull * N);     // outer loop: accumulated y
    double *Ay = (double *)ar.take(8ull * N);     // outer loop: A y
    double *ro = (double *)ar.take(8ull * N);     // outer loop: dd - A y
    double *wv = (double *)ar.take(8ull * N);     // outer loop: work vectors
    double *fv = (double *)ar.take(8ull * N);
    double *dp = (double *)ar.take(8ull * kDotBlocks);
    double *sc = (double *)ar.take(8ull * kSCount);
    const int cap = reorth_cap(p);
    double *Qb = cap ? (double *)ar.take(8ull * cap * N) : nullptr;   // reorthogonalisation basis [cap][N]
    double *cb = cap ? (double *)ar.take(8ull * cap) : nullptr;
    double *Wb = (cap && o.precond == 2) ? (double *)ar.take(8ull * cap * N) : nullptr;   // M^-1 Qb rows
    NysState ns;
    double *hsc = nullptr;     // [0, kSCount): synchronous reads; then two slots of the CG pipeline
    cudaMallocHost((void **)&hsc, 3 * 8 * kSCount);
    double *hpipe = hsc + kSCount;
    cudaEvent_t ev, evp[2];
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&evp[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&evp[1], cudaEventDisableTiming);
    int rc = GRAV_OK;
    double lam = o.lambda, trace = 0.0;
    int iters = 0;
    bool converged = false;
    auto sync_scalars = [&](const char *what) -> int {
        cudaMemcpyAsync(hsc, sc, 8 * kSCount, cudaMemcpyDeviceToHost, s);
        cudaEventRecord(ev, s);
        return wait_event(ctx, ev, o.timeout_s, what);
    };
    if (hist && hist_len > 0) vec_fill(hist, hist_len, -1.0, s);
    do {
        cudaMemsetAsync(sc, 0, 8 * kSCount, s);
        // dd = d - G m_ref
        if (m_ref) {
            if ((rc = plan_forward_ex(p, m_ref, Ap, nullptr, 0.0, s))) break;
            vec_axpby(1.0, d, -1.0, Ap, N, dd, s);
        } else {
            cudaMemcpyAsync(dd, d, 8ull * N, cudaMemcpyDeviceToDevice, s);
        }
        // lambda = lambda_scale * trace(G W^-2 G^T) / N; the diagonal also feeds
        // the Jacobi preconditioner M = diag(G W^-2 G^T + lambda I)
        const bool jac = o.precond == 1, nys = o.precond == 2, pc = jac || nys;
        if (!(lam > 0) && !jac && p->trace_cache > 0) {
            // a resident plan (serving) keeps the trace of its first solve: the
            // same deterministic value, without another diagonal pass
            trace = p->trace_cache;
            lam = o.lambda_scale * trace / (double)N;
        } else if (!(lam > 0) || jac) {
            if ((rc = plan_diag(p, dinv, s))) break;
            if (!(lam > 0)) {
                launch_dot(dinv, nullptr, N, dp, sc + kSTrace, s);
                if ((rc = sync_scalars("trace"))) break;
                trace = hsc[kSTrace];
                if (trace > 0 && std::isfinite(trace)) p->trace_cache = trace;
                lam = o.lambda_scale * trace / (double)N;
                if (!(lam > 0) || !std::isfinite(lam)) {
                    rc = set_error(ctx, GRAV_EDEVICE, "lambda from the trace is not positive (trace %g)", trace);
                    break;
                }
            }
            if (jac) vec_jacobi_inv(dinv, lam, N, dinv, s);
        }
        const double t_nys = now_s();
        if (nys) {
            int ell = o.nys_rank, cf = o.nys_coarsen;
            nys_sizes(p, &ell, &cf);
            const uint64_t seed = 0x243F6A8885A308D3ull;
            const double key[4] = {lam, (double)ell, (double)cf, (double)(seed >> 11)};
            NysState *kept = static_cast<NysState *>(p->nys_kept);
            if (kept && std::equal(key, key + 4, p->nys_key)) {
                ns = *kept;   // the resident preconditioner of an earlier solve on this plan
                *kept = NysState{};
                delete kept;
                p->nys_kept = nullptr;
            } else {
                if (kept) {   // different lambda or sizes: replace it
                    nys_free(p, kept, s);
                    delete kept;
                    p->nys_kept = nullptr;
                }
                if ((rc = nys_build(p, lam, ell, cf, seed, &ns, s))) break;
            }
            std::copy(key, key + 4, p->nys_key);
        }
        const double nys_setup_s = nys ? now_s() - t_nys : 0.0;
        // z = M^-1 r: Jacobi or the Nystrom preconditioner
        auto apply_prec = [&](const double *rv, double *z) {
            if (nys) nys_apply(ns, rv, z, s);
            else vec_mul(dinv, rv, N, z, s);
        };
        double true_rel = 0.0;
        // one CG iteration on A x = b with x in `xv`, residual `rv`, direction pv
        auto cg_step = [&](double *xv, double *rv, int it_global) -> int {
            int r2 = plan_adjoint_ex(p, pv, q, 1, nullptr, s);
            if (!r2) r2 = plan_forward_ex(p, q, Ap, pv, lam, s);
            if (r2) return r2;
            launch_dot(pv, Ap, N, dp, sc + kSPAp, s);
            cg_alpha(sc, s);
            cg_update_yr(xv, rv, pv, Ap, N, sc, s);
            if (pc) {
                apply_prec(rv, zv);
                launch_dot(rv, zv, N, dp, sc + kSRRNew, s);
                launch_dot(rv, rv, N, dp, sc + kSResNew, s);
                cg_beta(sc, it_global, kSResNew, s);
                cg_update_p(pv, zv, N, sc, s);
            } else {
                launch_dot(rv, rv, N, dp, sc + kSRRNew, s);
                cg_beta(sc, it_global, kSRRNew, s);
                cg_update_p(pv, rv, N, sc, s);
            }
            return GRAV_OK;
        };
        int outer_done = 0, restarts = 0;
        double alpha_min = 1.0;
        if (o.outer_max > 0) {
            // The paper's outer model-update loop in data space (m = m_ref + W^-2 G^T y):
            // dy from <= inner_max CG iterations on A dy = dd - A y, then y += alpha dy
            // with alpha halved until the objective of Eq. 7 decreases.  Along the
            // step phi(alpha) is a quadratic whose coefficients are dot products:
            //   d - G m = e0 + alpha e1, e0 = r + lam y, e1 = lam dy - A dy
            //   (m - m_ref)^T W_m^-1 (m - m_ref) = (y + alpha dy)^T (f0 + alpha f1),
            //   f0 = A y - lam y, f1 = A dy - lam dy.
            if (y0) cudaMemcpyAsync(yo, y0, 8ull * N, cudaMemcpyDeviceToDevice, s);
            else vec_fill(yo, N, 0.0, s);
            launch_dot(dd, dd, N, dp, sc + kSTmp, s);
            if ((rc = sync_scalars("outer start"))) break;
            const double bb0 = hsc[kSTmp];
            int total_it = 0;
            for (int k = 0;; ++k) {
                if ((rc = plan_adjoint_ex(p, yo, q, 1, nullptr, s))) break;
                if ((rc = plan_forward_ex(p, q, Ay, yo, lam, s))) break;
                vec_axpby(1.0, dd, -1.0, Ay, N, ro, s);
                launch_dot(ro, ro, N, dp, sc + kSTmp, s);
                if ((rc = sync_scalars("outer residual"))) break;
                true_rel = bb0 > 0 ? std::sqrt(hsc[kSTmp] / bb0) : 0.0;
                if (true_rel <= o.tol || k >= o.outer_max || total_it >= o.max_iter) break;
                if (cancel && cancel->load()) {
                    rc = set_error(ctx, GRAV_ECANCELED, "solve cancelled");
                    break;
                }
                // inner CG from dy = 0 (dy in y, residual in r)
                cudaMemcpyAsync(r, ro, 8ull * N, cudaMemcpyDeviceToDevice, s);
                vec_fill(y, N, 0.0, s);
                if (pc) {
                    vec_mul(dinv, r, N, zv, s);
                    cudaMemcpyAsync(pv, zv, 8ull * N, cudaMemcpyDeviceToDevice, s);
                    launch_dot(r, zv, N, dp, sc + kSRR, s);
                    launch_dot(r, r, N, dp, sc + kSTmp, s);
                    cg_set_scalars(sc, o.tol * o.tol, kSTmp, s);
                } else {
                    cudaMemcpyAsync(pv, r, 8ull * N, cudaMemcpyDeviceToDevice, s);
                    launch_dot(r, r, N, dp, sc + kSRR, s);
                    cg_set_scalars(sc, o.tol * o.tol, kSRR, s);
                }
                const int n_in = std::min(o.inner_max, o.max_iter - total_it);
                for (int it = 0; it < n_in && !rc; ++it) rc = cg_step(y, r, total_it + it);
                if (rc) break;
                // A dy and the line-search dot products
                if ((rc = plan_adjoint_ex(p, y, q, 1, nullptr, s))) break;
                if ((rc = plan_forward_ex(p, q, Ap, y, lam, s))) break;
                vec_axpby(1.0, ro, lam, yo, N, wv, s);          // e0
                vec_axpby(lam, y, -1.0, Ap, N, fv, s);          // e1
                launch_dot(wv, wv, N, dp, sc + kSPhi + 0, s);
                launch_dot(wv, fv, N, dp, sc + kSPhi + 1, s);
                launch_dot(fv, fv, N, dp, sc + kSPhi + 2, s);
                vec_axpby(1.0, Ay, -lam, yo, N, wv, s);         // f0
                vec_axpby(1.0, Ap, -lam, y, N, fv, s);          // f1
                launch_dot(yo, wv, N, dp, sc + kSPhi + 3, s);
                launch_dot(yo, fv, N, dp, sc + kSPhi + 4, s);
                launch_dot(y, wv, N, dp, sc + kSPhi + 5, s);
                launch_dot(y, fv, N, dp, sc + kSPhi + 6, s);
                if ((rc = sync_scalars("outer line search"))) break;
                if (hsc[kSFrozen] == 2.0) {
                    rc = set_error(ctx, GRAV_EDEVICE, "CG breakdown: p.Ap <= 0 (operator not SPD in this precision)");
                    break;
                }
                total_it = (int)hsc[kSIters];
                const double *c = hsc + kSPhi;
                auto phi = [&](double a) {
                    return (c[0] + 2 * a * c[1] + a * a * c[2]) / lam + c[3] + a * (c[4] + c[5]) + a * a * c[6];
                };
                const double phi0 = phi(0.0);
                double alpha = 1.0;
                while (phi(alpha) >= phi0 && alpha > 1.0 / 1024) alpha *= 0.5;
                alpha_min = std::min(alpha_min, alpha);
                vec_axpby(1.0, yo, alpha, y, N, yo, s);
                outer_done = k + 1;
            }
            if (rc) break;
            cudaMemcpyAsync(y, yo, 8ull * N, cudaMemcpyDeviceToDevice, s);
            iters = total_it;
            converged = true_rel <= o.tol;
        } else {
        // start: y = y0 (or 0), r = dd - A y; convergence is relative to ||dd||
        if (y0) {
            cudaMemcpyAsync(y, y0, 8ull * N, cudaMemcpyDeviceToDevice, s);
            if ((rc = plan_adjoint_ex(p, y, q, 1, nullptr, s))) break;
            if ((rc = plan_forward_ex(p, q, Ap, y, lam, s))) break;
            vec_axpby(1.0, dd, -1.0, Ap, N, r, s);
        } else {
            cudaMemcpyAsync(r, dd, 8ull * N, cudaMemcpyDeviceToDevice, s);
            vec_fill(y, N, 0.0, s);
        }
        launch_dot(dd, dd, N, dp, sc + kSBB0, s);
        if (pc) {
            apply_prec(r, zv);
            cudaMemcpyAsync(pv, zv, 8ull * N, cudaMemcpyDeviceToDevice, s);
            launch_dot(r, zv, N, dp, sc + kSRR, s);
        } else {
            cudaMemcpyAsync(pv, r, 8ull * N, cudaMemcpyDeviceToDevice, s);
            launch_dot(r, r, N, dp, sc + kSRR, s);
        }
        cg_set_scalars(sc, o.tol * o.tol, kSBB0, s);
        // an iterate that already meets tol needs no iteration
        launch_dot(r, r, N, dp, sc + kSTmp, s);
        cg_restart(sc, 0, s);
        int kb = 0;            // basis vectors stored (reorthogonalised CG)
        const bool reo = cap > 0;   // reorthogonalise (every restart starts a fresh basis)
        // first basis vector: r / sqrt(r.z) (and z / sqrt(r.z) with the Nystrom preconditioner)
        auto basis_start = [&]() {
            cg_basis_append(Qb, r, N, sc, kSRR, s);
            if (Wb) cg_basis_append(Wb, zv, N, sc, kSRR, s);
            kb = 1;
        };
        if (reo) basis_start();
        if ((rc = sync_scalars("cg start"))) break;
        if (hsc[kSFrozen] != 0.0) {
            converged = true;
        }
        const double work = (double)N * (double)M;
        const int every = o.check_every > 0 ? o.check_every : (work > 2e8 ? 1 : 8);
        int it = 0;
        // CG; when the recurrence residual reaches tol, the residual is
        // recomputed from y with the operator itself (r = dd - A y); if that
        // true residual is still above tol, CG restarts from it (p = r).
        for (restarts = 0;; ++restarts) {
            // Batches of `every` iterations are enqueued one ahead of the
            // convergence check: while the host waits for the scalars of batch
            // b (copied into a pinned slot of their own), batch b + 1 already
            // runs, so the GPU does not idle on the host between batches.  An
            // iteration after the device froze the state (converged or broken
            // down) changes no vector, and the work after this loop is ordered
            // behind it on the stream.
            int queued = 0, head = 0;   // batches in flight; slot of the oldest
            while (!converged) {
                while (queued < 2 && it < o.max_iter) {
                    const int n_it = std::min(every, o.max_iter - it);
                    for (int k = 0; k < n_it; ++k, ++it) {
                        if ((rc = plan_adjoint_ex(p, pv, q, 1, nullptr, s))) break;
                        if ((rc = plan_forward_ex(p, q, Ap, pv, lam, s))) break;
                        launch_dot(pv, Ap, N, dp, sc + kSPAp, s);
                        cg_alpha(sc, s);
                        cg_update_yr(y, r, pv, Ap, N, sc, s);
                        if (pc) {
                            // precond = 2: the residual is made orthogonal to the earlier ones in
                            // the M^-1 inner product (r -= V (W^T r), twice) before z = M^-1 r
                            if (reo) cg_reorth2(Wb, Qb, kb, N, r, cb, sc, s);
                            apply_prec(r, zv);
                            launch_dot(r, zv, N, dp, sc + kSRRNew, s);
                            launch_dot(r, r, N, dp, sc + kSResNew, s);
                            cg_beta(sc, it, kSResNew, s, hist, hist_len);
                            if (reo && kb < cap) {
                                cg_basis_append(Qb + (size_t)kb * N, r, N, sc, kSRRNew, s);
                                cg_basis_append(Wb + (size_t)kb * N, zv, N, sc, kSRRNew, s);
                                ++kb;
                            }
                            cg_update_p(pv, zv, N, sc, s);
                        } else {
                            if (reo) cg_reorth(Qb, kb, N, r, cb, sc, s);
                            launch_dot(r, r, N, dp, sc + kSRRNew, s);
                            cg_beta(sc, it, kSRRNew, s, hist, hist_len);
                            if (reo && kb < cap) {
                                cg_basis_append(Qb + (size_t)kb * N, r, N, sc, kSRRNew, s);
                                ++kb;
                            }
                            cg_update_p(pv, r, N, sc, s);
                        }
                    }
                    if (rc) break;
                    const int slot = (head + queued) & 1;
                    cudaMemcpyAsync(hpipe + (size_t)slot * kSCount, sc, 8 * kSCount, cudaMemcpyDeviceToHost, s);
                    cudaEventRecord(evp[slot], s);
                    ++queued;
                }
                if (rc || queued == 0) break;
                if ((rc = wait_event(ctx, evp[head], o.timeout_s, "cg iteration"))) break;
                const double *hb = hpipe + (size_t)head * kSCount;
                head ^= 1;
                --queued;
                if (hb[kSFrozen] == 2.0) {
                    rc = set_error(ctx, GRAV_EDEVICE, "CG breakdown: p.Ap <= 0 (operator not SPD in this precision)");
                    break;
                }
                if (hb[kSFrozen] != 0.0) converged = true;
                if (cancel && cancel->load()) {
                    rc = set_error(ctx, GRAV_ECANCELED, "solve cancelled");
                    break;
                }
            }
            if (rc) break;
            // true residual dd - (G W^-2 G^T y + lambda y) into r
            if ((rc = plan_adjoint_ex(p, y, q, 1, nullptr, s))) break;
            if ((rc = plan_forward_ex(p, q, Ap, y, lam, s))) break;
            vec_axpby(1.0, dd, -1.0, Ap, N, r, s);
            launch_dot(r, r, N, dp, sc + kSTmp, s);
            if ((rc = sync_scalars("cg true residual"))) break;
            true_rel = hsc[kSBB] > 0 ? std::sqrt(hsc[kSTmp] / hsc[kSBB]) : 0.0;
            iters = (int)hsc[kSIters];   // iterations that updated y (no-ops after a freeze excluded)
            it = iters;                  // the next cycle numbers its iterations after the real ones
            if (true_rel <= o.tol || restarts >= 16 || it >= o.max_iter) {
                converged = true_rel <= o.tol;
                break;
            }
            converged = false;
            if (pc) {
                apply_prec(r, zv);
                cudaMemcpyAsync(pv, zv, 8ull * N, cudaMemcpyDeviceToDevice, s);
                launch_dot(r, zv, N, dp, sc + kSRR, s);
                cg_restart(sc, 0, s);
                if (reo) basis_start();
            } else {
                cudaMemcpyAsync(pv, r, 8ull * N, cudaMemcpyDeviceToDevice, s);
                cg_restart(sc, 1, s);
                // Projecting the residual out of the stored span also removes the
                // part that the operator's rounding puts there, which the iterate
                // never sees; that gap between the recurrence and the true
                // residual is what a restart finds.  The restart solves for the
                // correction with a fresh basis (the old span is dropped), so the
                // gap left after it scales with the small correction, not with y.
                // Measured against plain CG after the restart: 539 instead of 688
                // iterations at 210 x 210 x 75 x 178,797, 230 instead of 241 on
                // the noisy 80 x 80 x 40 slab, equal where no restart happens.
                if (reo) basis_start();
            }
        }
        if (rc) break;
        }  // single CG solve
        // m = m_ref + W^-2 G^T y: q already holds W^-2 G^T y of the final y (the
        // true residual's adjoint, the last product of either branch), so the
        // recovery is one vector add (the adjoint's own add of m_ref is the same
        // last operation: the result is bitwise that of another adjoint)
        if (m_ref) vec_axpby(1.0, m_ref, 1.0, q, M, m_out, s);
        else cudaMemcpyAsync(m_out, q, 8ull * M, cudaMemcpyDeviceToDevice, s);
        if (y_out) cudaMemcpyAsync(y_out, y, 8ull * N, cudaMemcpyDeviceToDevice, s);
        if ((rc = sync_scalars("cg finish"))) break;
        double fp64_rel = -1.0;
        if (o.check_stations > 0 && o.precision != GRAV_FP64) {
            // the predicted data of the recovered model, mixed against FP64
            if ((rc = plan_forward_ex(p, m_out, Ap, nullptr, 0.0, s))) break;
            if ((rc = check_fp64(p, m_out, Ap, (int)std::min<int64_t>(o.check_stations, N), nullptr, &fp64_rel, s)))
                break;
        }
        if (info) {
            info->iters = iters;
            info->converged = converged ? 1 : 0;
            info->rel_res = o.outer_max > 0 ? true_rel
                                            : (hsc[kSBB] > 0 ? std::sqrt(hsc[o.precond == 1 ? kSResNew : kSRR] / hsc[kSBB]) : 0.0);
            info->outer = outer_done;
            info->alpha_min = alpha_min;
            info->restarts = restarts;
            info->fp64_rel_err = fp64_rel;
            info->true_rel_res = true_rel;
            info->lambda = lam;
            info->trace = trace;
            info->nys_shift = (o.precond == 2 && ns.mu > 0) ? ns.nu / ns.mu : 0.0;
            info->nys_setup_s = nys_setup_s;
        }
        rc = read_status(ctx, s, o.timeout_s);
    } while (false);
    if (p->keep_nys && ns.mem && rc != GRAV_EDEVICE && rc != GRAV_ETIMEDOUT) {
        p->nys_kept = new NysState(ns);   // stays with the plan (freed by plan_destroy)
        ns = NysState{};
    }
    nys_free(p, &ns, s);
    cudaFreeAsync(base, s);
    ctx->hbm_used -= bytes;
    cudaEventDestroy(ev);
    cudaEventDestroy(evp[0]);
    cudaEventDestroy(evp[1]);
    if (rc != GRAV_ETIMEDOUT) cudaStreamSynchronize(s);
    cudaFreeHost(hsc);
    if (info) info->seconds = now_s() - t0;
    if (rc) return rc;
    if (!converged)
        return set_error(ctx, GRAV_ENOTCONVERGED, "CG reached max_iter=%d without reaching tol=%g", o.max_iter, o.tol);
    return GRAV_OK;
}

// FP64 data-space inversion by mixed-precision iterative refinement (the
// refine option; no counterpart in the paper).  The system solved is the FP64
// one, A y = dd with A = G W^-2 G^T + lambda I from the FP64 operator and
// lambda from its trace; each correction step solves the GRAV_MIXED system
// for the current FP64 residual by CG and adds that solution to y, and the
// residual is then recomputed with the FP64 operator, so the stopping test
// ||dd - A y|| <= tol ||dd|| is the FP64 one.  A step reduces the FP64
// residual to about its inner tolerance plus the mixed operator's deviation
// from the FP64 one: measured, the first step (tol 1e-6) leaves an FP64
// residual of 0.9e-6 to 1.7e-6 and one more step with inner tolerance 1e-2
// brings it to ~1e-8, on 4,000 / 256,000 / 1.35M cells.  Costs per step: one
// mixed CG solve and one FP64 operator pair (G^T then G), against one FP64
// pair per CG iteration without it.
int solve_refined(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const double *d,
                  const double *m_ref, double *m_out, double *y_out, grav_solve_info *info, const grav_options &o,
                  cudaStream_t s) {
    NvtxRange nv("grav::solve_refined");
    const double t0 = now_s();
    int rc = check_options(ctx, o);
    if (rc) return rc;
    grav_options o64 = o, om = o;
    o64.refine = 0;
    o64.precond = 0;
    om.refine = 0;
    om.precision = GRAV_MIXED;
    om.check_stations = 0;
    om.cache_g = 0;
    grav_plan *p64 = nullptr, *pm = nullptr;
    if ((rc = plan_create(ctx, mesh, survey, o64, &p64, s))) return rc;
    if ((rc = plan_create(ctx, mesh, survey, om, &pm, s))) {
        plan_destroy(p64, s);
        return rc;
    }
    pm->keep_nys = 1;   // a Nystrom preconditioner built by the first step serves the later ones
    const int64_t N = p64->N, M = p64->M;
    const size_t bytes = 8ull * (5 * N + 2 * M + kDotBlocks + kSCount) + 10 * 256;
    char *base = nullptr;
    double *hsc = nullptr;
    cudaEvent_t ev = nullptr;
    if (ctx->hbm_used.load() + bytes > ctx->hbm_budget) {
        rc = set_error(ctx, GRAV_ENOMEM, "refinement vectors exceed budget");
    } else {
        const cudaError_t e = cudaMallocFromPoolAsync((void **)&base, bytes, ctx->pool, s);
        if (e != cudaSuccess) rc = cuda_error(ctx, e, "refinement allocation");
        else ctx->hbm_used += bytes;
    }
    bool converged = false;
    double rel = 1.0, lam = o.lambda, trace = 0.0, nys_setup = 0.0, nys_shift = 0.0;
    int inner_iters = 0, steps = 0;
    do {
        if (rc) break;
        Arena ar;
        ar.base = base;
        ar.size = bytes;
        double *dd = (double *)ar.take(8ull * N), *y = (double *)ar.take(8ull * N), *r = (double *)ar.take(8ull * N);
        double *dl = (double *)ar.take(8ull * N), *Ay = (double *)ar.take(8ull * N);
        double *q = (double *)ar.take(8ull * M), *mscr = (double *)ar.take(8ull * M);
        double *dp = (double *)ar.take(8ull * kDotBlocks), *sc = (double *)ar.take(8ull * kSCount);
        cudaMallocHost((void **)&hsc, 8 * kSCount);
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        auto sync_scalars = [&](const char *what) -> int {
            cudaMemcpyAsync(hsc, sc, 8 * kSCount, cudaMemcpyDeviceToHost, s);
            cudaEventRecord(ev, s);
            return wait_event(ctx, ev, o.timeout_s, what);
        };
        // dd = d - G m_ref (FP64)
        if (m_ref) {
            if ((rc = plan_forward_ex(p64, m_ref, Ay, nullptr, 0.0, s))) break;
            vec_axpby(1.0, d, -1.0, Ay, N, dd, s);
        } else {
            cudaMemcpyAsync(dd, d, 8ull * N, cudaMemcpyDeviceToDevice, s);
        }
        cudaMemsetAsync(sc, 0, 8 * kSCount, s);
        launch_dot(dd, dd, N, dp, sc + kSBB, s);
        // lambda = lambda_scale * trace(G W^-2 G^T) / N with the FP64 diagonal
        if (!(lam > 0)) {
            if ((rc = plan_diag(p64, Ay, s))) break;
            launch_dot(Ay, nullptr, N, dp, sc + kSTrace, s);
        }
        if ((rc = sync_scalars("refinement start"))) break;
        const double bb = hsc[kSBB];
        if (!(lam > 0)) {
            trace = hsc[kSTrace];
            lam = o.lambda_scale * trace / (double)N;
            if (!(lam > 0) || !std::isfinite(lam)) {
                rc = set_error(ctx, GRAV_EDEVICE, "lambda from the trace is not positive (trace %g)", trace);
                break;
            }
        }
        vec_fill(y, N, 0.0, s);
        cudaMemcpyAsync(r, dd, 8ull * N, cudaMemcpyDeviceToDevice, s);
        if (!(bb > 0)) {   // zero data: y = 0 is the solution
            converged = true;
            rel = 0.0;
        }
        for (int k = 0; k < o.refine && !converged; ++k) {
            pm->opt = om;
            pm->opt.lambda = lam;
            // first step: half the requested tolerance (not below 2e-7, near the mixed
            // operator's rounding floor), so that its FP64 residual -- the inner one
            // plus the operators' difference, a few 1e-7 -- usually meets tol at once
            pm->opt.tol = (k == 0) ? std::max(0.5 * o.tol, std::min(o.tol, 2e-7)) : 1e-2;
            grav_solve_info ii{};
            const int rci = solve_on_plan(pm, r, nullptr, mscr, dl, &ii, s, nullptr, nullptr, nullptr, 0);
            if (rci != GRAV_OK && rci != GRAV_ENOTCONVERGED) {
                rc = rci;
                break;
            }
            inner_iters += ii.iters;
            nys_setup += ii.nys_setup_s;
            if (ii.nys_shift > 0) nys_shift = ii.nys_shift;
            vec_axpby(1.0, y, 1.0, dl, N, y, s);
            // r = dd - (G W^-2 G^T y + lambda y), FP64 operator
            if ((rc = plan_adjoint_ex(p64, y, q, 1, nullptr, s))) break;
            if ((rc = plan_forward_ex(p64, q, Ay, y, lam, s))) break;
            vec_axpby(1.0, dd, -1.0, Ay, N, r, s);
            launch_dot(r, r, N, dp, sc + kSTmp, s);
            if ((rc = sync_scalars("refinement residual"))) break;
            ++steps;
            rel = std::sqrt(std::max(hsc[kSTmp], 0.0) / bb);
            converged = rel <= o.tol;
        }
        if (rc) break;
        // m = m_ref + W^-2 G^T y: q holds the FP64 W^-2 G^T y of the final y
        // (the last residual's adjoint); y = 0 when no step ran
        if (steps == 0) vec_fill(q, M, 0.0, s);
        if (m_ref) vec_axpby(1.0, m_ref, 1.0, q, M, m_out, s);
        else cudaMemcpyAsync(m_out, q, 8ull * M, cudaMemcpyDeviceToDevice, s);
        if (y_out) cudaMemcpyAsync(y_out, y, 8ull * N, cudaMemcpyDeviceToDevice, s);
        rc = read_status(ctx, s, o.timeout_s);
    } while (false);
    if (base) {
        cudaFreeAsync(base, s);
        ctx->hbm_used -= bytes;
    }
    if (ev) cudaEventDestroy(ev);
    if (rc != GRAV_ETIMEDOUT) cudaStreamSynchronize(s);
    if (hsc) cudaFreeHost(hsc);
    plan_destroy(pm, s);
    plan_destroy(p64, s);
    if (info) {
        info->iters = inner_iters;
        info->converged = converged ? 1 : 0;
        info->rel_res = rel;
        info->true_rel_res = rel;
        info->lambda = lam;
        info->trace = trace;
        info->outer = steps;
        info->alpha_min = 1.0;
        info->restarts = 0;
        info->fp64_rel_err = -1.0;
        info->nys_shift = nys_shift;
        info->nys_setup_s = nys_setup;
        info->seconds = now_s() - t0;
    }
    if (rc) return rc;
    if (!converged)
        return set_error(ctx, GRAV_ENOTCONVERGED, "iterative refinement reached %d steps at FP64 residual %g (tol %g)",
                         o.refine, rel, o.tol);
    return GRAV_OK;
}

}  // namespace grav

using namespace grav;

// ---------------------------------------------------------------------------
// exported C ABI
// ---------------------------------------------------------------------------
extern "C" {

void grav_options_default(grav_options *o) {
    if (!o) return;
    o->precision = GRAV_FP64;
    o->z0 = 50.0;
    o->lambda_scale = 1e-2;
    o->lambda = 0.0;
    o->tol = 1e-6;
    o->max_iter = 1000;
    o->check_every = 0;
    o->near_cells = 8.0;
    o->timeout_s = 3600.0;
    o->precond = 0;
    o->cache_g = 0;
    o->outer_max = 0;
    o->inner_max = 20;
    o->reorth = 1000;
    o->check_stations = 0;
    o->nys_rank = 0;
    o->nys_coarsen = 0;
    o->refine = 0;
    o->near_fp64 = 0;
    o->diag_fp64 = 0;
}

const char *grav_version(void) { return "libgrav 0.1.0 (sm_103a)"; }

int grav_ctx_create(grav_ctx **out, int device, size_t hbm_budget) {
    if (!out) return set_error(nullptr, GRAV_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return set_error(nullptr, GRAV_EINVAL, "device %d out of range [0, %d)", device, n);
    DeviceGuard g(device);
    grav_ctx *ctx = new grav_ctx();
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        delete ctx;
        return cuda_error(nullptr, e, "cudaMemGetInfo");
    }
    ctx->hbm_budget = hbm_budget ? hbm_budget : (size_t)(0.9 * (double)fr);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&ctx->pool, &props);
    if (e != cudaSuccess) {
        delete ctx;
        return cuda_error(nullptr, e, "cudaMemPoolCreate");
    }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    std::vector<double> fn(fn_table_size());
    fill_fn_table(fn.data());
    if ((e = cudaMalloc((void **)&ctx->d_status, 256)) != cudaSuccess ||
        (e = cudaMemset(ctx->d_status, 0, 256)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&ctx->h_status, 256)) != cudaSuccess ||
        (e = cudaMalloc((void **)&ctx->d_fn, 8 * fn.size())) != cudaSuccess ||
        (e = cudaMemcpy(ctx->d_fn, fn.data(), 8 * fn.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
        if (ctx->d_status) cudaFree(ctx->d_status);
        if (ctx->h_status) cudaFreeHost(ctx->h_status);
        if (ctx->d_fn) cudaFree(ctx->d_fn);
        cudaMemPoolDestroy(ctx->pool);
        delete ctx;
        return cuda_error(nullptr, e, "context allocation");
    }
    *out = ctx;
    return GRAV_OK;
}

int grav_ctx_destroy(grav_ctx *ctx) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    serve_shutdown(ctx);
    cudaDeviceSynchronize();
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    cudaFree(ctx->d_fn);
    cudaMemPoolDestroy(ctx->pool);
    delete ctx;
    return GRAV_OK;
}

const char *grav_last_error(grav_ctx *ctx) {
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        thread_local std::string copy;
        copy = ctx->last_error;
        return copy.c_str();
    }
    std::lock_guard<std::mutex> lk(g_err_mu);
    thread_local std::string copy2;
    copy2 = g_last_error;
    return copy2.c_str();
}

int grav_ctx_sync(grav_ctx *ctx, grav_stream_t stream, double timeout_s) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    if (!(timeout_s > 0)) return set_error(ctx, GRAV_EINVAL, "timeout_s must be > 0");
    DeviceGuard g(ctx->device);
    return read_status(ctx, (cudaStream_t)stream, timeout_s);
}

int grav_plan_create(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const grav_options *opt,
                     grav_plan **out, grav_stream_t stream) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    return plan_create(ctx, mesh, survey, resolve(opt), out, (cudaStream_t)stream);
}

int grav_plan_forward(grav_plan *p, const double *m, double *d, grav_stream_t stream) {
    if (!p) return set_error(nullptr, GRAV_EINVAL, "plan is NULL");
    DeviceGuard g(p->ctx->device);
    if (!is_device_ptr(m, p->ctx->device) || !is_device_ptr(d, p->ctx->device))
        return set_error(p->ctx, GRAV_EINVAL, "m and d must be device pointers");
    return plan_forward_ex(p, m, d, nullptr, 0.0, (cudaStream_t)stream);
}

int grav_plan_adjoint(grav_plan *p, const double *r, double *gtr, int depth_weighted, grav_stream_t stream) {
    if (!p) return set_error(nullptr, GRAV_EINVAL, "plan is NULL");
    DeviceGuard g(p->ctx->device);
    if (!is_device_ptr(r, p->ctx->device) || !is_device_ptr(gtr, p->ctx->device))
        return set_error(p->ctx, GRAV_EINVAL, "r and gtr must be device pointers");
    return plan_adjoint_ex(p, r, gtr, depth_weighted, nullptr, (cudaStream_t)stream);
}

size_t grav_plan_bytes(const grav_plan *p) { return p ? p->bytes : 0; }

uint64_t grav_launch_count(void) { return g_launches.load(); }

int grav_plan_describe(const grav_plan *p, char *buf, size_t len) {
    if (!p) return set_error(nullptr, GRAV_EINVAL, "plan is NULL");
    char tmp[1024];
    int n;
    if (p->opt.precision == GRAV_FP64) {
        n = snprintf(tmp, sizeof(tmp),
                     "{\"precision\": \"fp64\", \"fwd_kernel\": \"%s\", \"adj_kernel\": \"%s\", "
                     "\"stored_g\": %s, \"fwd_row_chunks\": %d, \"adj_station_chunks\": %d, \"bytes\": %zu}",
                     p->cached ? "k_gemv_cached" : "k_fwd64<2>", p->cached ? "k_gemvt_cached" : "k_adj64<8>",
                     p->cached ? "true" : "false", p->f64_nchunk, p->a64_nschunk, p->bytes);
    } else {
        char adj[64];
        // template arguments as the compiled kernels carry them (the last one:
        // quadrupole far field for non-cubic prisms)
        const int quad = p->cubic ? 0 : 1;
        char fwd[64];
        snprintf(fwd, sizeof(fwd), "k_mfwd<8, %d, %d>", quad, mixed_fwd_tail(p));
        if (p->m_adj_bc)
            snprintf(adj, sizeof(adj), "k_madj_bc<%d, %d, %d>", p->m_adj_tz, mixed_adj_last_group(p), quad);
        else
            snprintf(adj, sizeof(adj), "k_madj<%d, %d>", p->m_adj_tz, quad);
        const bool corner = p->opt.precision == GRAV_MIXED_CORNER;
        n = snprintf(tmp, sizeof(tmp),
                     "{\"precision\": \"%s\", \"fwd_kernel\": \"%s\", \"adj_kernel\": \"%s\", "
                     "\"adj_layout\": \"%s\", \"fwd_column_chunks\": %d, \"adj_station_chunks\": %d, "
                     "\"near_cells\": %g, \"near_box\": [%d, %d, %d], \"bytes\": %zu}",
                     corner ? "mixed_corner" : "mixed", corner ? "k_cfwd32<4>" : fwd, corner ? "none" : adj,
                     p->m_adj_bc ? "broadcast" : "shuffle", corner ? p->cr_nchunk : p->m_fwd_nchunk, p->m_adj_nschunk,
                     p->opt.near_cells, p->ng.bx, p->ng.by, p->ng.bz, p->bytes);
    }
    if (n < 0) return set_error(p->ctx, GRAV_EDEVICE, "describe failed");
    if (buf && len > 0) {
        std::strncpy(buf, tmp, len - 1);
        buf[len - 1] = 0;
    }
    return n + 1;
}

int grav_plan_timing(grav_plan *p, int enable, double *ms, int64_t *counts) {
    if (!p) return set_error(nullptr, GRAV_EINVAL, "plan is NULL");
    DeviceGuard g(p->ctx->device);
    StageTimer &t = p->timer;
    if (ms || counts) {
        for (int k = 0; k < t.used; ++k) {
            cudaEventSynchronize(t.pool[2 * k + 1]);
            float e = 0.f;
            cudaEventElapsedTime(&e, t.pool[2 * k], t.pool[2 * k + 1]);
            t.ms[t.stage_of[k]] += e;
            t.count[t.stage_of[k]] += 1;
        }
        t.used = 0;
        for (int k = 0; k < kStageCount; ++k) {
            if (ms) ms[k] = t.ms[k];
            if (counts) counts[k] = t.count[k];
            t.ms[k] = 0.0;
            t.count[k] = 0;
        }
    }
    t.enabled = enable != 0;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRAV_OK : cuda_error(p->ctx, e, "stage timing");
}

int grav_plan_check_fp64(grav_plan *p, const double *m, const double *d, int n_check, double *max_abs_err,
                         double *rel_err, grav_stream_t stream) {
    if (!p) return set_error(nullptr, GRAV_EINVAL, "plan is NULL");
    DeviceGuard g(p->ctx->device);
    if (!is_device_ptr(m, p->ctx->device) || !is_device_ptr(d, p->ctx->device))
        return set_error(p->ctx, GRAV_EINVAL, "m and d must be device pointers");
    return check_fp64(p, m, d, n_check, max_abs_err, rel_err, (cudaStream_t)stream);
}

int grav_plan_destroy(grav_plan *p, grav_stream_t stream) {
    if (!p) return set_error(nullptr, GRAV_EINVAL, "plan is NULL");
    DeviceGuard g(p->ctx->device);
    plan_destroy(p, (cudaStream_t)stream);
    return GRAV_OK;
}

int grav_forward(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const double *m, double *d,
                 const grav_options *opt, grav_stream_t stream) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    int e0 = empty_survey(ctx, mesh, survey, opt);
    if (e0 < 0) return e0;
    if (e0) return GRAV_OK;   // no stations: nothing to write
    if (!is_device_ptr(m, ctx->device) || !is_device_ptr(d, ctx->device))
        return set_error(ctx, GRAV_EINVAL, "m and d must be device pointers on device %d", ctx->device);
    grav_plan *p = nullptr;
    int rc = plan_create(ctx, mesh, survey, resolve(opt), &p, (cudaStream_t)stream);
    if (rc) return rc;
    rc = plan_forward_ex(p, m, d, nullptr, 0.0, (cudaStream_t)stream);
    plan_destroy(p, (cudaStream_t)stream);
    return rc;
}

int grav_adjoint(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const double *r, double *gtr,
                 int depth_weighted, const grav_options *opt, grav_stream_t stream) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    int e0 = empty_survey(ctx, mesh, survey, opt);
    if (e0 < 0) return e0;
    if (e0) {   // no stations: G^T r = 0
        if (!is_device_ptr(gtr, ctx->device)) return set_error(ctx, GRAV_EINVAL, "gtr must be a device pointer");
        const cudaError_t e = cudaMemsetAsync(gtr, 0, 8ull * mesh->nx * mesh->ny * mesh->nz, (cudaStream_t)stream);
        return e == cudaSuccess ? GRAV_OK : cuda_error(ctx, e, "adjoint of an empty survey");
    }
    if (!is_device_ptr(r, ctx->device) || !is_device_ptr(gtr, ctx->device))
        return set_error(ctx, GRAV_EINVAL, "r and gtr must be device pointers on device %d", ctx->device);
    grav_plan *p = nullptr;
    int rc = plan_create(ctx, mesh, survey, resolve(opt), &p, (cudaStream_t)stream);
    if (rc) return rc;
    rc = plan_adjoint_ex(p, r, gtr, depth_weighted, nullptr, (cudaStream_t)stream);
    plan_destroy(p, (cudaStream_t)stream);
    return rc;
}

int grav_diag(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, double *diag, double *trace,
              const grav_options *opt, grav_stream_t stream) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    int e0 = empty_survey(ctx, mesh, survey, opt);
    if (e0 < 0) return e0;
    if (e0) {   // no stations: an empty diagonal, trace 0
        if (trace) *trace = 0.0;
        return GRAV_OK;
    }
    if (!is_device_ptr(diag, ctx->device)) return set_error(ctx, GRAV_EINVAL, "diag must be a device pointer");
    const grav_options o = resolve(opt);
    grav_plan *p = nullptr;
    const cudaStream_t s = (cudaStream_t)stream;
    int rc = plan_create(ctx, mesh, survey, o, &p, s);
    if (rc) return rc;
    rc = plan_diag(p, diag, s);
    if (!rc && trace) {
        double *buf = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync((void **)&buf, 8ull * (kDotBlocks + 1), ctx->pool, s);
        if (e != cudaSuccess) {
            rc = cuda_error(ctx, e, "trace scratch");
        } else {
            launch_dot(diag, nullptr, p->N, buf, buf + kDotBlocks, s);
            double *h = nullptr;
            cudaMallocHost((void **)&h, 8);
            cudaMemcpyAsync(h, buf + kDotBlocks, 8, cudaMemcpyDeviceToHost, s);
            cudaFreeAsync(buf, s);
            rc = read_status(ctx, s, o.timeout_s);
            if (!rc) *trace = *h;
            cudaFreeHost(h);
        }
    }
    plan_destroy(p, s);
    return rc;
}

int grav_nystrom_coarse_apply(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, int coarsen,
                              const double *X, int k, double *Y, const grav_options *opt,
                              grav_stream_t stream) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    if (k < 1 || coarsen < 1 || coarsen > 8) return set_error(ctx, GRAV_EINVAL, "need k >= 1 and coarsen in [1, 8]");
    if (!is_device_ptr(X, ctx->device) || !is_device_ptr(Y, ctx->device))
        return set_error(ctx, GRAV_EINVAL, "X and Y must be device pointers");
    const grav_options o = resolve(opt);
    grav_plan *p = nullptr;
    int rc = plan_prepare(ctx, mesh, survey, o, &p);   // geometry only: no device allocation
    if (rc) return rc;
    const cudaStream_t s = (cudaStream_t)stream;
    rc = nys_coarse_apply(p, coarsen, X, k, Y, s);
    if (!rc) rc = read_status(ctx, s, o.timeout_s);
    delete p;
    return rc;
}

int grav_dense_check(grav_ctx *ctx, int op, int M, int N, int K, const float *A, int64_t lda, const float *B,
                     int64_t ldb, void *C, int64_t ldc, int accumulate, grav_stream_t stream) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    if (op < 0 || op > 6 || M < 0 || N < 0 || K < 0) return set_error(ctx, GRAV_EINVAL, "bad op or size");
    const cudaStream_t s = (cudaStream_t)stream;
    if (op == 6) {   // FP64 Cholesky and triangular inverse of the Nystrom factorisation
        if (!is_device_ptr(A, ctx->device) || !is_device_ptr(C, ctx->device))
            return set_error(ctx, GRAV_EINVAL, "A and C must be device pointers");
        if (N == 0) return GRAV_OK;
        double *L = (double *)C, *Li = L + (size_t)N * N;
        int *fail = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync((void **)&fail, sizeof(int), ctx->pool, s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "dense check scratch");
        cudaMemcpyAsync(L, A, 8ull * N * N, cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(fail, 0, sizeof(int), s);
        launch_potrf_lower(L, N, fail, s);
        launch_trinv_lower(L, Li, N, s);
        int hf = 0;
        cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaFreeAsync(fail, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_error(ctx, e, "dense check factorisation");
        return hf ? set_error(ctx, GRAV_EDEVICE, "matrix is not positive definite") : GRAV_OK;
    }
    const bool gram = op == 2 || op == 5;
    if (!is_device_ptr(A, ctx->device) || !is_device_ptr(C, ctx->device) || (!gram && !is_device_ptr(B, ctx->device)))
        return set_error(ctx, GRAV_EINVAL, "A, B and C must be device pointers");
    int rc = gram ? launch_gram_df(N, K, A, lda, (double *)C, accumulate != 0, s, op == 5)
                  : launch_sgemm(op == 0, M, N, K, A, lda, B, ldb, (float *)C, ldc, accumulate != 0, s,
                                 op == 3 || op == 4, op == 3);
    if (rc) return set_error(ctx, GRAV_EINVAL, "unsupported layout (leading dimensions, K, M multiples of 4, "
                                               "16-byte aligned pointers)");
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRAV_OK : cuda_error(ctx, e, "dense kernel launch");
}

int grav_datainv_solve(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const double *d,
                       const double *m_ref, double *m_out, double *y_out, grav_solve_info *info,
                       const grav_options *opt, grav_stream_t stream) {
    return grav_datainv_solve_ex(ctx, mesh, survey, d, m_ref, m_out, y_out, info, opt, stream, nullptr, nullptr, 0);
}

int grav_datainv_solve_ex(grav_ctx *ctx, const grav_mesh *mesh, const grav_survey *survey, const double *d,
                          const double *m_ref, double *m_out, double *y_out, grav_solve_info *info,
                          const grav_options *opt, grav_stream_t stream, const double *y0, double *res_hist,
                          int res_hist_len) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    DeviceGuard g(ctx->device);
    int e0 = empty_survey(ctx, mesh, survey, opt);
    if (e0 < 0) return e0;
    if (e0) {   // no data: the minimiser of Eq. 7 is m_ref (0 when not given)
        if (!is_device_ptr(m_out, ctx->device) || (m_ref && !is_device_ptr(m_ref, ctx->device)))
            return set_error(ctx, GRAV_EINVAL, "m_out (and m_ref when given) must be device pointers");
        if (info) {
            std::memset(info, 0, sizeof(*info));
            info->converged = 1;
            info->alpha_min = 1.0;
        }
        const size_t bytes = 8ull * mesh->nx * mesh->ny * mesh->nz;
        const cudaError_t e = m_ref ? cudaMemcpyAsync(m_out, m_ref, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream)
                                    : cudaMemsetAsync(m_out, 0, bytes, (cudaStream_t)stream);
        return e == cudaSuccess ? GRAV_OK : cuda_error(ctx, e, "inversion of an empty survey");
    }
    if (!is_device_ptr(d, ctx->device) || !is_device_ptr(m_out, ctx->device) ||
        (m_ref && !is_device_ptr(m_ref, ctx->device)) || (y_out && !is_device_ptr(y_out, ctx->device)) ||
        (y0 && !is_device_ptr(y0, ctx->device)) || (res_hist && !is_device_ptr(res_hist, ctx->device)))
        return set_error(ctx, GRAV_EINVAL,
                         "d, m_out (and m_ref, y_out, y0, res_hist when given) must be device pointers");
    if (res_hist_len < 0 || (res_hist && res_hist_len == 0))
        return set_error(ctx, GRAV_EINVAL, "res_hist_len must be >= 1 when res_hist is given");
    if (info) std::memset(info, 0, sizeof(*info));
    const cudaStream_t s = (cudaStream_t)stream;
    const grav_options ro = resolve(opt);
    if (ro.refine > 0) {
        if (y0 || res_hist)
            return set_error(ctx, GRAV_EINVAL, "refine does not take y0 or res_hist");
        return solve_refined(ctx, mesh, survey, d, m_ref, m_out, y_out, info, ro, s);
    }
    grav_plan *p = nullptr;
    int rc = plan_create(ctx, mesh, survey, ro, &p, s);
    if (rc) return rc;
    rc = solve_on_plan(p, d, m_ref, m_out, y_out, info, s, nullptr, y0, res_hist, res_hist ? res_hist_len : 0);
    plan_destroy(p, s);
    return rc;
}

}  // extern "C"
