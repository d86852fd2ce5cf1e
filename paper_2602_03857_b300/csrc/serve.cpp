// Serving scheduler: continuous admission of forward and inversion jobs.
//
// Jobs enter a queue (grav_submit never touches the GPU).  K slots, each a
// worker thread with its own non-blocking CUDA stream, take a queued job as
// soon as they are free AND the job's device footprint (its plan plus, for an
// inversion, the CG vectors) fits next to the jobs already running -- so jobs
// that arrive while others are on the GPU start as soon as a slot and memory
// free up, and their kernels overlap on the device.  Admission is FIFO with
// backfill: when the oldest job does not fit, the first later job that does
// may start instead, at most kMaxBypass times before the oldest job is served
// first (no starvation).
//
// Plans stay resident: a finished job leaves its plan (mesh tables, station
// arrays, near-field table, the trace of G W^-2 G^T) in a cache, and a later
// job on the same mesh, the same survey arrays with unchanged contents and the
// same plan-shaping options takes it instead of building one.  Idle cached
// plans count against the context's HBM budget and are evicted, least
// recently used first, when an admission needs the memory.  A reused plan
// runs the same deterministic kernels on the same tables, so a job's result
// is bitwise the same alone, in a mix, and with a fresh or a resident plan.
// Inversions check a cancel flag between CG iteration chunks.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>

#include "internal.h"

namespace grav {

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr int kMaxBypass = 8;   // later jobs that may start ahead of a waiting oldest job

struct Job {
    uint64_t id = 0;
    grav_job desc{};
    std::vector<double> xe, ye, ze;   // host copies of the mesh edges
    int state = GRAV_JOB_QUEUED;
    int result = GRAV_OK;
    std::string error;
    grav_solve_info info{};
    double t_submit = 0, t_start = 0, t_end = 0;
    size_t est_bytes = 0;
    int bypassed = 0;                 // times a later job started while this one was the oldest
    int plan_reused = 0;              // 1: ran on a resident plan
    double setup_s = 0;               // host wall time of plan creation (0 when reused)
    std::atomic<int> cancel{0};
};

// What a plan depends on: the mesh, the survey (arrays and their contents)
// and the options that shape it.
struct PlanKey {
    std::vector<double> xe, ye, ze;
    const double *sx = nullptr, *sy = nullptr, *sz = nullptr;
    int64_t n = 0;
    uint64_t survey_hash = 0;
    int precision = 0, cache_g = 0, near_fp64 = 0, diag_fp64 = 0;
    double z0 = 0, near_cells = 0;
    bool operator==(const PlanKey &o) const {
        return sx == o.sx && sy == o.sy && sz == o.sz && n == o.n && survey_hash == o.survey_hash &&
               precision == o.precision && cache_g == o.cache_g && z0 == o.z0 && near_cells == o.near_cells &&
               near_fp64 == o.near_fp64 && diag_fp64 == o.diag_fp64 &&
               xe == o.xe && ye == o.ye && ze == o.ze;
    }
};

struct CachedPlan {
    PlanKey key;
    grav_plan *plan = nullptr;
    size_t bytes = 0;                 // device bytes it holds (plan + resident preconditioner)
    double last_used = 0;
};

struct Scheduler {
    grav_ctx *ctx = nullptr;
    int slots = 4;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_id = 1;
    size_t bytes_active = 0;          // footprints reserved by running jobs
    size_t bytes_cached = 0;          // idle resident plans
    int max_cached = 16;              // 0: no plan cache
    std::vector<CachedPlan> cache;
    int64_t plans_built = 0, plans_reused = 0;
    bool started = false, stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::vector<unsigned long long *> d_hash, h_hash;   // per slot: survey-hash result (device, pinned host)
    std::vector<cudaEvent_t> ev_hash;
    size_t max_queue = 1 << 16;
};

Scheduler *sched_of(grav_ctx *ctx, bool create) {
    if (!ctx->serve && create) {
        Scheduler *s = new Scheduler();
        s->ctx = ctx;
        if (const char *env = std::getenv("GRAV_SERVE_SLOTS")) {
            const int k = std::atoi(env);
            if (k >= 1 && k <= 64) s->slots = k;
        }
        ctx->serve = s;
    }
    return static_cast<Scheduler *>(ctx->serve);
}

bool fits(const Scheduler *s, const Job &j) {
    return s->bytes_active + j.est_bytes <= s->ctx->hbm_budget || s->bytes_active == 0;
}

// FIFO with bounded backfill: the oldest job if it fits; else the first later
// job that fits, unless the oldest has already been passed kMaxBypass times.
// Returns the queue position, or -1.
int pick(Scheduler *s) {
    if (s->queue.empty()) return -1;
    if (fits(s, *s->queue.front())) return 0;
    if (s->queue.front()->bypassed >= kMaxBypass) return -1;
    for (size_t k = 1; k < s->queue.size(); ++k)
        if (fits(s, *s->queue[k])) return (int)k;
    return -1;
}

// Idle cached plans to release so that running jobs plus the cache stay
// within the budget and the cache within max_cached entries (least recently
// used first).  Called with the lock held; the caller destroys them outside.
void evict(Scheduler *s, std::vector<grav_plan *> &out) {
    while (!s->cache.empty() && (s->bytes_active + s->bytes_cached > s->ctx->hbm_budget ||
                                 (int)s->cache.size() > s->max_cached)) {
        size_t lru = 0;
        for (size_t k = 1; k < s->cache.size(); ++k)
            if (s->cache[k].last_used < s->cache[lru].last_used) lru = k;
        s->bytes_cached -= s->cache[lru].bytes;
        out.push_back(s->cache[lru].plan);
        s->cache.erase(s->cache.begin() + (long)lru);
    }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {   // SplitMix64 finaliser
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// XOR over stations of mixed (bit pattern, position) of x, y and z: a 64-bit
// fingerprint of the survey's contents, independent of summation order.
__global__ void k_survey_hash(const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ z, int64_t n, unsigned long long *out) {
    unsigned long long h = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = 3ull * (unsigned long long)i * 0x9e3779b97f4a7c15ull;
        h ^= mix64((unsigned long long)__double_as_longlong(x[i]) + k);
        h ^= mix64((unsigned long long)__double_as_longlong(y[i]) + k + 0x632be59bd9b4e019ull);
        h ^= mix64((unsigned long long)__double_as_longlong(z[i]) + k + 0x8cb92ba72f3d8dd7ull);
    }
    for (int o = 16; o > 0; o >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0 && h) atomicXor(out, h);
}

int survey_hash(Scheduler *s, int slot, const grav_survey &sv, double timeout_s, uint64_t *out) {
    cudaStream_t st = s->streams[slot];
    cudaMemsetAsync(s->d_hash[slot], 0, 8, st);
    const int blocks = (int)std::min<int64_t>((sv.n + 255) / 256, 148 * 4);
    k_survey_hash<<<std::max(blocks, 1), 256, 0, st>>>(sv.x, sv.y, sv.z, sv.n, s->d_hash[slot]);
    note_launches(1);
    cudaMemcpyAsync(s->h_hash[slot], s->d_hash[slot], 8, cudaMemcpyDeviceToHost, st);
    cudaEventRecord(s->ev_hash[slot], st);
    const int rc = host_wait(s->ctx, s->ev_hash[slot], timeout_s, "survey hash");
    if (rc == GRAV_OK) *out = *s->h_hash[slot];
    return rc;
}

void run_job(Scheduler *s, Job *job, int slot) {
    NvtxRange nv(job->desc.kind == GRAV_JOB_FORWARD ? "grav::job_forward" : "grav::job_invert");
    grav_ctx *ctx = s->ctx;
    cudaStream_t stream = s->streams[slot];
    const grav_job &d = job->desc;
    grav_mesh mesh = d.mesh;
    mesh.xe = job->xe.data();
    mesh.ye = job->ye.data();
    mesh.ze = job->ze.data();
    grav_plan *p = nullptr;
    int rc = GRAV_OK;
    PlanKey key;
    bool use_cache = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        use_cache = s->max_cached > 0;
    }
    if (use_cache) {
        key.xe = job->xe; key.ye = job->ye; key.ze = job->ze;
        key.sx = d.survey.x; key.sy = d.survey.y; key.sz = d.survey.z; key.n = d.survey.n;
        key.precision = d.opt.precision; key.cache_g = d.opt.cache_g;
        key.z0 = d.opt.z0; key.near_cells = d.opt.near_cells; key.near_fp64 = d.opt.near_fp64;
        key.diag_fp64 = d.opt.diag_fp64;
        rc = survey_hash(s, slot, d.survey, d.opt.timeout_s, &key.survey_hash);
        if (rc == GRAV_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t k = 0; k < s->cache.size(); ++k)
                if (s->cache[k].key == key) {
                    p = s->cache[k].plan;
                    s->bytes_cached -= s->cache[k].bytes;
                    s->cache.erase(s->cache.begin() + (long)k);
                    ++s->plans_reused;
                    break;
                }
        }
    }
    if (rc == GRAV_OK) {
        if (p) {
            p->opt = d.opt;   // same plan-shaping fields (the key); the solve's own options are this job's
            job->plan_reused = 1;
            if (use_cache) p->keep_nys = 1;
        } else {
            const double t0 = now_s();
            rc = plan_create(ctx, &mesh, &d.survey, d.opt, &p, stream);
            job->setup_s = now_s() - t0;
            if (rc == GRAV_OK) {
                if (use_cache) p->keep_nys = 1;   // a Nystrom preconditioner stays with the plan
                std::lock_guard<std::mutex> lk(s->mu);
                ++s->plans_built;
            }
        }
    }
    if (rc == GRAV_OK) {
        if (d.kind == GRAV_JOB_FORWARD) {
            rc = plan_forward_ex(p, d.input, d.output, nullptr, 0.0, stream);
            if (rc == GRAV_OK) rc = read_status(ctx, stream, d.opt.timeout_s);
            job->info.fp64_rel_err = -1.0;
            if (rc == GRAV_OK && d.opt.check_stations > 0 && d.opt.precision != GRAV_FP64)
                rc = check_fp64(p, d.input, d.output, (int)std::min<int64_t>(d.opt.check_stations, d.survey.n),
                                nullptr, &job->info.fp64_rel_err, stream);
        } else {
            rc = solve_on_plan(p, d.input, d.m_ref, d.output, nullptr, &job->info, stream, &job->cancel);
        }
        const int rc2 = read_status(ctx, stream, d.opt.timeout_s);
        if (rc == GRAV_OK) rc = rc2;
        // keep the plan resident when the job ran cleanly (its work has completed:
        // read_status synchronised the stream)
        const bool keep = use_cache && (rc == GRAV_OK || rc == GRAV_ENOTCONVERGED || rc == GRAV_ECANCELED);
        if (keep) {
            std::lock_guard<std::mutex> lk(s->mu);
            CachedPlan c;
            c.key = std::move(key);
            c.plan = p;
            c.bytes = plan_resident_bytes(p);
            c.last_used = now_s();
            s->bytes_cached += c.bytes;
            s->cache.push_back(std::move(c));
            p = nullptr;
        }
        if (p) plan_destroy(p, stream);
    }
    job->result = rc;
    if (rc != GRAV_OK) job->error = grav_last_error(ctx);
}

void destroy_plans(std::vector<grav_plan *> &v, cudaStream_t stream) {
    for (grav_plan *p : v) plan_destroy(p, stream);
    v.clear();
}

void worker(Scheduler *s, int slot) {
    cudaSetDevice(s->ctx->device);
    cudaStream_t stream = s->streams[slot];
    std::vector<grav_plan *> evicted;
    while (true) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            int k = -1;
            s->cv_work.wait(lk, [&] { return s->stop || (k = pick(s)) >= 0; });
            if (s->stop) return;
            job = s->queue[(size_t)k];
            if (k > 0) s->queue.front()->bypassed++;
            s->queue.erase(s->queue.begin() + k);
            s->bytes_active += job->est_bytes;
            evict(s, evicted);
            job->state = GRAV_JOB_RUNNING;
            job->t_start = now_s();
        }
        destroy_plans(evicted, stream);
        run_job(s, job.get(), slot);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->bytes_active -= job->est_bytes;
            evict(s, evicted);
            job->t_end = now_s();
            if (job->result == GRAV_ECANCELED) job->state = GRAV_JOB_CANCELED;
            else if (job->result == GRAV_OK || job->result == GRAV_ENOTCONVERGED) job->state = GRAV_JOB_DONE;
            else job->state = GRAV_JOB_FAILED;
        }
        destroy_plans(evicted, stream);
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

void start_workers(Scheduler *s) {
    s->streams.resize(s->slots);
    s->d_hash.assign(s->slots, nullptr);
    s->h_hash.assign(s->slots, nullptr);
    s->ev_hash.resize(s->slots);
    for (int k = 0; k < s->slots; ++k) {
        cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
        cudaMalloc((void **)&s->d_hash[k], 8);
        cudaMallocHost((void **)&s->h_hash[k], 8);
        cudaEventCreateWithFlags(&s->ev_hash[k], cudaEventDisableTiming);
    }
    for (int k = 0; k < s->slots; ++k) s->workers.emplace_back(worker, s, k);
    s->started = true;
}

bool is_device(const void *p, int device) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

}  // namespace

void serve_shutdown(grav_ctx *ctx) {
    Scheduler *s = sched_of(ctx, false);
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto &j : s->queue) {
            j->state = GRAV_JOB_CANCELED;
            j->result = GRAV_ECANCELED;
        }
        s->queue.clear();
        for (auto &kv : s->jobs)
            if (kv.second->state == GRAV_JOB_RUNNING) kv.second->cancel = 1;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto &t : s->workers)
        if (t.joinable()) t.join();
    if (!s->streams.empty()) {
        for (auto &c : s->cache) plan_destroy(c.plan, s->streams[0]);
        cudaStreamSynchronize(s->streams[0]);
    }
    s->cache.clear();
    for (size_t k = 0; k < s->streams.size(); ++k) {
        cudaStreamDestroy(s->streams[k]);
        cudaFree(s->d_hash[k]);
        cudaFreeHost(s->h_hash[k]);
        cudaEventDestroy(s->ev_hash[k]);
    }
    delete s;
    ctx->serve = nullptr;
}

}  // namespace grav

using namespace grav;

extern "C" {

int grav_serve_config(grav_ctx *ctx, int slots) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    if (slots < 1 || slots > 64) return set_error(ctx, GRAV_EINVAL, "slots must lie in [1, 64]");
    Scheduler *s = sched_of(ctx, true);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started) return set_error(ctx, GRAV_EBUSY, "the scheduler is already running");
    s->slots = slots;
    return GRAV_OK;
}

int grav_serve_plan_cache(grav_ctx *ctx, int max_plans) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    if (max_plans < 0 || max_plans > 1024) return set_error(ctx, GRAV_EINVAL, "max_plans must lie in [0, 1024]");
    Scheduler *s = sched_of(ctx, true);
    std::lock_guard<std::mutex> lk(s->mu);
    s->max_cached = max_plans;   // excess entries go at the next admission or job end
    return GRAV_OK;
}

int grav_serve_stats(grav_ctx *ctx, int64_t *plans_built, int64_t *plans_reused, int *plans_resident,
                     size_t *bytes_resident) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    Scheduler *s = sched_of(ctx, true);
    std::lock_guard<std::mutex> lk(s->mu);
    if (plans_built) *plans_built = s->plans_built;
    if (plans_reused) *plans_reused = s->plans_reused;
    if (plans_resident) *plans_resident = (int)s->cache.size();
    if (bytes_resident) *bytes_resident = s->bytes_cached;
    return GRAV_OK;
}

int grav_submit(grav_ctx *ctx, const grav_job *job, uint64_t *job_id) {
    if (!ctx || !job || !job_id) return set_error(ctx, GRAV_EINVAL, "ctx, job and job_id must not be NULL");
    if (job->kind != GRAV_JOB_FORWARD && job->kind != GRAV_JOB_INVERT)
        return set_error(ctx, GRAV_EINVAL, "job kind must be GRAV_JOB_FORWARD or GRAV_JOB_INVERT");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    grav_plan *p = nullptr;
    int rc = plan_prepare(ctx, &job->mesh, &job->survey, job->opt, &p);
    if (rc == GRAV_OK && job->opt.refine > 0)
        rc = set_error(ctx, GRAV_EINVAL, "refine is supported by grav_datainv_solve only, not by serving jobs");
    if (rc == GRAV_OK) {
        const bool ok = is_device(job->input, ctx->device) && is_device(job->output, ctx->device) &&
                        (!job->m_ref || is_device(job->m_ref, ctx->device));
        if (!ok) rc = set_error(ctx, GRAV_EINVAL, "job input/output (and m_ref) must be device pointers");
    }
    if (rc != GRAV_OK) {   // the prepared (host-only) plan of a rejected job
        delete p;
        p = nullptr;
    }
    size_t est = 0;
    if (rc == GRAV_OK) {
        est = p->bytes + (job->kind == GRAV_JOB_INVERT ? solve_bytes(p) : 0);
        if (job->kind == GRAV_JOB_INVERT && p->opt.precond == 2)   // Nystrom factors and set-up scratch
            est += nys_peak_bytes(p);
        if (job->opt.check_stations > 0 && job->opt.precision != GRAV_FP64) {
            // the FP64 check's transient plan: node weights, the adjoint's node-sized
            // scratch (two arrays plus station-chunk partials), station arrays and partials
            const size_t nodes = (size_t)(job->mesh.nx + 2) * (job->mesh.ny + 1) * (job->mesh.nz + 1);
            est += 32 * nodes + 256ull * (size_t)job->opt.check_stations + (1u << 20);
        }
        delete p;
        if (est > ctx->hbm_budget)
            rc = set_error(ctx, GRAV_ENOMEM, "job needs %.3f GB, more than the context budget %.3f GB", est / 1e9,
                           ctx->hbm_budget / 1e9);
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (rc) return rc;
    auto j = std::make_shared<Job>();
    j->desc = *job;
    j->xe.assign(job->mesh.xe, job->mesh.xe + job->mesh.nx + 1);
    j->ye.assign(job->mesh.ye, job->mesh.ye + job->mesh.ny + 1);
    j->ze.assign(job->mesh.ze, job->mesh.ze + job->mesh.nz + 1);
    j->est_bytes = est;
    j->t_submit = now_s();
    Scheduler *s = sched_of(ctx, true);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return set_error(ctx, GRAV_ECANCELED, "the scheduler is shutting down");
        if (s->queue.size() >= s->max_queue) return set_error(ctx, GRAV_EBUSY, "serving queue full");
        if (!s->started) start_workers(s);
        j->id = s->next_id++;
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        *job_id = j->id;
    }
    s->cv_work.notify_one();
    return GRAV_OK;
}

int grav_poll(grav_ctx *ctx, uint64_t job_id, int *state, grav_solve_info *info) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    Scheduler *s = sched_of(ctx, false);
    if (!s) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    if (state) *state = it->second->state;
    if (info) *info = it->second->info;
    return GRAV_OK;
}

int grav_wait(grav_ctx *ctx, uint64_t job_id, double timeout_s) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    if (!(timeout_s >= 0)) return set_error(ctx, GRAV_EINVAL, "timeout_s must be >= 0");
    Scheduler *s = sched_of(ctx, false);
    if (!s) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    std::shared_ptr<Job> j = it->second;
    const bool done = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        return j->state == GRAV_JOB_DONE || j->state == GRAV_JOB_FAILED || j->state == GRAV_JOB_CANCELED;
    });
    if (!done) return set_error(ctx, GRAV_ETIMEDOUT, "job %llu still %s after %.3f s", (unsigned long long)job_id,
                                j->state == GRAV_JOB_QUEUED ? "queued" : "running", timeout_s);
    if (j->result != GRAV_OK) set_error(ctx, j->result, "job %llu: %s", (unsigned long long)job_id, j->error.c_str());
    return j->result;
}

int grav_cancel(grav_ctx *ctx, uint64_t job_id) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    Scheduler *s = sched_of(ctx, false);
    if (!s) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
        Job *j = it->second.get();
        if (j->state == GRAV_JOB_QUEUED) {
            for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
                if ((*q)->id == job_id) {
                    s->queue.erase(q);
                    break;
                }
            j->state = GRAV_JOB_CANCELED;
            j->result = GRAV_ECANCELED;
            j->error = "cancelled while queued";
            j->t_end = now_s();
        } else if (j->state == GRAV_JOB_RUNNING) {
            j->cancel = 1;
        }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    return GRAV_OK;
}

int grav_job_times(grav_ctx *ctx, uint64_t job_id, double *t_submit, double *t_start, double *t_end) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    Scheduler *s = sched_of(ctx, false);
    if (!s) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    if (t_submit) *t_submit = it->second->t_submit;
    if (t_start) *t_start = it->second->t_start;
    if (t_end) *t_end = it->second->t_end;
    return GRAV_OK;
}

int grav_job_plan(grav_ctx *ctx, uint64_t job_id, int *plan_reused, double *setup_s, size_t *footprint) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    Scheduler *s = sched_of(ctx, false);
    if (!s) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    if (plan_reused) *plan_reused = it->second->plan_reused;
    if (setup_s) *setup_s = it->second->setup_s;
    if (footprint) *footprint = it->second->est_bytes;
    return GRAV_OK;
}

int grav_job_release(grav_ctx *ctx, uint64_t job_id) {
    if (!ctx) return set_error(nullptr, GRAV_EINVAL, "ctx is NULL");
    Scheduler *s = sched_of(ctx, false);
    if (!s) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(ctx, GRAV_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    const int st = it->second->state;
    if (st == GRAV_JOB_QUEUED || st == GRAV_JOB_RUNNING)
        return set_error(ctx, GRAV_EBUSY, "job %llu has not finished", (unsigned long long)job_id);
    s->jobs.erase(it);
    return GRAV_OK;
}

}  // extern "C"
