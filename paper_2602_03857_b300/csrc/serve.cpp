// Serving scheduler: continuous admission of forward and inversion jobs.
//
// Jobs enter a FIFO queue (grav_submit never touches the GPU).  K slots, each
// a worker thread with its own non-blocking CUDA stream, take the head job as
// soon as they are free AND the job's device footprint (its plan plus, for an
// inversion, the CG vectors) fits next to the jobs already running — so jobs
// that arrive while others are on the GPU start as soon as a slot and memory
// free up, and their kernels overlap on the device.  Every job builds its own
// plan, so its result is the same whether it runs alone or in the mix (the
// kernels are deterministic).  Inversions check a cancel flag between CG
// iteration chunks.
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
    std::atomic<int> cancel{0};
};

struct Scheduler {
    grav_ctx *ctx = nullptr;
    int slots = 4;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_id = 1;
    size_t bytes_active = 0;
    bool started = false, stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
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

bool head_admissible(Scheduler *s) {
    if (s->queue.empty()) return false;
    return s->bytes_active + s->queue.front()->est_bytes <= s->ctx->hbm_budget || s->bytes_active == 0;
}

void run_job(Scheduler *s, Job *job, cudaStream_t stream) {
    NvtxRange nv(job->desc.kind == GRAV_JOB_FORWARD ? "grav::job_forward" : "grav::job_invert");
    grav_ctx *ctx = s->ctx;
    const grav_job &d = job->desc;
    grav_mesh mesh = d.mesh;
    mesh.xe = job->xe.data();
    mesh.ye = job->ye.data();
    mesh.ze = job->ze.data();
    grav_plan *p = nullptr;
    int rc = plan_create(ctx, &mesh, &d.survey, d.opt, &p, stream);
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
        plan_destroy(p, stream);
        const int rc2 = read_status(ctx, stream, d.opt.timeout_s);
        if (rc == GRAV_OK) rc = rc2;
    }
    job->result = rc;
    if (rc != GRAV_OK) job->error = grav_last_error(ctx);
}

void worker(Scheduler *s, int slot) {
    cudaSetDevice(s->ctx->device);
    cudaStream_t stream = s->streams[slot];
    while (true) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || head_admissible(s); });
            if (s->stop) return;
            job = s->queue.front();
            s->queue.pop_front();
            s->bytes_active += job->est_bytes;
            job->state = GRAV_JOB_RUNNING;
            job->t_start = now_s();
        }
        run_job(s, job.get(), stream);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->bytes_active -= job->est_bytes;
            job->t_end = now_s();
            if (job->result == GRAV_ECANCELED) job->state = GRAV_JOB_CANCELED;
            else if (job->result == GRAV_OK || job->result == GRAV_ENOTCONVERGED) job->state = GRAV_JOB_DONE;
            else job->state = GRAV_JOB_FAILED;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

void start_workers(Scheduler *s) {
    s->streams.resize(s->slots);
    for (int k = 0; k < s->slots; ++k) cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
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
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
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

int grav_submit(grav_ctx *ctx, const grav_job *job, uint64_t *job_id) {
    if (!ctx || !job || !job_id) return set_error(ctx, GRAV_EINVAL, "ctx, job and job_id must not be NULL");
    if (job->kind != GRAV_JOB_FORWARD && job->kind != GRAV_JOB_INVERT)
        return set_error(ctx, GRAV_EINVAL, "job kind must be GRAV_JOB_FORWARD or GRAV_JOB_INVERT");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    grav_plan *p = nullptr;
    int rc = plan_prepare(ctx, &job->mesh, &job->survey, job->opt, &p);
    if (rc == GRAV_OK) {
        const bool ok = is_device(job->input, ctx->device) && is_device(job->output, ctx->device) &&
                        (!job->m_ref || is_device(job->m_ref, ctx->device));
        if (!ok) rc = set_error(ctx, GRAV_EINVAL, "job input/output (and m_ref) must be device pointers");
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
