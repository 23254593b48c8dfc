// Request loop with continuous batching (lbks_server_* / lbks_submit /
// lbks_poll): solves of different grid sizes are admitted into worker slots
// as slots and device memory free up; each slot owns a CUDA stream, so the
// slots' relaxation, Poisson and reduction kernels overlap on the GPU.
// Systems are pooled by shape and kept resident between requests.
#include "lbks.h"
#include "lbks_internal.cuh"

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t id;
    lbks_request req;
    std::vector<double> xyz, Z;
    size_t bytes = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    int rc = LBKS_OK;
    std::string err;
    lbks_result res;
    Clock::time_point t_submit, t_start, t_end;
};

using ShapeKey = std::tuple<int, int, int, int, int, int, double, double, double, long long, int>;

}  // namespace

struct lbks_server {
    lbks_params defaults;
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;  // bytes reserved by running jobs and pooled systems
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job*> queue;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    std::multimap<ShapeKey, std::pair<lbks_system*, size_t>> pool;  // idle systems, bytes
    std::vector<std::thread> workers;
    uint64_t next_id = 1;
    bool stop = false;
    uint64_t completed = 0;
    int running = 0;
};

namespace {

ShapeKey key_of(const lbks_params& p, const lbks_request& r) {
    return ShapeKey(r.nx, r.ny, r.nz, r.n_orb, p.precision, p.n_inner, r.h, p.theta, p.omega,
                    (long long)(p.e_tol * 1e15), p.storage);
}

lbks_params params_of(const lbks_server* s, const lbks_request& r) {
    lbks_params p = s->defaults;
    if (r.precision >= 0) p.precision = r.precision;
    if (r.n_inner > 0) p.n_inner = r.n_inner;
    if (r.e_tol > 0) p.e_tol = r.e_tol;
    if (r.max_cycles > 0) p.max_cycles = r.max_cycles;
    return p;
}

// Frees pooled systems (oldest first) until `need` more bytes fit; lock held.
bool make_room(lbks_server* s, size_t need) {
    while (s->in_use + need > s->budget && !s->pool.empty()) {
        auto it = s->pool.begin();
        lbks_destroy_system(it->second.first);
        s->in_use -= it->second.second;
        s->pool.erase(it);
    }
    return s->in_use + need <= s->budget;
}

void worker_main(lbks_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Job* job = nullptr;
        lbks_system* sys = nullptr;
        lbks_params p;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stop) break;
                // first queued job whose system is pooled or fits in the free budget
                for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                    Job* j = *it;
                    p = params_of(s, j->req);
                    auto pit = s->pool.find(key_of(p, j->req));
                    if (pit != s->pool.end()) {
                        sys = pit->second.first;
                        s->pool.erase(pit);  // bytes stay reserved while running
                        job = j;
                    } else if (make_room(s, j->bytes)) {
                        s->in_use += j->bytes;
                        job = j;
                    }
                    if (job) {
                        s->queue.erase(it);
                        break;
                    }
                }
                if (job) break;
                s->cv_work.wait(lk);
            }
            if (!job) break;
            job->state = 1;
            job->t_start = Clock::now();
            ++s->running;
        }
        int rc = LBKS_OK;
        const lbks_request& r = job->req;
        if (!sys) rc = lbks_create_system(&p, r.nx, r.ny, r.nz, r.h, r.n_orb, &sys);
        if (rc == LBKS_OK) rc = lbks_set_geometry(sys, r.n_atoms, job->xyz.data(), job->Z.data());
        if (rc == LBKS_OK) rc = lbks_scf(sys, st, &job->res);
        if (rc != LBKS_OK) {
            char buf[512];
            lbks_last_error(buf, sizeof buf);
            job->err = buf;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            job->rc = rc;
            job->t_end = Clock::now();
            job->state = 2;
            --s->running;
            ++s->completed;
            if (sys && (rc == LBKS_OK || rc == LBKS_ENOTCONV))
                s->pool.emplace(key_of(p, r), std::make_pair(sys, job->bytes));
            else {
                if (sys) lbks_destroy_system(sys);
                s->in_use -= job->bytes;
            }
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

int lbks_server_create(const lbks_params* defaults, size_t budget_bytes, int max_slots, lbks_server** out) {
    if (!out) return lbks::set_last_error(LBKS_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64) return lbks::set_last_error(LBKS_EINVAL, "max_slots must be in [1, 64]");
    lbks_params p;
    if (defaults) p = *defaults;
    else lbks_params_default(&p);
    if (lbks_system_bytes(&p, 4, 4, 4, 1) == 0) return lbks::set_last_error(LBKS_EINVAL, "invalid lbks_params");
    auto* s = new lbks_server();
    s->defaults = p;
    cudaGetDevice(&s->device);
    if (budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) {
            delete s;
            return lbks::set_last_error(LBKS_ECUDA, cudaGetErrorString(e));
        }
        budget_bytes = (size_t)(0.85 * (double)free_b);
    }
    s->budget = budget_bytes;
    s->max_slots = max_slots;
    for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_main, s);
    *out = s;
    return LBKS_OK;
}

int lbks_server_destroy(lbks_server* s) {
    if (!s) return lbks::set_last_error(LBKS_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->pool) lbks_destroy_system(kv.second.first);
    delete s;
    return LBKS_OK;
}

int lbks_submit(lbks_server* s, const lbks_request* r, uint64_t* id) {
    if (!s || !r || !id) return lbks::set_last_error(LBKS_EINVAL, "null argument");
    if (r->n_atoms < 1 || !r->xyz || !r->Z) return lbks::set_last_error(LBKS_EINVAL, "request has no atoms");
    lbks_params p = params_of(s, *r);
    const size_t bytes = lbks_system_bytes(&p, r->nx, r->ny, r->nz, r->n_orb);
    if (bytes == 0 || !(r->h > 0.0)) return lbks::set_last_error(LBKS_EINVAL, "invalid request size or parameters");
    if (bytes > s->budget) return lbks::set_last_error(LBKS_ENOMEM, "request needs more device memory than the budget");
    auto job = std::make_unique<Job>();
    job->req = *r;
    job->xyz.assign(r->xyz, r->xyz + 3 * r->n_atoms);
    job->Z.assign(r->Z, r->Z + r->n_atoms);
    job->req.xyz = nullptr;
    job->req.Z = nullptr;
    job->bytes = bytes;
    job->t_submit = Clock::now();
    memset(&job->res, 0, sizeof job->res);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        job->id = s->next_id++;
        *id = job->id;
        s->queue.push_back(job.get());
        s->jobs.emplace(job->id, std::move(job));
    }
    s->cv_work.notify_one();
    return LBKS_OK;
}

int lbks_poll(lbks_server* s, uint64_t id, lbks_result* out, lbks_timing* timing, int* done) {
    if (!s || !done) return lbks::set_last_error(LBKS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return lbks::set_last_error(LBKS_ENOTFOUND, "unknown request id");
    Job* j = it->second.get();
    *done = j->state == 2;
    if (!*done) return LBKS_OK;
    if (out) *out = j->res;
    if (timing) {
        timing->queue_s = std::chrono::duration<double>(j->t_start - j->t_submit).count();
        timing->run_s = std::chrono::duration<double>(j->t_end - j->t_start).count();
        timing->latency_s = std::chrono::duration<double>(j->t_end - j->t_submit).count();
    }
    const int rc = j->rc;
    std::string err = j->err;
    s->jobs.erase(it);
    if (rc != LBKS_OK) return lbks::set_last_error(rc, err.c_str());
    return LBKS_OK;
}

int lbks_server_wait(lbks_server* s, uint64_t id, double timeout_s) {
    if (!s) return lbks::set_last_error(LBKS_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        auto it = s->jobs.find(id);
        return it == s->jobs.end() || it->second->state == 2;
    };
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
        return lbks::set_last_error(LBKS_ETIMEDOUT, "request still running at the deadline");
    if (s->jobs.find(id) == s->jobs.end()) return lbks::set_last_error(LBKS_ENOTFOUND, "unknown request id");
    return LBKS_OK;
}

int lbks_server_get_stats(lbks_server* s, lbks_server_stats* out) {
    if (!s || !out) return lbks::set_last_error(LBKS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->queued = (int)s->queue.size();
    out->running = s->running;
    out->completed = s->completed;
    out->pooled = (int)s->pool.size();
    out->bytes_in_use = s->in_use;
    out->budget_bytes = s->budget;
    return LBKS_OK;
}

}  // extern "C"
