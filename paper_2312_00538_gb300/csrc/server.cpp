// Serving loop for SVM solves (svm_server_* in anova_svm.h): continuous admission of queued
// requests by free worker and device-memory budget, each worker solving on its own CUDA stream.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/anova_svm.h"
#include "anova_internal.h"

namespace {

using clock_type = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    svm_problem *problem = nullptr;
    int64_t footprint = 0;
    clock_type::time_point submitted;
    bool done = false;
    int passed = 0;  // younger requests started ahead of this one while it did not fit
};

// A queued request that does not fit the budget may be passed by at most this many younger
// requests that do fit; after that nothing younger starts until it has started.
constexpr int kMaxPass = 4;

// The admission rule over `count` queued requests in arrival order (footprint(k), passed(k)):
// the index of the request to start, or -1. The oldest starts once it fits the budget beside the
// running requests, or when nothing runs (a request larger than the budget runs alone); while
// it does not fit and has been passed fewer than kMaxPass times, the oldest younger request
// that fits starts instead (backfill).
template <class Footprint, class Passed>
int admission_index(int count, Footprint footprint, Passed passed, int64_t reserved, int64_t budget,
                    int64_t running) {
    if (count <= 0) return -1;
    if (reserved + footprint(0) <= budget || running == 0) return 0;
    if (passed(0) >= kMaxPass) return -1;
    for (int k = 1; k < count; ++k)
        if (reserved + footprint(k) <= budget) return k;
    return -1;
}

}  // namespace

struct svm_server {
    svm_opts opts;
    double tol = 1e-6;
    int device = 0;
    int64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::map<int64_t, Request *> all;
    std::vector<std::thread> workers;
    bool stopping = false;
    int64_t next_ticket = 1, submitted = 0, completed = 0, running = 0;
    int64_t reserved = 0, peak_reserved = 0, backfilled = 0;
    std::vector<double> latencies_ms;
};

extern "C" {

static int64_t plan_bytes(int64_t n, int P, int N, int m, int B, int es) {
    // mirrors the plan's own allocations: sorted keys/perm/fractions/window coordinates,
    // the grids of the fused FFT, the per-work-item tiles (at most one per occupied bin; points
    // lie in a box of half-width kBoxHalf, i.e. 0.4 of the torus per axis), partial results
    const int64_t total = n * P;
    const int64_t g = 2 * (int64_t)N;
    const int64_t tw = B + 2 * m - 1;
    const int64_t bins_axis = (int64_t)(2 * anova::kBoxHalf * g / B) + 2;
    const int64_t bins = std::min<int64_t>(total, P * bins_axis * bins_axis * bins_axis);
    int64_t b = total * (4 + 4 + 4 + 4 + 3 * es + 3 * 8);
    b += (int64_t)es * 4 * P * g * g * g;
    b += (int64_t)es * bins * tw * tw * tw;
    b += (int64_t)es * total;
    return b;
}

int64_t svm_request_footprint(int64_t n, int P, const svm_opts *opts) {
    svm_opts o;
    svm_opts_default(&o);
    if (opts) o = *opts;
    if (n < 1 || P < 1) return 0;
    const int64_t r = std::min<int64_t>(std::max(o.rank, 1), n);
    int64_t b = plan_bytes(n, P, o.N, o.m, 4, 4) + plan_bytes(n, P, o.N_precise, o.m_precise, 2, 8);
    if (o.m_refine != 0 && o.m_refine != o.m_precise) b += plan_bytes(n, P, o.N_precise, o.m_refine, 2, 8);
    b += n * r * (8 + 4) + r * r * 8 * 2;  // low-rank factor (FP64 + FP32 panel) and Woodbury core
    if (o.precond == NYSTROM_RANDOM)
        b += n * r * 8 * 2 + ((r + 31) / 32) * ((r + 31) / 32) * 8192 * ((n + 2047) / 2048);  // K G, K Q, Q^T K Q
    b += n * 8 * 48;                      // iterates, Krylov vectors and scratch of the solver
    if (o.krylov == SVM_KRYLOV_GMRES) b += (n + 1) * 8 * (int64_t)(o.krylov_max + 5);  // GMRES basis
    b += n * 8 * 3;                       // the points on the device
    if (o.autotune)                       // a candidate plan and the timing vectors while tuning
        b += plan_bytes(n, P, o.N_precise, o.m_precise, 2, 8) + n * 8 * 2;
    return b + ((int64_t)16 << 20);       // fixed tables and reduction scratch
}

static void worker_loop(svm_server *s) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Request *req = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // admission (admission_index): the oldest request once it fits the budget, else a
            // younger one that fits (backfill), at most kMaxPass times past the same oldest one
            auto chosen = s->queue.end();
            auto pick = [&]() {
                const int k = admission_index(
                    (int)s->queue.size(), [&](int i) { return s->queue[i]->footprint; },
                    [&](int i) { return s->queue[i]->passed; }, s->reserved, s->budget, s->running);
                chosen = k < 0 ? s->queue.end() : s->queue.begin() + k;
            };
            s->cv_work.wait(lk, [&] {
                if (s->stopping && s->queue.empty()) return true;
                pick();
                return chosen != s->queue.end();
            });
            if (s->queue.empty()) break;
            req = *chosen;
            if (chosen != s->queue.begin()) {
                s->queue.front()->passed += 1;
                s->backfilled += 1;
            }
            s->queue.erase(chosen);
            s->running += 1;
            s->reserved += req->footprint;
            s->peak_reserved = std::max(s->peak_reserved, s->reserved);
        }
        svm_problem &pr = *req->problem;
        svm_opts o = s->opts;
        o.cuda_stream = st;
        if (pr.ell > 0) o.ell = pr.ell;
        if (pr.windows) {
            o.windows = pr.windows;
            o.P = pr.P;
        }
        std::memset(&pr.stats, 0, sizeof(pr.stats));
        pr.b = 0.0;
        pr.status = st ? svm_ipm_solve(pr.X, pr.n, pr.d, pr.y, pr.C, s->tol, &o, pr.alpha, &pr.b, &pr.stats)
                       : ANOVA_ERR_CUDA;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->running -= 1;
            s->reserved -= req->footprint;
            s->completed += 1;
            req->done = true;
            s->latencies_ms.push_back(
                std::chrono::duration<double, std::milli>(clock_type::now() - req->submitted).count());
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
}

anova_status svm_server_admission(const int64_t *footprints, const int32_t *passed, int count,
                                  int64_t reserved_bytes, int64_t budget_bytes, int running, int *pick) {
    if (!pick) return anova::fail(ANOVA_ERR_INVALID_ARG, "pick is NULL");
    *pick = -1;
    if (count < 0) return anova::fail(ANOVA_ERR_INVALID_ARG, "count must be >= 0");
    if (count > 0 && (!footprints || !passed)) return anova::fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    *pick = admission_index(
        count, [&](int i) { return footprints[i]; }, [&](int i) { return (int)passed[i]; }, reserved_bytes,
        budget_bytes, running);
    return ANOVA_OK;
}

anova_status svm_server_create(const svm_opts *opts, double tol, int slots, int64_t hbm_budget_bytes,
                               svm_server_t *out) {
    if (!out) return anova::fail(ANOVA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (slots < 1 || slots > 256) return anova::fail(ANOVA_ERR_INVALID_ARG, "slots must be in [1, 256]");
    if (hbm_budget_bytes <= 0) return anova::fail(ANOVA_ERR_INVALID_ARG, "budget must be positive");
    if (!(tol > 0)) return anova::fail(ANOVA_ERR_INVALID_ARG, "tol must be positive");
    svm_server *s = new (std::nothrow) svm_server();
    if (!s) return anova::fail(ANOVA_ERR_OOM, "host allocation failed");
    svm_opts_default(&s->opts);
    if (opts) s->opts = *opts;
    s->tol = tol;
    s->budget = hbm_budget_bytes;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return anova::fail(ANOVA_ERR_CUDA, "cudaGetDevice failed");
    }
    try {
        for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_loop, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
        }
        s->cv_work.notify_all();
        for (auto &t : s->workers) t.join();
        delete s;
        return anova::fail(ANOVA_ERR_OOM, "cannot start worker threads");
    }
    *out = s;
    return ANOVA_OK;
}

anova_status svm_server_submit(svm_server_t s, svm_problem *problem, int64_t *ticket) {
    if (!s || !problem || !ticket) return anova::fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    if (!problem->X || !problem->y || !problem->alpha || problem->n < 2 || problem->d < 1)
        return anova::fail(ANOVA_ERR_INVALID_ARG, "bad problem");
    Request *req = new (std::nothrow) Request();
    if (!req) return anova::fail(ANOVA_ERR_OOM, "host allocation failed");
    const int P = problem->windows ? problem->P : (s->opts.windows ? s->opts.P : (problem->d + 2) / 3);
    req->problem = problem;
    req->footprint = svm_request_footprint(problem->n, P, &s->opts);
    req->submitted = clock_type::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            delete req;
            return anova::fail(ANOVA_ERR_INVALID_ARG, "server is stopping");
        }
        req->ticket = s->next_ticket++;
        s->all[req->ticket] = req;
        s->queue.push_back(req);
        s->submitted += 1;
        problem->status = ANOVA_OK;
    }
    *ticket = req->ticket;
    s->cv_work.notify_all();
    return ANOVA_OK;
}

anova_status svm_server_wait(svm_server_t s, int64_t ticket) {
    if (!s) return anova::fail(ANOVA_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return anova::fail(ANOVA_ERR_INVALID_ARG, "unknown ticket");
    Request *req = it->second;
    s->cv_done.wait(lk, [&] { return req->done; });
    return req->problem->status;
}

anova_status svm_server_drain(svm_server_t s) {
    if (!s) return anova::fail(ANOVA_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->completed == s->submitted; });
    return ANOVA_OK;
}

anova_status svm_server_get_stats(svm_server_t s, svm_server_stats *out) {
    if (!s || !out) return anova::fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->running = s->running;
    out->queued = (int64_t)s->queue.size();
    out->reserved_bytes = s->reserved;
    out->peak_reserved_bytes = s->peak_reserved;
    out->backfilled = s->backfilled;
    if (!s->latencies_ms.empty()) {
        std::vector<double> v = s->latencies_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const double x = p * (v.size() - 1);
            const size_t i = (size_t)x;
            const double f = x - i;
            return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
        };
        out->p50_latency_ms = pct(0.50);
        out->p99_latency_ms = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_latency_ms = sum / v.size();
    }
    return ANOVA_OK;
}

void svm_server_destroy(svm_server_t s) {
    if (!s) return;
    svm_server_drain(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->all) delete kv.second;
    delete s;
}

}  // extern "C"
