// Exported C ABI of the ANOVA-NFFT matvec (declarations and contracts in include/anova.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "anova_internal.h"

namespace anova {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

anova_status fail(anova_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

anova_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return ANOVA_ERR_OOM;
    return ANOVA_ERR_CUDA;
}

anova_status create_plan(const double *points, int64_t n, int d, const int32_t *windows, int P,
                         const double *ell, const double *eta, int N, int m, int flags,
                         void *stream, anova_plan_t *out);
void destroy_plan(anova_plan *p);
anova_status tune_plan(const double *points, int64_t n, int d, const int32_t *windows, int P, const double *ell,
                       const double *eta, int N, int m, int flags, void *stream, int nrhs, int reps,
                       anova_tune_report *report, anova_plan_t *out);

// Runs a plan call on the plan's device, restoring the caller's current device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename F>
anova_status guarded(F &&f) {
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return fail(ANOVA_ERR_OOM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(ANOVA_ERR_INVALID_ARG, e.what());
    } catch (...) {
        return fail(ANOVA_ERR_INVALID_ARG, "unknown exception");
    }
}

cudaEvent_t stage_event(anova_plan *p) {
    if (!p->timing) return nullptr;
    cudaEvent_t e = nullptr;
    if (!p->evt_pool.empty()) {
        e = p->evt_pool.back();
        p->evt_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    if (cudaEventRecord(e, p->stream) != cudaSuccess) {
        p->evt_pool.push_back(e);
        return nullptr;
    }
    return e;
}

void stage_record(anova_plan *p, int stage, cudaEvent_t a, cudaEvent_t b) {
    if (!p->timing || !a || !b) return;
    p->evts.push_back({stage, a, b});
}

static void reset_timing(anova_plan *p) {
    std::vector<cudaEvent_t> seen;
    for (auto &x : p->evts) {
        for (cudaEvent_t e : {x.a, x.b})
            if (std::find(seen.begin(), seen.end(), e) == seen.end()) seen.push_back(e);
    }
    for (cudaEvent_t e : seen) p->evt_pool.push_back(e);
    p->evts.clear();
    p->launches = 0;
}

void release_timing(anova_plan *p) {
    reset_timing(p);
    for (cudaEvent_t e : p->evt_pool) cudaEventDestroy(e);
    p->evt_pool.clear();
}

}  // namespace anova

using namespace anova;

extern "C" {

anova_status anova_nfft_plan(const double *points, int64_t n, int d, const int32_t *windows, int P,
                             double sigma, int N, int m, int flags, void *cuda_stream,
                             anova_plan_t *out) {
    return guarded([&]() -> anova_status {
        if (P < 1 || P > kMaxWindows) return fail(ANOVA_ERR_INVALID_ARG, "P must be in [1, 64]");
        std::vector<double> ell(P, sigma);
        return create_plan(points, n, d, windows, P, ell.data(), nullptr, N, m, flags, cuda_stream, out);
    });
}

anova_status anova_nfft_plan_ex(const double *points, int64_t n, int d, const int32_t *windows,
                                int P, const double *ell, const double *eta, int N, int m,
                                int flags, void *cuda_stream, anova_plan_t *out) {
    return guarded([&]() -> anova_status {
        return create_plan(points, n, d, windows, P, ell, eta, N, m, flags, cuda_stream, out);
    });
}

anova_status anova_nfft_plan_tuned(const double *points, int64_t n, int d, const int32_t *windows, int P,
                                   const double *ell, const double *eta, int N, int m, int flags,
                                   void *cuda_stream, int nrhs, int reps, anova_tune_report *report,
                                   anova_plan_t *out) {
    return guarded([&]() -> anova_status {
        return tune_plan(points, n, d, windows, P, ell, eta, N, m, flags, cuda_stream, nrhs, reps, report, out);
    });
}

anova_status anova_matvec(anova_plan_t plan, const void *v, void *Kv, int nrhs) {
    return guarded([&]() -> anova_status {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        if (!v || !Kv) return fail(ANOVA_ERR_INVALID_ARG, "v or Kv is NULL");
        if (nrhs < 1) return fail(ANOVA_ERR_INVALID_ARG, "nrhs must be >= 1");
        const size_t bytes = elem_size(plan) * (size_t)plan->n * nrhs;
        const char *a = (const char *)v, *b = (const char *)Kv;
        if (a < b + bytes && b < a + bytes) return fail(ANOVA_ERR_INVALID_ARG, "v and Kv overlap");
        DeviceGuard g(plan->device);
        if (!g.ok) return fail(ANOVA_ERR_CUDA, "cannot select the plan's device");
        if (plan->prec == ANOVA_FP64) return run_matvec_t<double>(plan, v, Kv, nrhs, -1);
        return run_matvec_t<float>(plan, v, Kv, nrhs, -1);
    });
}

anova_status anova_plan_grid_size(anova_plan_t plan, int64_t *grid_total) {
    if (!plan || !grid_total) return fail(ANOVA_ERR_INVALID_ARG, "NULL argument");
    *grid_total = plan->grid_total;
    return ANOVA_OK;
}

anova_status anova_matvec_grids(anova_plan_t plan, const void *v, void *grids, int nrhs) {
    return guarded([&]() -> anova_status {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        if (!v || !grids) return fail(ANOVA_ERR_INVALID_ARG, "v or grids is NULL");
        if (nrhs < 1) return fail(ANOVA_ERR_INVALID_ARG, "nrhs must be >= 1");
        const size_t vb = elem_size(plan) * (size_t)plan->n * nrhs, gb = elem_size(plan) * (size_t)plan->grid_total * nrhs;
        const char *a = (const char *)v, *b = (const char *)grids;
        if (a < b + gb && b < a + vb) return fail(ANOVA_ERR_INVALID_ARG, "v and grids overlap");
        DeviceGuard g(plan->device);
        if (!g.ok) return fail(ANOVA_ERR_CUDA, "cannot select the plan's device");
        if (plan->prec == ANOVA_FP64) return run_matvec_grids_t<double>(plan, v, grids, nrhs);
        return run_matvec_grids_t<float>(plan, v, grids, nrhs);
    });
}

anova_status anova_matvec_from_grids(anova_plan_t plan, const void *grids, void *Kv, int nrhs) {
    return guarded([&]() -> anova_status {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        if (!grids || !Kv) return fail(ANOVA_ERR_INVALID_ARG, "grids or Kv is NULL");
        if (nrhs < 1) return fail(ANOVA_ERR_INVALID_ARG, "nrhs must be >= 1");
        const size_t kb = elem_size(plan) * (size_t)plan->n * nrhs, gb = elem_size(plan) * (size_t)plan->grid_total * nrhs;
        const char *a = (const char *)Kv, *b = (const char *)grids;
        if (a < b + gb && b < a + kb) return fail(ANOVA_ERR_INVALID_ARG, "Kv and grids overlap");
        DeviceGuard g(plan->device);
        if (!g.ok) return fail(ANOVA_ERR_CUDA, "cannot select the plan's device");
        if (plan->prec == ANOVA_FP64) return run_matvec_from_grids_t<double>(plan, grids, Kv, nrhs);
        return run_matvec_from_grids_t<float>(plan, grids, Kv, nrhs);
    });
}

// Captures the host-buffer matvec (copy in, stage chain, copy out) on the plan's private stream as
// one graph for the next call with the same buffers. Any failure leaves no graph behind (the next
// call takes the stream path again); the plan's own stream is restored in every case.
static void capture_host_graph(anova_plan *p, const void *v_host, void *Kv_host, int nrhs, size_t bytes) {
    if (p->host_exec) {
        cudaGraphExecDestroy(p->host_exec);
        p->host_exec = nullptr;
    }
    if (!p->host_cap && cudaStreamCreateWithFlags(&p->host_cap, cudaStreamNonBlocking) != cudaSuccess) {
        p->host_cap = nullptr;
        cudaGetLastError();
        return;
    }
    cudaStream_t saved = p->stream;
    p->stream = p->host_cap;
    cudaGraph_t graph = nullptr;
    anova_status s = ANOVA_OK;
    cudaError_t e = cudaStreamBeginCapture(p->host_cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = cudaMemcpyAsync(p->dv, v_host, bytes, cudaMemcpyHostToDevice, p->host_cap);
        if (e == cudaSuccess)
            s = p->prec == ANOVA_FP64 ? run_matvec_t<double>(p, p->dv, p->dkv, nrhs, -1)
                                      : run_matvec_t<float>(p, p->dv, p->dkv, nrhs, -1);
        if (e == cudaSuccess && s == ANOVA_OK)
            e = cudaMemcpyAsync(Kv_host, p->dkv, bytes, cudaMemcpyDeviceToHost, p->host_cap);
        const cudaError_t e_end = cudaStreamEndCapture(p->host_cap, &graph);
        if (e == cudaSuccess) e = e_end;
    }
    p->stream = saved;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && s == ANOVA_OK && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        p->host_exec = exec;
        p->host_v = v_host;
        p->host_kv = Kv_host;
        p->host_dv = p->dv;
        p->host_nrhs = nrhs;
        p->host_gen = p->ws_gen;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();  // a refused capture leaves only a non-sticky error behind
}

anova_status anova_matvec_host(anova_plan_t plan, const void *v_host, void *Kv_host, int nrhs) {
    return guarded([&]() -> anova_status {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        if (!v_host || !Kv_host) return fail(ANOVA_ERR_INVALID_ARG, "v or Kv is NULL");
        if (nrhs < 1) return fail(ANOVA_ERR_INVALID_ARG, "nrhs must be >= 1");
        DeviceGuard g(plan->device);
        if (!g.ok) return fail(ANOVA_ERR_CUDA, "cannot select the plan's device");
        const size_t bytes = elem_size(plan) * (size_t)plan->n * nrhs;
        if (!plan->timing && plan->host_exec && plan->host_v == v_host && plan->host_kv == Kv_host &&
            plan->host_nrhs == nrhs && plan->host_gen == plan->ws_gen && plan->host_dv == plan->dv &&
            nrhs <= plan->stage_rhs) {
            ANOVA_CUDA_TRY(cudaGraphLaunch(plan->host_exec, plan->stream));
            ANOVA_CUDA_TRY(cudaStreamSynchronize(plan->stream));
            return ANOVA_OK;
        }
        if (nrhs > plan->stage_rhs) {
            cudaStreamSynchronize(plan->stream);
            if (plan->dv) cudaFree(plan->dv);
            if (plan->dkv) cudaFree(plan->dkv);
            plan->dv = plan->dkv = nullptr;
            plan->stage_rhs = 0;
            cudaError_t e;
            if ((e = cudaMalloc(&plan->dv, bytes)) != cudaSuccess ||
                (e = cudaMalloc(&plan->dkv, bytes)) != cudaSuccess)
                return fail(ANOVA_ERR_OOM, "staging allocation failed");
            plan->stage_rhs = nrhs;
        }
        ANOVA_CUDA_TRY(cudaMemcpyAsync(plan->dv, v_host, bytes, cudaMemcpyHostToDevice, plan->stream));
        anova_status st = plan->prec == ANOVA_FP64
                              ? run_matvec_t<double>(plan, plan->dv, plan->dkv, nrhs, -1)
                              : run_matvec_t<float>(plan, plan->dv, plan->dkv, nrhs, -1);
        if (st != ANOVA_OK) return st;
        ANOVA_CUDA_TRY(cudaMemcpyAsync(Kv_host, plan->dkv, bytes, cudaMemcpyDeviceToHost, plan->stream));
        ANOVA_CUDA_TRY(cudaStreamSynchronize(plan->stream));
        if (!plan->timing) capture_host_graph(plan, v_host, Kv_host, nrhs, bytes);
        return ANOVA_OK;
    });
}

static anova_status window_index(anova_plan_t plan, int l, int *w) {
    if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
    if (l < 0 || l >= plan->P) return fail(ANOVA_ERR_INVALID_ARG, "window index out of range");
    *w = plan->user_to_internal[l];
    return ANOVA_OK;
}

anova_status anova_window_matvec(anova_plan_t plan, int l, const void *v, void *Kv) {
    return guarded([&]() -> anova_status {
        int w;
        anova_status st = window_index(plan, l, &w);
        if (st != ANOVA_OK) return st;
        if (!v || !Kv) return fail(ANOVA_ERR_INVALID_ARG, "v or Kv is NULL");
        DeviceGuard g(plan->device);
        if (plan->prec == ANOVA_FP64) return run_matvec_t<double>(plan, v, Kv, 1, w);
        return run_matvec_t<float>(plan, v, Kv, 1, w);
    });
}

anova_status anova_spread_grid(anova_plan_t plan, int l, const void *v, void *grid) {
    return guarded([&]() -> anova_status {
        int w;
        anova_status st = window_index(plan, l, &w);
        if (st != ANOVA_OK) return st;
        if (!v || !grid) return fail(ANOVA_ERR_INVALID_ARG, "NULL buffer");
        DeviceGuard g(plan->device);
        if (plan->prec == ANOVA_FP64) return run_spread_grid_t<double>(plan, w, v, grid);
        return run_spread_grid_t<float>(plan, w, v, grid);
    });
}

anova_status anova_conv_grid(anova_plan_t plan, int l, const void *grid_in, void *grid_out) {
    return guarded([&]() -> anova_status {
        int w;
        anova_status st = window_index(plan, l, &w);
        if (st != ANOVA_OK) return st;
        if (!grid_in || !grid_out) return fail(ANOVA_ERR_INVALID_ARG, "NULL buffer");
        DeviceGuard g(plan->device);
        if (plan->prec == ANOVA_FP64) return run_conv_grid_t<double>(plan, w, grid_in, grid_out);
        return run_conv_grid_t<float>(plan, w, grid_in, grid_out);
    });
}

anova_status anova_interp_grid(anova_plan_t plan, int l, const void *grid, void *f) {
    return guarded([&]() -> anova_status {
        int w;
        anova_status st = window_index(plan, l, &w);
        if (st != ANOVA_OK) return st;
        if (!grid || !f) return fail(ANOVA_ERR_INVALID_ARG, "NULL buffer");
        DeviceGuard g(plan->device);
        if (plan->prec == ANOVA_FP64) return run_interp_grid_t<double>(plan, w, grid, f);
        return run_interp_grid_t<float>(plan, w, grid, f);
    });
}

anova_status anova_plan_info(anova_plan_t plan, int64_t *n, int *P, int *n_os, int *flags,
                             int64_t *device_bytes) {
    if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
    if (n) *n = plan->n;
    if (P) *P = plan->P;
    if (n_os) *n_os = plan->n_os;
    if (flags) *flags = plan->prec | plan->interp_flags;
    if (device_bytes) *device_bytes = plan->static_bytes + plan->ws_bytes;
    return ANOVA_OK;
}

anova_status anova_cross_matvec(anova_plan_t source, anova_plan_t target, const void *w, void *f) {
    return guarded([&]() -> anova_status {
        if (!source || !target) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        if (!w || !f) return fail(ANOVA_ERR_INVALID_ARG, "w or f is NULL");
        if (source->device != target->device) return fail(ANOVA_ERR_INVALID_ARG, "plans on different devices");
        if (source->prec != target->prec || source->N != target->N || source->m != target->m ||
            source->P != target->P || source->user_to_internal != target->user_to_internal)
            return fail(ANOVA_ERR_INVALID_ARG, "source and target plans differ in precision, N, m or windows");
        for (int k = 0; k < source->P; ++k) {
            const WindowInfo &a = source->win[k], &b = target->win[k];
            if (a.dw != b.dw || a.ell != b.ell || a.eta != b.eta)
                return fail(ANOVA_ERR_INVALID_ARG, "source and target plans differ in a window's dimension, ell or eta");
        }
        DeviceGuard g(source->device);
        if (source->prec == ANOVA_FP64) return run_cross_matvec_t<double>(source, target, w, f);
        return run_cross_matvec_t<float>(source, target, w, f);
    });
}

anova_status anova_model_create(anova_plan_t source, const void *w, anova_model_t *out) {
    return guarded([&]() -> anova_status {
        if (!out) return fail(ANOVA_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        if (!source) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        if (!w) return fail(ANOVA_ERR_INVALID_ARG, "w is NULL");
        DeviceGuard g(source->device);
        if (!g.ok) return fail(ANOVA_ERR_CUDA, "cannot select the plan's device");
        std::unique_ptr<anova_model> m(new anova_model());
        m->device = source->device;
        m->prec = source->prec;
        m->N = source->N;
        m->m = source->m;
        m->P = source->P;
        m->user_to_internal = source->user_to_internal;
        m->win = source->win;
        m->grid_total = source->grid_total;
        ANOVA_CUDA_TRY(cudaMalloc(&m->grid, elem_size(source) * (size_t)source->grid_total));
        const anova_status st = source->prec == ANOVA_FP64 ? run_model_create_t<double>(source, w, m.get())
                                                           : run_model_create_t<float>(source, w, m.get());
        if (st != ANOVA_OK) {
            cudaFree(m->grid);
            return st;
        }
        *out = m.release();
        return ANOVA_OK;
    });
}

anova_status anova_model_eval(anova_model_t model, anova_plan_t target, void *f) {
    return guarded([&]() -> anova_status {
        if (!model || !target) return fail(ANOVA_ERR_INVALID_ARG, "model or plan is NULL");
        if (!f) return fail(ANOVA_ERR_INVALID_ARG, "f is NULL");
        if (model->device != target->device) return fail(ANOVA_ERR_INVALID_ARG, "model and plan on different devices");
        if (model->prec != target->prec || model->N != target->N || model->m != target->m || model->P != target->P ||
            model->user_to_internal != target->user_to_internal || model->grid_total != target->grid_total)
            return fail(ANOVA_ERR_INVALID_ARG, "model and target plan differ in precision, N, m or windows");
        for (int k = 0; k < model->P; ++k) {
            const WindowInfo &a = model->win[k], &b = target->win[k];
            if (a.dw != b.dw || a.ell != b.ell || a.eta != b.eta || a.grid_off != b.grid_off)
                return fail(ANOVA_ERR_INVALID_ARG, "model and target plan differ in a window's dimension, ell or eta");
        }
        DeviceGuard g(target->device);
        if (!g.ok) return fail(ANOVA_ERR_CUDA, "cannot select the plan's device");
        if (target->prec == ANOVA_FP64) return run_model_eval_t<double>(model, target, f);
        return run_model_eval_t<float>(model, target, f);
    });
}

void anova_model_destroy(anova_model_t model) {
    if (!model) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != model->device) cudaSetDevice(model->device);
    cudaFree(model->grid);
    if (prev >= 0 && prev != model->device) cudaSetDevice(prev);
    delete model;
}

anova_status anova_plan_check(anova_plan_t plan) {
    return guarded([&]() -> anova_status {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        DeviceGuard g(plan->device);
        ANOVA_CUDA_TRY(cudaStreamSynchronize(plan->stream));
        int flag = 0;
        ANOVA_CUDA_TRY(cudaMemcpy(&flag, plan->dev_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) return fail(ANOVA_ERR_TIMEOUT, "a bounded tensor-core wait inside a kernel ran out");
        return ANOVA_OK;
    });
}

anova_status anova_plan_set_wait_limit(anova_plan_t plan, int64_t polls) {
    return guarded([&]() -> anova_status {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        DeviceGuard g(plan->device);
        ANOVA_CUDA_TRY(cudaStreamSynchronize(plan->stream));
        const int64_t full = (int64_t)1 << 22;
        plan->wait_polls = (unsigned)(polls < 0 ? full : std::min(polls, full));
        return ANOVA_OK;
    });
}

void anova_plan_destroy(anova_plan_t plan) {
    if (!plan) return;
    DeviceGuard g(plan->device);
    cudaStreamSynchronize(plan->stream);
    release_timing(plan);
    destroy_plan(plan);
}

anova_status anova_plan_set_timing(anova_plan_t plan, int enable) {
    return guarded([&]() -> anova_status {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        DeviceGuard g(plan->device);
        ANOVA_CUDA_TRY(cudaStreamSynchronize(plan->stream));
        reset_timing(plan);
        plan->timing = enable != 0;
        return ANOVA_OK;
    });
}

anova_status anova_plan_stage_times(anova_plan_t plan, double *ms, int64_t *launches) {
    return guarded([&]() -> anova_status {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        DeviceGuard g(plan->device);
        ANOVA_CUDA_TRY(cudaStreamSynchronize(plan->stream));
        double acc[NUM_STAGES] = {0, 0, 0, 0, 0};
        for (auto &x : plan->evts) {
            float t = 0.f;
            ANOVA_CUDA_TRY(cudaEventElapsedTime(&t, x.a, x.b));
            acc[x.stage] += t;
        }
        if (ms)
            for (int s = 0; s < NUM_STAGES; ++s) ms[s] = acc[s];
        if (launches) *launches = plan->launches;
        return ANOVA_OK;
    });
}

anova_status anova_kernel_coeffs(double ell, int N, double *b) {
    return guarded([&]() -> anova_status {
        if (!b) return fail(ANOVA_ERR_INVALID_ARG, "b is NULL");
        if (N < 2 || N > 1024 || (N & 1)) return fail(ANOVA_ERR_INVALID_ARG, "N must be even, 2..1024");
        if (!(ell > 0.0) || !std::isfinite(ell)) return fail(ANOVA_ERR_INVALID_ARG, "ell must be positive");
        std::vector<double> c;
        if (!kernel_coeffs(ell, N, c)) return fail(ANOVA_ERR_INVALID_ARG, "coefficient fit failed");
        std::memcpy(b, c.data(), sizeof(double) * c.size());
        return ANOVA_OK;
    });
}

anova_status anova_window_hat(int m, int n_os, int count, double *Psi) {
    return guarded([&]() -> anova_status {
        if (!Psi || count < 0) return fail(ANOVA_ERR_INVALID_ARG, "bad output");
        if (m < 1 || m > 16 || n_os < 2 * m) return fail(ANOVA_ERR_INVALID_ARG, "bad m / n_os");
        window_hat(m, n_os, count, Psi);
        return ANOVA_OK;
    });
}

const char *anova_last_error(void) { return g_last_error.c_str(); }

const char *anova_version(void) { return "anova-nfft-gb300 0.1"; }

}  // extern "C"
