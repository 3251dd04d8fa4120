// Matvecs of several plans (independent problems of uneven size) as one CUDA graph: each plan's
// stage chain (spread, reduce, FFT passes, interpolation, window sum) is captured on its own
// branch, so one graph launch runs them all and small problems fill the GPU together.
#include <vector>

#include "anova_internal.h"

namespace anova {
anova_status fail(anova_status st, const std::string &msg);
anova_status cuda_fail(cudaError_t e, const char *what);
}  // namespace anova

using namespace anova;

struct anova_batch {
    int device = 0;
    cudaStream_t stream = nullptr;  // the stream the graph is launched on (not owned)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the graph holds the addresses of each plan's workspace as captured; a later call that
    // grows a plan's workspace frees those buffers, which this generation check detects
    std::vector<anova_plan *> plans;
    std::vector<uint64_t> ws_gen;
};

namespace {

anova_status run_one(anova_plan *p, const void *v, void *kv, int nrhs) {
    return p->prec == ANOVA_FP64 ? run_matvec_t<double>(p, v, kv, nrhs, -1) : run_matvec_t<float>(p, v, kv, nrhs, -1);
}

void release(anova_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

}  // namespace

extern "C" {

anova_status anova_matvec_batch_create(int count, anova_plan_t const *plans, const void *const *v,
                                       void *const *Kv, const int *nrhs, void *cuda_stream,
                                       anova_batch_t *out) {
    try {
        if (!out) return fail(ANOVA_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        if (count < 1 || count > 4096) return fail(ANOVA_ERR_INVALID_ARG, "count must be in [1, 4096]");
        if (!plans || !v || !Kv) return fail(ANOVA_ERR_INVALID_ARG, "NULL array");
        int device = -1;
        for (int k = 0; k < count; ++k) {
            anova_plan *p = plans[k];
            if (!p || !v[k] || !Kv[k]) return fail(ANOVA_ERR_INVALID_ARG, "NULL plan or vector");
            const int nr = nrhs ? nrhs[k] : 1;
            if (nr < 1) return fail(ANOVA_ERR_INVALID_ARG, "nrhs must be >= 1");
            if (device < 0) device = p->device;
            if (p->device != device) return fail(ANOVA_ERR_INVALID_ARG, "plans on different devices");
            if (p->timing) return fail(ANOVA_ERR_INVALID_ARG, "stage timing is on for a plan");
            for (int k2 = 0; k2 < k; ++k2)
                if (plans[k2] == p) return fail(ANOVA_ERR_INVALID_ARG, "a plan appears twice (its workspace is shared)");
        }
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != device && cudaSetDevice(device) != cudaSuccess) return fail(ANOVA_ERR_CUDA, "cudaSetDevice");
        struct Restore {
            int prev, dev;
            ~Restore() {
                if (prev >= 0 && prev != dev) cudaSetDevice(prev);
            }
        } restore{prev, device};
        // one ordinary run of every matvec first: it sizes the workspaces and sets the kernels'
        // attributes, so that the capture below records launches only
        for (int k = 0; k < count; ++k) {
            anova_status s = run_one(plans[k], v[k], Kv[k], nrhs ? nrhs[k] : 1);
            if (s != ANOVA_OK) return s;
        }
        for (int k = 0; k < count; ++k) ANOVA_CUDA_TRY(cudaStreamSynchronize(plans[k]->stream));

        anova_batch *b = new anova_batch();
        b->device = device;
        b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
        struct Owned {
            anova_batch *b;
            ~Owned() { release(b); }
        } owned{b};
        // capture: a root stream forks to one private stream per plan and joins them again
        cudaStream_t root = nullptr;
        std::vector<cudaStream_t> cs(count, nullptr);
        std::vector<cudaEvent_t> ev(count + 1, nullptr);
        std::vector<cudaStream_t> saved(count);
        struct Streams {
            cudaStream_t &root;
            std::vector<cudaStream_t> &cs;
            std::vector<cudaEvent_t> &ev;
            ~Streams() {
                for (cudaEvent_t e : ev)
                    if (e) cudaEventDestroy(e);
                for (cudaStream_t s : cs)
                    if (s) cudaStreamDestroy(s);
                if (root) cudaStreamDestroy(root);
            }
        } streams{root, cs, ev};
        ANOVA_CUDA_TRY(cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking));
        for (int k = 0; k < count; ++k) ANOVA_CUDA_TRY(cudaStreamCreateWithFlags(&cs[k], cudaStreamNonBlocking));
        for (int k = 0; k <= count; ++k) ANOVA_CUDA_TRY(cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming));
        for (int k = 0; k < count; ++k) {
            saved[k] = plans[k]->stream;
            plans[k]->stream = cs[k];
        }
        anova_status s = ANOVA_OK;
        cudaError_t e = cudaStreamBeginCapture(root, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) e = cudaEventRecord(ev[count], root);
        for (int k = 0; k < count && e == cudaSuccess && s == ANOVA_OK; ++k) {
            e = cudaStreamWaitEvent(cs[k], ev[count], 0);
            if (e == cudaSuccess) s = run_one(plans[k], v[k], Kv[k], nrhs ? nrhs[k] : 1);
            if (e == cudaSuccess && s == ANOVA_OK) e = cudaEventRecord(ev[k], cs[k]);
            if (e == cudaSuccess && s == ANOVA_OK) e = cudaStreamWaitEvent(root, ev[k], 0);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t e_end = cudaStreamEndCapture(root, &graph);
        for (int k = 0; k < count; ++k) plans[k]->stream = saved[k];
        if (s != ANOVA_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e, "batch capture");
        }
        if (e_end != cudaSuccess) return cuda_fail(e_end, "cudaStreamEndCapture");
        b->graph = graph;
        ANOVA_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
        b->plans.assign(plans, plans + count);
        for (int k = 0; k < count; ++k) b->ws_gen.push_back(plans[k]->ws_gen);
        owned.b = nullptr;
        *out = b;
        return ANOVA_OK;
    } catch (const std::bad_alloc &) {
        return fail(ANOVA_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(ANOVA_ERR_INVALID_ARG, "unexpected exception");
    }
}

anova_status anova_matvec_batch_run(anova_batch_t batch) {
    if (!batch) return fail(ANOVA_ERR_INVALID_ARG, "batch is NULL");
    for (size_t k = 0; k < batch->plans.size(); ++k)
        if (batch->plans[k]->ws_gen != batch->ws_gen[k])
            return fail(ANOVA_ERR_INVALID_ARG,
                        "plan " + std::to_string(k) +
                            " reallocated its workspace after the batch was captured (a later call used "
                            "more right-hand sides); create the batch again");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != batch->device && cudaSetDevice(batch->device) != cudaSuccess)
        return fail(ANOVA_ERR_CUDA, "cudaSetDevice");
    const cudaError_t e = cudaGraphLaunch(batch->exec, batch->stream);
    if (prev >= 0 && prev != batch->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return ANOVA_OK;
}

void anova_matvec_batch_destroy(anova_batch_t batch) { release(batch); }

}  // extern "C"
