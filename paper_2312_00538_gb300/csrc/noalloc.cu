// anova_spread_grid_noalloc: the spread stage of one window (the same kernels and result as
// anova_spread_grid) for callers that must not allocate device memory. Its scratch -- the
// partial tiles that the spread kernel writes and the reduction kernels read -- lives in a
// file-scope device array of fixed size instead of the plan's on-demand workspace.
#include <cstdint>
#include <mutex>
#include <new>

#include "matvec_impl.cuh"

namespace anova {
namespace {

// 16 MiB, resident on every device that loads this library until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on device `dev` (which must be current). Looked up once
// per device with cudaGetSymbolAddress: in host code the array's name is only a host-side
// stand-in, never a device address.
anova_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(ANOVA_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_addr[dev] = addr;
    }
    *out = g_scratch_addr[dev];
    return ANOVA_OK;
}

template <typename T>
anova_status spread_noalloc(anova_plan *p, int w, const void *v, void *grid) {
    const WindowInfo &wi = p->win[w];
    const size_t tv = (size_t)tile_volume<T>(p, wi.dw);
    // only this window's work items [wi_begin, wi_end) need tiles
    const size_t need = (size_t)(wi.wi_end - wi.wi_begin) * tv * sizeof(T);
    if (need > kNoAllocScratchBytes)
        return fail(ANOVA_ERR_INVALID_ARG,
                    "anova_spread_grid_noalloc: this window needs " + std::to_string(need) +
                        " bytes of scratch; the static scratch holds " +
                        std::to_string(kNoAllocScratchBytes) + " bytes (use anova_spread_grid)");
    void *base = nullptr;
    anova_status st = scratch_address(p->device, &base);
    if (st != ANOVA_OK) return st;
    // the kernels address tiles by plan-wide work-item index; shifting the base by the window's
    // first item puts that item's tile at the start of the array (no access below the array:
    // every index the kernels use is >= wi_begin)
    void *scratch = reinterpret_cast<void *>(reinterpret_cast<uintptr_t>(base) -
                                             (uintptr_t)wi.wi_begin * tv * sizeof(T));
    cudaStream_t s = p->stream;

    SpreadArgs sa;
    sa.packed = 0;  // the generic spread kernel
    sa.order = nullptr;
    sa.wis = p->wis;
    sa.segs = p->segs;
    sa.frac = p->frac;
    sa.perm = p->perm;
    sa.v = v;
    sa.tiles = scratch;
    sa.n = p->n;
    sa.total = p->n * p->P;
    sa.nrhs = 1;
    sa.wi_begin = wi.wi_begin;
    sa.wi_end = wi.wi_end;
    sa.wp = make_winparams<T>(p);
    if (wi.wi_end > wi.wi_begin) {
        cudaError_t e = dispatch_spread<T>(wi.dw, p->m, sa, wi.wi_end - wi.wi_begin, 1, s);
        if (e != cudaSuccess) return cuda_fail(e, "spread launch");
    }
    long long gsz = 1;
    for (int k = 0; k < wi.dw; ++k) gsz *= p->n_os;
    // the grid must start at zero: only the box of the window's footprints is written below
    ANOVA_CUDA_TRY(cudaMemsetAsync(grid, 0, sizeof(T) * gsz, s));

    BinReduceArgs ba;
    ba.tiles = scratch;
    ba.mbins = p->mbins;
    ba.mb_begin = wi.mb_begin;
    ba.nmbins = wi.mb_end - wi.mb_begin;
    ba.nrhs = 1;
    ba.tv_max = (int)tv;
    if (ba.nmbins > 0) {
        const int chunks = (ba.tv_max + kBinReduceChunk - 1) / kBinReduceChunk;
        k_bin_reduce<T><<<dim3(ba.nmbins * chunks, 1), 256, 0, s>>>(ba);
        ANOVA_CUDA_TRY(cudaGetLastError());
    }
    ReduceArgs ra;
    ra.tiles = scratch;
    ra.grid0 = grid;
    ra.dwin = p->dwin;
    ra.bins = p->bins;
    ra.grid_total = gsz;
    ra.w_begin = w;
    ra.w_end = w + 1;
    ra.nrhs = 1;
    ra.n_os = p->n_os;
    ra.NB = p->NB;
    ra.M = p->m;
    ra.B = Prec<T>::B;
    ra.zero_offset = 1;
    ra.box_cum[0] = 0;
    ra.box_cum[1] = wi.box_volume();
    const int nb = (int)((ra.box_cum[1] + 255) / 256);
    if (nb > 0) {
        if (wi.dw == 3) k_reduce<T, 3><<<dim3(nb, 1), 256, 0, s>>>(ra);
        else if (wi.dw == 2) k_reduce<T, 2><<<dim3(nb, 1), 256, 0, s>>>(ra);
        else k_reduce<T, 1><<<dim3(nb, 1), 256, 0, s>>>(ra);
        ANOVA_CUDA_TRY(cudaGetLastError());
    }
    return ANOVA_OK;
}

}  // namespace
}  // namespace anova

using namespace anova;

extern "C" anova_status anova_spread_grid_noalloc(anova_plan_t plan, int l, const void *v, void *grid) {
    try {
        if (!plan) return fail(ANOVA_ERR_INVALID_ARG, "plan is NULL");
        if (l < 0 || l >= plan->P) return fail(ANOVA_ERR_INVALID_ARG, "window index out of range");
        if (!v || !grid) return fail(ANOVA_ERR_INVALID_ARG, "NULL buffer");
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) return fail(ANOVA_ERR_CUDA, "cudaGetDevice failed");
        if (prev != plan->device && cudaSetDevice(plan->device) != cudaSuccess)
            return fail(ANOVA_ERR_CUDA, "cannot select the plan's device");
        const int w = plan->user_to_internal[l];
        anova_status st = plan->prec == ANOVA_FP64 ? spread_noalloc<double>(plan, w, v, grid)
                                                   : spread_noalloc<float>(plan, w, v, grid);
        if (prev != plan->device) cudaSetDevice(prev);
        return st;
    } catch (const std::bad_alloc &) {
        return fail(ANOVA_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(ANOVA_ERR_INVALID_ARG, "unexpected exception");
    }
}
