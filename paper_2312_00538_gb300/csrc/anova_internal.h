// Internal declarations of the ANOVA-NFFT library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/anova.h"

namespace anova {

// ----------------------------------------------------------------------------- fixed choices
constexpr double kOversampling = 2.0;  // n_os = 2N
constexpr double kEpsB = 0.1;          // kernel fit on |t| <= 1/2 - eps_B
constexpr double kBoxHalf = 0.2;       // points in [-0.2, 0.2]
constexpr int kSegMax = 256;           // points per segment (one cell, split at this size)
constexpr int kSpreadSplit = 8;        // warps of the packed FP32 spread (cost-balanced point ranges)
#ifndef ANOVA_WI_MAX
#define ANOVA_WI_MAX 2048
#endif
constexpr int kWiMax = ANOVA_WI_MAX;  // points per spread work item (at most)
#ifndef ANOVA_F64_B
#define ANOVA_F64_B 4
#endif
constexpr int kBinF64 = ANOVA_F64_B;   // cells per bin edge of FP64 plans
#ifndef ANOVA_F32_B
#define ANOVA_F32_B 4
#endif
constexpr int kBinF32 = ANOVA_F32_B;   // cells per bin edge of FP32 plans
// a point's cell index inside its bin is stored in one byte
static_assert(kBinF32 * kBinF32 * kBinF32 <= 256 && kBinF64 * kBinF64 * kBinF64 <= 256, "bin too large");
#ifndef ANOVA_CONV_LINES
#define ANOVA_CONV_LINES 16
#endif
constexpr int kConvLines = ANOVA_CONV_LINES;  // default grid lines per CTA of an FFT pass (8, 16 or 32)
constexpr int kPolyDeg = 7;            // Horner degree of the FP32 window polynomials
constexpr int kPolyDeg64 = 13;         // Horner degree of the FP64 window polynomials
constexpr int kMaxWindows = 64;
constexpr int kTcChunkRows = 128;        // points per chunk of the tensor-core interpolation
constexpr int kTcMinPointsPerItem = 512;  // mean points per work item for the tensor-core
                                          // interpolation (FP32, m = 4, 3-D windows)
constexpr int kStatusAlloc = 128;      // ints of a plan's status/counter block (>= 1 + 3 x 32)

// ----------------------------------------------------------------------------- host maths
double kb_beta();
double kb_window(double t, int m);
bool kernel_coeffs(double ell, int N, std::vector<double> &b);
void window_hat(int m, int n_os, int count, double *Psi);
bool window_poly(int m, int deg, std::vector<double> &coef);
bool deconv_diag(double ell, int N, int m, int n_os, std::vector<double> &D1);

// ----------------------------------------------------------------------------- error state
void set_error(const std::string &msg);
anova_status fail(anova_status st, const std::string &msg);
anova_status cuda_fail(cudaError_t e, const char *what);

#define ANOVA_CUDA_TRY(call)                                             \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return ::anova::cuda_fail(_e, #call);     \
    } while (0)

// ----------------------------------------------------------------------------- plan layout
struct WindowInfo {
    int dw = 0;                 // number of features, 1..3
    int feat[3] = {-1, -1, -1};
    double ell = 1.0, eta = 1.0;
    int seg_begin = 0, seg_end = 0;  // global segment range
    int wi_begin = 0, wi_end = 0;    // global spread work-item range
    int box_lo[3] = {0, 0, 0}, box_hi[3] = {0, 0, 0};  // grid box touched by footprints
    int64_t grid_off = 0;            // element offset of this window's grid (one RHS)
    int bin_off = 0;                 // offset of this window's bin table
    int tile_begin[3] = {0, 0, 0}, tile_end[3] = {0, 0, 0};  // FFT tiles of each axis pass
    int full_begin[3] = {0, 0, 0}, full_end[3] = {0, 0, 0};  // the same over the whole grid
    int mb_begin = 0, mb_end = 0;    // bins split into several work items
    int64_t box_volume() const {
        int64_t v = 1;
        for (int k = 0; k < dw; ++k) v *= (box_hi[k] - box_lo[k]);
        return v;
    }
};

// A group of consecutive windows with the same number of features (one launch per group).
struct Group {
    int dw = 0;
    int w_begin = 0, w_end = 0;
    int seg_begin = 0, seg_end = 0;
    int wi_begin = 0, wi_end = 0;
    int tiles_begin[3] = {0, 0, 0}, tiles_end[3] = {0, 0, 0};  // FFT tiles per pass
};

// Per-window constants of the device kernels (small; copied into a device table).
struct DevWindow {
    int dw;
    int box_lo[3], box_hi[3];
    long long grid_off;
    int bin_off;
    int pad;
};

}  // namespace anova

struct anova_plan {
    int64_t n = 0;
    int d = 0, P = 0, N = 0, m = 0, n_os = 0, prec = 0;
    int B = 4;          // bin edge in cells
    int NB = 0;         // bins per dimension
    int tile_w = 0;     // spread tile edge: B + 2m - 1
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<anova::WindowInfo> win;   // internal window order (grouped by dw)
    std::vector<int> user_to_internal;    // user window index -> internal index
    std::vector<anova::Group> groups;
    int nseg = 0, nwi = 0, ntiles = 0;
    int64_t grid_total = 0;               // elements of all windows' grids (one RHS)
    std::vector<double> poly;             // window polynomial coefficients (FP32 kernels)
    std::vector<double> poly64;           // window polynomial coefficients (FP64 kernels)

    // device memory
    void *frac = nullptr;         // T[3][P*n]: fractional cell offsets, sorted per window
    double *xw = nullptr;         // double[P][3][n]: window coordinates in original point order
    int32_t *perm = nullptr;      // [P*n]: sorted position -> original point index
    unsigned char *cellloc = nullptr;  // [P*n]: cell index inside its bin, (l0 B + l1) B + l2
    int4 *segs = nullptr;         // {cell packed, sorted start, count, window}
    int4 *wis = nullptr;          // {window, seg_begin, seg_end, tile origin packed}
    int4 *chunks = nullptr;       // tensor-core interpolation chunks: up to kTcChunkRows
                                  // consecutive points of one cell column of a work item,
                                  // {sorted start, count, l0 | l1 << 8 (column in the bin), 0}
    int *wi_chunk = nullptr;      // [nwi + 1]: work item x owns chunks [wi_chunk[x], wi_chunk[x + 1])
    int *wsplit = nullptr;        // [nwi][kSpreadSplit + 1]: sorted-point ranges of the packed spread's warps
    int *wi_order = nullptr;      // per window: its work items by decreasing point count
    int *wi_gorder = nullptr;     // per dimension group: all its work items by decreasing point count
    int2 *bins = nullptr;         // per window per bin: {first work item, count}
    int4 *mbins = nullptr;        // multi-item bins: {first work item, count, tile volume, 0}
    int nmbins = 0;
    int4 *ftiles = nullptr;       // FFT tiles: {window, p, q0, pass}
    int4 *ftiles_full = nullptr;  // FFT tiles over whole grids (products from summed grids)
    anova::DevWindow *dwin = nullptr;
    void *D1br = nullptr;         // T[P][3][n_os]: deconvolution diagonal per axis, bit-reversed
    void *tw = nullptr;           // T[n_os]: twiddles (re, im) pairs for k < n_os/2
    int *dev_status = nullptr;    // [0]: kernel-side error bits (a bounded tensor-core wait ran
                                  // out); [1 + 32 k + r] / [1 + 32 k + 16 + r]: work and exit
                                  // counters of RHS r of a persistent launch on window stream k
                                  // (kStatusAlloc ints)
    int sm_count = 0;
    // windows of one matvec run concurrently on these streams (forked from and joined back to
    // `stream`); window w uses aux[w % kAuxStreams] and work-counter block w % kAuxStreams
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork_evt = nullptr, join_evt[3] = {nullptr, nullptr, nullptr};
    int interp_flags = 0;         // ANOVA_INTERP_TENSOR / ANOVA_INTERP_SIMT as created or tuned
    int wi_max = anova::kWiMax;   // points per work item (at most); set at plan creation
    int conv_lines = anova::kConvLines;  // grid lines per CTA of an FFT pass (8, 16 or 32)
    int rhs_chunk = 16;           // right-hand sides per pass of the multi-RHS matvec (1..16)
    int fork_windows = 1;         // FP64: run windows of one dimension group on the aux streams
    unsigned wait_polls = 1u << 22;  // polls of a bounded tensor-core completion wait (about a
                                     // second); anova_plan_set_wait_limit lowers it
    int64_t static_bytes = 0;

    // workspace, grown on demand
    int ws_rhs = 0;
    void *grids = nullptr;        // T[4][ws_rhs][grid_total]
    void *tiles = nullptr;        // T[nwi][ws_rhs][tile_vol]
    void *part = nullptr;         // T[P][ws_rhs][n]
    int64_t ws_bytes = 0;
    uint64_t ws_gen = 0;          // bumped whenever the workspace buffers are freed, so that a
                                  // batch graph that captured their addresses can refuse to run
    // host-call staging
    void *dv = nullptr, *dkv = nullptr;
    int stage_rhs = 0;
    // anova_matvec_host: the copy in, the matvec and the copy out captured as one graph for the
    // buffers of the last call (rebuilt when they, nrhs or the workspace change)
    cudaGraphExec_t host_exec = nullptr;
    cudaStream_t host_cap = nullptr;   // private stream the graph is captured on
    const void *host_v = nullptr;
    void *host_kv = nullptr, *host_dv = nullptr;
    int host_nrhs = 0;
    uint64_t host_gen = 0;

    // optional per-stage CUDA-event timing (anova_plan_set_timing)
    struct StageEvt {
        int stage;
        cudaEvent_t a, b;
    };
    bool timing = false;
    std::vector<StageEvt> evts;
    std::vector<cudaEvent_t> evt_pool;
    int64_t launches = 0;          // kernels launched since the last timing reset
};

// A kept source half of the cross product: every window's convolved grid for fixed weights w.
struct anova_model {
    int device = 0, prec = 0, N = 0, m = 0, P = 0;
    std::vector<int> user_to_internal;
    std::vector<anova::WindowInfo> win;  // the source plan's windows (dw, ell, eta, grid_off used)
    long long grid_total = 0;
    void *grid = nullptr;                // T[grid_total]
};

namespace anova {
enum { STAGE_SPREAD = 0, STAGE_REDUCE = 1, STAGE_FFT = 2, STAGE_INTERP = 3, STAGE_SUM = 4, NUM_STAGES = 5 };
// Records a CUDA event on the plan's stream when timing is on; returns the event (or null).
cudaEvent_t stage_event(anova_plan *p);
void stage_record(anova_plan *p, int stage, cudaEvent_t a, cudaEvent_t b);
size_t elem_size(const anova_plan *p);
anova_status ensure_workspace(anova_plan *p, int nrhs);
// Runs the fast summation for `nrhs` columns (element type T). If only_window >= 0, only that
// internal window contributes. Defined per precision in matvec_f32.cu / matvec_f64.cu.
template <typename T>
anova_status run_matvec_t(anova_plan *p, const void *v, void *Kv, int nrhs, int only_window);
template <typename T>
anova_status run_spread_grid_t(anova_plan *p, int w, const void *v, void *grid);
template <typename T>
anova_status run_conv_grid_t(anova_plan *p, int w, const void *in, void *out);
template <typename T>
anova_status run_interp_grid_t(anova_plan *p, int w, const void *grid, void *f);
template <typename T>
anova_status run_cross_matvec_t(anova_plan *src, anova_plan *tgt, const void *w, void *f);
// Split matvec of a row-sharded product: the spread of v into every window's grid (grids:
// nrhs x grid_total, overwritten), and the rest of the product from summed grids.
template <typename T>
anova_status run_matvec_grids_t(anova_plan *p, const void *v, void *grids, int nrhs);
template <typename T>
anova_status run_matvec_from_grids_t(anova_plan *p, const void *grids, void *Kv, int nrhs);
// Source half into model->grid (allocated by the caller, grid_total elements); synchronises.
template <typename T>
anova_status run_model_create_t(anova_plan *src, const void *w, anova_model *model);
// Target half: interpolation at tgt's points from the model's grids, then the window sum.
template <typename T>
anova_status run_model_eval_t(const anova_model *model, anova_plan *tgt, void *f);
// How a plan cuts its work (the arithmetic of a point-window product does not depend on it):
// points per spread work item (kSegMax <= wi_max <= 1 << 16) and grid lines per CTA of an FFT
// pass (8, 16 or 32).
struct PlanShape {
    int wi_max = kWiMax;
    int conv_lines = kConvLines;
};
anova_status create_plan_shaped(const double *points, int64_t n, int d, const int32_t *windows, int P,
                                const double *ell, const double *eta, int N, int m, int flags, void *stream,
                                const PlanShape &shape, anova_plan_t *out);
void destroy_plan(anova_plan *p);
}  // namespace anova
