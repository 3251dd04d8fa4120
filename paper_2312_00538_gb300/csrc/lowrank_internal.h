// Internal layout of a low-rank preconditioner (not part of the C ABI).
#pragma once

#include <vector>

#include "anova_internal.h"

struct lowrank {
    anova_plan *plan = nullptr;  // not owned: the plan must outlive the preconditioner
    int kind = 0, rmax = 0, rank = 0;
    long long n = 0;
    std::vector<long long> piv;  // pivots in the order chosen
    double *L64 = nullptr;       // n x rmax, column-major, FP64 factor (K ~ L L^T)
    float *L32 = nullptr;        // n x rank, column-major FP32 panel used by the Woodbury steps
    double *d = nullptr;         // residual diagonal during the build
    void *piv_dev = nullptr;     // long long[rmax + 1]
    double *dpiv = nullptr;
    int *stop = nullptr;
    void *partial = nullptr;
    // Woodbury core
    double *M = nullptr;         // rank x rank, Cholesky factor after set_theta
    double *Wl = nullptr, *Wc = nullptr;  // its inverse W (lower): row-major and column-major
    double *itheta = nullptr;    // 1 / theta of the last set_theta (n)
    double *hbuf = nullptr;      // y .* g ./ theta of the current apply (n)
    double *tmp2 = nullptr;      // W u (rank)
    double *dinv = nullptr;      // reciprocals of the Cholesky factor's diagonal (rank)
    int core_rows = 0;           // rows per chunk of the core's partial Gram tiles
    double *u = nullptr, *upart = nullptr, *z = nullptr;
    void *tiles = nullptr;
    double *cpart = nullptr;
    int *info = nullptr;
    double *tmp = nullptr, *dpart = nullptr, *schur = nullptr;
    int ntiles = 0, nchunks = 0, napply = 0;
    double schur_host = 0.0;
    bool core_ready = false;
    double *Mcore = nullptr;     // the core M of the last set_theta before its factorisation (r x r)
    int core_path = 0;           // LOWRANK_CORE_AUTO / _SIMT / _TENSOR
    int core_used = 0;           // the path the last set_theta took (LOWRANK_CORE_SIMT / _TENSOR)
    // tensor-core core (csrc/core_tc.cu): integer slices of Theta^{-1/2} L, the per-row scales
    // Theta^{-1/2}, per-column maxima (double bits), exact integer accumulators of the slice
    // products, the CTA work list, an error word
    void *tc_Q = nullptr;
    double *tc_I = nullptr;
    double *tc_srow = nullptr;
    float *tc_srow32 = nullptr;
    unsigned *tc_cmax = nullptr;
    void *tc_work = nullptr;
    int *tc_status = nullptr;
    long long tc_np = 0;
    int tc_RP = 0, tc_nwork = 0;
};

namespace anova {
anova_status lowrank_build_impl(anova_plan *p, int kind, int r, double err_tol, uint64_t seed, lowrank **out);
anova_status lowrank_set_theta_impl(lowrank *lr, const double *theta, const double *y);
anova_status lowrank_apply_impl(lowrank *lr, const double *theta, const double *y, const double *g, double *x);
anova_status woodbury_apply(lowrank *lr, const double *theta, const double *y, const double *g, double *x,
                            bool with_schur);
void lowrank_release(lowrank *lr);
bool core_tc_supported(const lowrank *lr);
anova_status core_tc(lowrank *lr);
}  // namespace anova
