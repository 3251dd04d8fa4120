/*
 * ORACLE -- test infrastructure only. Plain FP64 CPU code; it shares nothing with the CUDA path.
 * Only tests/, __graft_entry__.smoke() and bench.py (its CPU-baseline leg) may load it.
 *
 * Direct ANOVA-kernel matrix-vector product, written as its definition
 * (Sec. 3, the entry (Kv)_j of the Gaussian-kernel product, and the extended Gaussian ANOVA
 * kernel with windows W_l and K v = K_1 v + ... + K_P v):
 *
 *     (K v)_j = sum_l eta_l sum_i v_i exp( - sum_{k in W_l} (x_{j,k} - x_{i,k})^2 / ell_l^2 ).
 *
 * O(n^2 P |W|) work, FP64 accumulation, OpenMP over output rows. Nothing is blocked, fused,
 * reordered or approximated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of OpenMP threads the oracle will use (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * X       : n x d, row-major, FP64.
 * windows : P x 3 feature indices (0-based), -1 pads windows of one or two features.
 * ell     : P kernel length scales (ell_l); eta : P window weights (NULL means all ones).
 * V       : n x nrhs, column-major (column r starts at V + r*n).
 * rows    : the output rows j to compute (NULL means all n rows, then nrows must equal n).
 * out     : nrows x nrhs, column-major (column r starts at out + r*nrows).
 */
void oracle_anova_matvec(const double *X, int64_t n, int d, const int32_t *windows, int P,
                         const double *ell, const double *eta, const double *V, int nrhs,
                         const int64_t *rows, int64_t nrows, double *out) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t jj = 0; jj < nrows; ++jj) {
        const int64_t j = rows ? rows[jj] : jj;
        double acc[64];
        for (int r = 0; r < nrhs && r < 64; ++r) acc[r] = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double kij = 0.0;
            for (int l = 0; l < P; ++l) {
                double dist2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const int k = windows[3 * l + c];
                    if (k < 0) continue;
                    const double diff = X[j * d + k] - X[i * d + k];
                    dist2 += diff * diff;
                }
                const double w = eta ? eta[l] : 1.0;
                kij += w * exp(-dist2 / (ell[l] * ell[l]));
            }
            for (int r = 0; r < nrhs && r < 64; ++r) acc[r] += kij * V[(int64_t)r * n + i];
        }
        for (int r = 0; r < nrhs && r < 64; ++r) out[(int64_t)r * nrows + jj] = acc[r];
    }
}

/* Dense ANOVA kernel matrix K (n x n, row-major), the same definition entry by entry. */
void oracle_anova_kernel_matrix(const double *X, int64_t n, int d, const int32_t *windows, int P,
                                const double *ell, const double *eta, double *K) {
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < n; ++i) {
            double kij = 0.0;
            for (int l = 0; l < P; ++l) {
                double dist2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const int k = windows[3 * l + c];
                    if (k < 0) continue;
                    const double diff = X[j * d + k] - X[i * d + k];
                    dist2 += diff * diff;
                }
                const double w = eta ? eta[l] : 1.0;
                kij += w * exp(-dist2 / (ell[l] * ell[l]));
            }
            K[j * n + i] = kij;
        }
    }
}
