// Host-side FP64 plan mathematics of the NFFT fast summation (arXiv 2312.00538, Sec. 3).
//
//  * kernel_coeffs : the 1-D Fourier coefficients b_k of the trigonometric polynomial that
//    replaces the Gaussian (Sec. 3, kappa~ of bandwidth N). The paper does not say how b_k are
//    obtained; here they are the least-squares fit of an even cosine series to exp(-t^2/ell^2)
//    on |t| <= 1/2 - eps_B, eps_B = 0.1 (points in [-0.2, 0.2] give differences in [-0.4, 0.4]).
//    The 3-D coefficients are products of these (the Gaussian is separable).
//  * window_hat    : Psi(k), the Fourier transform of the normalised Kaiser-Bessel window that
//    spreads points onto the oversampled grid, by Gauss-Legendre quadrature of the truncated
//    window actually used (the NFFT's deconvolution factors).
//  * window_poly   : per grid offset j, a polynomial in z = 2f - 1 (f = fractional cell offset)
//    that reproduces psi(f + m - 1 - j); evaluated with Horner's rule in the FP32 kernels.
#include "anova_internal.h"

#include <cmath>
#include <vector>

namespace anova {

namespace {

// Least squares min ||A x - f|| by Householder QR (A is rows x cols, column-major, rows >= cols).
bool lstsq_householder(std::vector<double> A, int rows, int cols, std::vector<double> f,
                       std::vector<double> &x) {
    std::vector<double> diag(cols);
    for (int k = 0; k < cols; ++k) {
        double *a = &A[(size_t)k * rows];
        double norm = 0.0;
        for (int i = k; i < rows; ++i) norm += a[i] * a[i];
        norm = std::sqrt(norm);
        if (norm == 0.0) return false;
        const double alpha = a[k] > 0 ? -norm : norm;
        // v = a_k:rows - alpha e_k, stored in place
        a[k] -= alpha;
        double vnorm2 = 0.0;
        for (int i = k; i < rows; ++i) vnorm2 += a[i] * a[i];
        diag[k] = alpha;
        if (vnorm2 == 0.0) continue;
        for (int j = k + 1; j < cols; ++j) {
            double *c = &A[(size_t)j * rows];
            double s = 0.0;
            for (int i = k; i < rows; ++i) s += a[i] * c[i];
            s = 2.0 * s / vnorm2;
            for (int i = k; i < rows; ++i) c[i] -= s * a[i];
        }
        double s = 0.0;
        for (int i = k; i < rows; ++i) s += a[i] * f[i];
        s = 2.0 * s / vnorm2;
        for (int i = k; i < rows; ++i) f[i] -= s * a[i];
    }
    x.assign(cols, 0.0);
    for (int k = cols - 1; k >= 0; --k) {
        double s = f[k];
        for (int j = k + 1; j < cols; ++j) s -= A[(size_t)j * rows + k] * x[j];
        if (diag[k] == 0.0) return false;
        x[k] = s / diag[k];
    }
    return true;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_q.
void gauss_legendre(int q, std::vector<double> &x, std::vector<double> &w) {
    x.resize(q);
    w.resize(q);
    for (int i = 0; i < (q + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_q(z), p0 = P_{q-1}(z)
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        x[q - 1 - i] = z;
        w[i] = w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace

double kb_beta() { return M_PI * (2.0 - 1.0 / kOversampling); }

double kb_window(double t, int m) {
    const double beta = kb_beta();
    const double s2 = (double)m * m - t * t;
    const double scale = m / std::sinh(beta * m);
    if (s2 < 0.0) return 0.0;
    const double s = std::sqrt(s2);
    if (s < 1e-4) {
        // sinh(beta s)/s = beta (1 + (beta s)^2/6 + (beta s)^4/120 + ...)
        const double bs2 = beta * beta * s2;
        return beta * (1.0 + bs2 / 6.0 + bs2 * bs2 / 120.0) * scale;
    }
    return std::sinh(beta * s) / s * scale;
}

bool kernel_coeffs(double ell, int N, std::vector<double> &b) {
    if (N < 2 || (N & 1) || !(ell > 0.0) || !std::isfinite(ell)) return false;
    const int K = N / 2;
    const int M = 4 * N + 64;
    const double R = 0.5 - kEpsB;
    std::vector<double> A((size_t)M * K), f(M);
    for (int i = 0; i < M; ++i) {
        const double t = R * (1.0 - std::cos(M_PI * (i + 0.5) / M)) / 2.0;
        for (int k = 0; k < K; ++k)
            A[(size_t)k * M + i] = (k == 0 ? 1.0 : 2.0) * std::cos(2.0 * M_PI * k * t);
        f[i] = std::exp(-t * t / (ell * ell));
    }
    return lstsq_householder(A, M, K, f, b);
}

void window_hat(int m, int n_os, int count, double *Psi) {
    std::vector<double> x, w;
    gauss_legendre(256, x, w);
    for (int k = 0; k < count; ++k) {
        double s = 0.0;
        for (size_t q = 0; q < x.size(); ++q) {
            const double t = m * x[q];
            s += m * w[q] * kb_window(t, m) * std::cos(2.0 * M_PI * k * t / n_os);
        }
        Psi[k] = s;
    }
}

bool window_poly(int m, int deg, std::vector<double> &coef) {
    // coef[j * (deg + 1) + p]: psi(f + m - 1 - j) ~ sum_p coef z^p, z = 2f - 1, j = 0..2m-1
    const int S = 4 * (deg + 1) + 32;
    coef.assign((size_t)2 * m * (deg + 1), 0.0);
    for (int j = 0; j < 2 * m; ++j) {
        std::vector<double> A((size_t)S * (deg + 1)), f(S), c;
        for (int i = 0; i < S; ++i) {
            const double z = std::cos(M_PI * (i + 0.5) / S);
            const double fr = 0.5 * (z + 1.0);
            double zp = 1.0;
            for (int p = 0; p <= deg; ++p) {
                A[(size_t)p * S + i] = zp;
                zp *= z;
            }
            f[i] = kb_window(fr + m - 1 - j, m);
        }
        if (!lstsq_householder(A, S, deg + 1, f, c)) return false;
        for (int p = 0; p <= deg; ++p) coef[(size_t)j * (deg + 1) + p] = c[p];
    }
    return true;
}

bool deconv_diag(double ell, int N, int m, int n_os, std::vector<double> &D1) {
    std::vector<double> b;
    if (!kernel_coeffs(ell, N, b)) return false;
    std::vector<double> Psi(N / 2 + 1);
    window_hat(m, n_os, N / 2 + 1, Psi.data());
    D1.assign(n_os, 0.0);
    for (int J = -N / 2 + 1; J < N / 2; ++J) {
        const int a = J < 0 ? -J : J;
        D1[(J + n_os) % n_os] = b[a] / (Psi[a] * Psi[a]);
    }
    // J = -N/2 keeps D = 0 (b_{-N/2} = 0), as do all J outside I_N
    return true;
}

}  // namespace anova
