"""ORACLE -- test infrastructure only. The NFFT fast summation, step by step, in plain NumPy.

Sec. 3 replaces the Gaussian by a trigonometric polynomial of bandwidth N (N even),
    kappa~(t) = sum_{J in I_N} b_J exp(2 pi i J t),   I_N = {-N/2, ..., N/2 - 1},
and factors the matvec as an adjoint NFFT (inner sum), a diagonal scaling by b_J and an NFFT
(outer sum). The paper does not say how b_J are obtained, nor which NFFT window is used. The
readings taken here:

* b_J (reading C-4): the Gaussian is separable, so b_J = prod_k b_{J_k} with 1-D coefficients.
  The 1-D coefficients are the least-squares fit of an even cosine series
  b_0 + 2 sum_{k=1}^{N/2-1} b_k cos(2 pi k t) to exp(-t^2/ell^2) on |t| <= 1/2 - eps_B with
  eps_B = 0.1 (points lie in [-0.2, 0.2], so differences lie in [-0.4, 0.4]); b_{-N/2} = 0.
* window (reading C-5): oversampled grid of n_os = 2N points per dimension, Kaiser-Bessel window
  psi(t) = m sinh(beta sqrt(m^2 - t^2)) / (sqrt(m^2 - t^2) sinh(beta m)) for |t| <= m (t in grid
  units), beta = pi (2 - 1/2); 2m grid points per dimension. Grid point u (0 <= u < n_os) sits at
  u / n_os - 1/2. The deconvolution uses Psi(k) = int psi(t) cos(2 pi k t / n_os) dt.

The plain fast summation is then  f = sum_W interp_W( IDFT( D_W * DFT( spread_W(v) ) ) )  with
D_W = prod_k b_{J_k} / Psi(J_k)^2 on I_N^{d_W} and 0 elsewhere (unnormalised inverse DFT).
"""
import numpy as np

EPS_B = 0.1


# ---------------------------------------------------------------- trigonometric polynomial
def trig_coeffs(ell, N, radius=0.5 - EPS_B, samples=None):
    """1-D coefficients b_0..b_{N/2-1} of the even cosine fit to exp(-t^2/ell^2) on |t|<=radius.

    Least squares in FP64 on Chebyshev-distributed samples of [0, radius] (numpy lstsq)."""
    if N % 2:
        raise ValueError("bandwidth N must be even (Sec. 3: N in 2N)")
    K = N // 2
    M = samples or (4 * N + 64)
    t = radius * (1.0 - np.cos(np.pi * (np.arange(M) + 0.5) / M)) / 2.0
    A = np.cos(2.0 * np.pi * np.outer(t, np.arange(K)))
    A[:, 1:] *= 2.0
    f = np.exp(-t ** 2 / ell ** 2)
    b, *_ = np.linalg.lstsq(A, f, rcond=None)
    return b


def trig_coeffs_full(ell, N):
    """b_J for J in I_N (index J + N/2), with b_{-N/2} = 0 and b_{-J} = b_J."""
    b = trig_coeffs(ell, N)
    full = np.zeros(N)
    for J in range(-N // 2 + 1, N // 2):
        full[J + N // 2] = b[abs(J)]
    return full


def trig_poly_1d(t, ell, N):
    """kappa~_1(t) = sum_{J in I_N} b_J exp(2 pi i J t), real because b is even with b_{-N/2}=0."""
    bf = trig_coeffs_full(ell, N)
    J = np.arange(-N // 2, N // 2)
    return np.real(np.exp(2j * np.pi * np.outer(np.atleast_1d(t), J)) @ bf)


# ---------------------------------------------------------------- direct NDFTs
def _phases(x, N, sign):
    J = np.arange(-N // 2, N // 2)
    return np.exp(sign * 2j * np.pi * np.outer(x, J))


def ndft_adjoint(xw, v, N):
    """h_J = sum_i v_i exp(-2 pi i J . x_i), J in I_N^{d} (array axis k holds J_k + N/2)."""
    xw = np.asarray(xw, dtype=np.float64)
    if xw.ndim != 2:
        raise ValueError("xw must be (n, d_W)")
    n, dw = xw.shape
    E = [_phases(xw[:, k], N, -1.0) for k in range(dw)]
    v = np.asarray(v, dtype=np.complex128)
    if dw == 1:
        return v @ E[0]
    if dw == 2:
        return np.einsum("i,ia,ib->ab", v, E[0], E[1], optimize=True)
    return np.einsum("i,ia,ib,ic->abc", v, E[0], E[1], E[2], optimize=True)


def ndft_forward(xw, h, N):
    """f_j = sum_J h_J exp(2 pi i J . x_j)."""
    xw = np.asarray(xw, dtype=np.float64)
    if xw.ndim != 2 or xw.shape[1] != h.ndim:
        raise ValueError("xw must be (n, d_W) with d_W = h.ndim")
    n, dw = xw.shape
    E = [_phases(xw[:, k], N, +1.0) for k in range(dw)]
    if dw == 1:
        return E[0] @ h
    if dw == 2:
        return np.einsum("ia,ib,ab->i", E[0], E[1], h, optimize=True)
    return np.einsum("ia,ib,ic,abc->i", E[0], E[1], E[2], h, optimize=True)


def _outer(vecs):
    out = vecs[0]
    for w in vecs[1:]:
        out = np.multiply.outer(out, w)
    return out


def trig_poly_matvec(X, windows, ell, N, v):
    """sum_W sum_J b_J (sum_i v_i e^{-2 pi i J x_i}) e^{2 pi i J x_j}: the exact matvec with the
    trigonometric-polynomial kernel, through direct NDFTs (no window, no oversampled grid)."""
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros(X.shape[0])
    bf = trig_coeffs_full(ell, N)
    for W in np.asarray(windows).reshape(-1, 3):
        feats = [k for k in W if k >= 0]
        xw = X[:, feats]
        h = ndft_adjoint(xw, v, N)
        h = h * _outer([bf] * len(feats))
        out += np.real(ndft_forward(xw, h, N))
    return out


# ---------------------------------------------------------------- Kaiser-Bessel window
def kb_beta(oversampling=2.0):
    return np.pi * (2.0 - 1.0 / oversampling)


def kb_window(t, m, beta):
    """psi(t), normalised to psi(0) = 1; t in grid units, support |t| <= m."""
    t = np.asarray(t, dtype=np.float64)
    s2 = m * m - t * t
    out = np.zeros_like(t)
    scale = m / np.sinh(beta * m)
    pos = s2 > 0
    s = np.sqrt(s2[pos])
    out[pos] = np.sinh(beta * s) / s * scale
    out[s2 == 0] = beta * scale
    return out


def kb_hat(k, m, n_os, beta, nodes=256):
    """Psi(k) = int_{-m}^{m} psi(t) cos(2 pi k t / n_os) dt, Gauss-Legendre quadrature."""
    x, w = np.polynomial.legendre.leggauss(nodes)
    t = m * x
    w = m * w
    vals = kb_window(t, m, beta)
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    return (np.cos(2 * np.pi * np.outer(k, t) / n_os) * (w * vals)).sum(axis=1)


def kb_hat_closed_form(k, m, n_os, beta):
    """The textbook transform of the untruncated window: pi m / sinh(beta m) * I0(m sqrt(beta^2 -
    w^2)), w = 2 pi k / n_os < beta. Equal to kb_hat up to the truncated tail."""
    om = 2 * np.pi * np.asarray(k, dtype=np.float64) / n_os
    return np.pi * m / np.sinh(beta * m) * np.i0(m * np.sqrt(beta ** 2 - om ** 2))


def deconv_diag_1d(ell, N, m, n_os, beta):
    """D1[k] for FFT index k = 0..n_os-1 (frequency k or k - n_os): b_k / Psi(k)^2 on I_N, else 0."""
    bf = trig_coeffs_full(ell, N)
    D = np.zeros(n_os)
    for J in range(-N // 2, N // 2):
        D[J % n_os] = bf[J + N // 2] / kb_hat(J, m, n_os, beta)[0] ** 2
    return D


# ---------------------------------------------------------------- plain NFFT stages
def _footprint(s, m, n_os, beta):
    """Grid indices (mod n_os) and window weights of the 2m grid points around s (grid units)."""
    c = int(np.floor(s))
    u = np.arange(c - m + 1, c + m + 1)
    return u % n_os, kb_window(s - u, m, beta)


def spread_grid(xw, v, n_os, m, beta=None):
    """g[u] = sum_i v_i prod_k psi(s_{i,k} - u_k), s = (x + 1/2) n_os, on the periodic grid."""
    xw = np.asarray(xw, dtype=np.float64)
    beta = kb_beta() if beta is None else beta
    n, dw = xw.shape
    g = np.zeros((n_os,) * dw)
    for i in range(n):
        idx, wts = zip(*[_footprint((xw[i, k] + 0.5) * n_os, m, n_os, beta) for k in range(dw)])
        g[np.ix_(*idx)] += v[i] * _outer(list(wts))
    return g


def conv_grid(g, D1):
    """IDFT(D * DFT(g)) with the unnormalised inverse, D = tensor product of D1 over the axes.

    Array axis k of g is feature k of the window."""
    D = _outer([D1] * g.ndim)
    return np.real(np.fft.ifftn(np.fft.fftn(g) * D)) * g.size


def interp_grid(xw, g, n_os, m, beta=None):
    """f_i = sum_u g[u] prod_k psi(s_{i,k} - u_k)."""
    xw = np.asarray(xw, dtype=np.float64)
    beta = kb_beta() if beta is None else beta
    n, dw = xw.shape
    f = np.zeros(n)
    for i in range(n):
        idx, wts = zip(*[_footprint((xw[i, k] + 0.5) * n_os, m, n_os, beta) for k in range(dw)])
        f[i] = np.sum(g[np.ix_(*idx)] * _outer(list(wts)))
    return f


def nfft_fastsum(X, windows, ell, N, m, v, oversampling=2):
    """Plain NFFT fast summation of K v (windows summed, eta = 1)."""
    X = np.asarray(X, dtype=np.float64)
    n_os = int(oversampling * N)
    beta = kb_beta(oversampling)
    D1 = deconv_diag_1d(ell, N, m, n_os, beta)
    out = np.zeros(X.shape[0])
    for W in np.asarray(windows).reshape(-1, 3):
        feats = [k for k in W if k >= 0]
        xw = X[:, feats]
        g = spread_grid(xw, v, n_os, m, beta)
        out += interp_grid(xw, conv_grid(g, D1), n_os, m, beta)
    return out
