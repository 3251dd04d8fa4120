"""Pins of the oracle's NFFT pieces (Sec. 3, fast summation) against closed forms, textbook
transforms, library FFTs on equispaced nodes, and the direct kernel sum."""
import numpy as np
import pytest

from oracle import nfft as on
from oracle import kernel as ok
from synth import minmax_scale, consecutive_windows


@pytest.mark.parametrize("N,ell,bound", [(32, 0.5, 3e-7), (32, 1.0, 2e-7), (32, 2.0, 1e-7),
                                         (64, 0.5, 1e-11), (64, 1.0, 1e-11)])
def test_trig_polynomial_reproduces_gaussian(N, ell, bound):
    t = np.linspace(-0.4, 0.4, 4001)
    err = np.max(np.abs(on.trig_poly_1d(t, ell, N) - np.exp(-t ** 2 / ell ** 2)))
    assert err <= bound


def test_trig_coefficients_rejects_odd_bandwidth():
    with pytest.raises(ValueError):
        on.trig_coeffs(1.0, 31)


@pytest.mark.parametrize("m,rel", [(4, 2e-6), (6, 1e-9)])
def test_window_transform_matches_bessel_closed_form(m, rel):
    n_os, beta = 64, on.kb_beta(2.0)
    k = np.arange(-16, 16)
    q = on.kb_hat(k, m, n_os, beta)
    c = on.kb_hat_closed_form(k, m, n_os, beta)
    assert np.max(np.abs(q - c) / c) <= rel


def test_ndft_on_equispaced_nodes_is_fft():
    N = 16
    rng = np.random.default_rng(1)
    v = rng.standard_normal(N)
    x = (np.arange(N) / N - 0.5)[:, None]
    h = on.ndft_adjoint(x, v, N)
    J = np.arange(-N // 2, N // 2)
    expect = (-1.0) ** J * np.fft.fft(v)[J % N]
    assert np.allclose(h, expect, rtol=0, atol=1e-12)


def test_ndft_forward_is_adjoint_of_adjoint():
    rng = np.random.default_rng(2)
    x = rng.uniform(-0.2, 0.2, size=(30, 2))
    v = rng.standard_normal(30)
    h = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    lhs = np.vdot(on.ndft_adjoint(x, v, 8), h)            # <A^H v, h>
    rhs = np.vdot(v, on.ndft_forward(x, h, 8))             # <v, A h>
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_single_point_adjoint_closed_form():
    x = np.array([[0.125, -0.0625]])
    h = on.ndft_adjoint(x, np.array([2.0]), 8)
    J = np.arange(-4, 4)
    expect = 2.0 * np.multiply.outer(np.exp(-2j * np.pi * J * 0.125), np.exp(2j * np.pi * J * 0.0625))
    assert np.allclose(h, expect, atol=1e-14)


def test_spread_and_deconvolve_approximates_adjoint_ndft():
    # sum_u g[u] e^{-2 pi i J y_u} / Psi(J) ~ h_J, up to the window's aliasing error
    rng = np.random.default_rng(3)
    N, m, n_os = 16, 4, 32
    beta = on.kb_beta(2.0)
    x = rng.uniform(-0.2, 0.2, size=(25, 2))
    v = rng.standard_normal(25)
    g = on.spread_grid(x, v, n_os, m, beta)
    J = np.arange(-N // 2, N // 2)
    G = np.fft.fftn(g)
    sh = (-1.0) ** J
    Psi = on.kb_hat(J, m, n_os, beta)
    approx = np.outer(sh / Psi, sh / Psi) * G[np.ix_(J % n_os, J % n_os)]
    exact = on.ndft_adjoint(x, v, N)
    assert np.max(np.abs(approx - exact)) <= 1e-5 * np.max(np.abs(exact))


def _data(n, d, seed):
    rng = np.random.default_rng(seed)
    return minmax_scale(rng.standard_normal((n, d))), rng.standard_normal(n)


def test_trig_poly_matvec_close_to_direct_sum():
    X, v = _data(150, 6, 4)
    W = consecutive_windows(6)
    exact = ok.anova_matvec(X, W, 1.0, v)
    tp = on.trig_poly_matvec(X, W, 1.0, 32, v)
    assert np.linalg.norm(tp - exact) <= 1e-6 * np.linalg.norm(exact)


@pytest.mark.parametrize("ell", [0.5, 1.0])
def test_nfft_fastsum_close_to_trig_poly_and_direct(ell):
    X, v = _data(120, 3, 5)
    W = np.array([[0, 1, 2]])
    fs = on.nfft_fastsum(X, W, ell, 32, 4, v)
    tp = on.trig_poly_matvec(X, W, ell, 32, v)
    ex = ok.anova_matvec(X, W, ell, v)
    assert np.linalg.norm(fs - tp) <= 2e-6 * np.linalg.norm(tp)
    assert np.linalg.norm(fs - ex) <= 3e-6 * np.linalg.norm(ex)


def test_nfft_fastsum_precise_parameters():
    X, v = _data(60, 2, 6)
    W = np.array([[0, 1, -1]])
    fs = on.nfft_fastsum(X, W, 1.0, 64, 6, v)
    ex = ok.anova_matvec(X, W, 1.0, v)
    assert np.linalg.norm(fs - ex) <= 1e-10 * np.linalg.norm(ex)


def test_conv_grid_of_delta_is_kernel_samples():
    # a unit impulse at the grid centre convolved with D gives sum_J D_J e^{2 pi i J (u - c)/n_os}
    n_os, N, m = 32, 16, 4
    D1 = on.deconv_diag_1d(1.0, N, m, n_os, on.kb_beta())
    g = np.zeros(n_os)
    g[n_os // 2] = 1.0
    out = on.conv_grid(g, D1)
    k = np.fft.fftfreq(n_os, 1.0 / n_os)
    u = np.arange(n_os) - n_os // 2
    expect = np.real(np.exp(2j * np.pi * np.outer(u, k) / n_os) @ D1)
    assert np.allclose(out, expect, atol=1e-12)
