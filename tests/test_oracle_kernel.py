"""Pins of the direct ANOVA-kernel oracle against facts the paper and the mathematics fix.

Sec. 1: K is symmetric positive semi-definite. Sec. 3: each window kernel is a Gaussian of the
window's coordinates (K_l(x, x) = 1, coincident points give all-ones blocks, product over the
window's features) and K v = K_1 v + ... + K_P v.
"""
import numpy as np
import pytest

from oracle import kernel as ok
from synth import minmax_scale, consecutive_windows


def _pts(n, d, seed):
    rng = np.random.default_rng(seed)
    return minmax_scale(rng.standard_normal((n, d)))


def test_symmetry_bilinear():
    X = _pts(300, 7, 1)
    W = consecutive_windows(7)
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal(300), rng.standard_normal(300)
    Ku = ok.anova_matvec(X, W, 0.7, u)
    Kv = ok.anova_matvec(X, W, 0.7, v)
    assert abs(u @ Kv - v @ Ku) <= 1e-13 * np.abs(u) @ np.abs(Kv)


def test_psd():
    X = _pts(400, 6, 3)
    K = ok.anova_kernel_matrix(X, consecutive_windows(6), 0.5)
    assert np.allclose(K, K.T, rtol=0, atol=0)
    lam = np.linalg.eigvalsh(K)
    assert lam.min() >= -1e-12 * 400


def test_diagonal_is_P_and_coincident_points():
    X = _pts(50, 8, 4)
    W = consecutive_windows(8)       # P = 3 (3 + 3 + 2 features)
    K = ok.anova_kernel_matrix(X, W, 1.3)
    assert np.allclose(np.diag(K), 3.0, rtol=0, atol=1e-15)
    Xc = np.repeat(X[:1], 5, axis=0)
    Kc = ok.anova_kernel_matrix(Xc, W, 1.3)
    assert np.array_equal(Kc, np.full((5, 5), 3.0))


def test_separability_of_3d_window():
    X = _pts(40, 3, 5)
    K3 = ok.anova_kernel_matrix(X, np.array([[0, 1, 2]]), 0.8)
    prod = np.ones((40, 40))
    for k in range(3):
        prod *= ok.anova_kernel_matrix(X, np.array([[k, -1, -1]]), 0.8)
    assert np.allclose(K3, prod, rtol=1e-14, atol=0)


def test_sum_over_windows():
    X = _pts(60, 9, 6)
    W = consecutive_windows(9)
    rng = np.random.default_rng(7)
    v = rng.standard_normal(60)
    total = ok.anova_matvec(X, W, 1.1, v)
    parts = sum(ok.anova_matvec(X, W[l:l + 1], 1.1, v) for l in range(3))
    assert np.allclose(total, parts, rtol=1e-14, atol=1e-14)


def test_n1_and_n2_closed_forms():
    W = np.array([[0, 1, -1], [2, -1, -1]])
    x1 = np.array([[0.1, -0.05, 0.2]])
    assert ok.anova_matvec(x1, W, 0.9, np.array([2.5]))[0] == pytest.approx(2 * 2.5, rel=1e-15)
    X = np.array([[0.1, -0.05, 0.2], [-0.15, 0.05, 0.0]])
    ell = 0.9
    k01 = np.exp(-(0.25 ** 2 + 0.1 ** 2) / ell ** 2) + np.exp(-(0.2 ** 2) / ell ** 2)
    v = np.array([1.5, -2.0])
    expect = np.array([2 * 1.5 + k01 * -2.0, k01 * 1.5 + 2 * -2.0])
    assert np.allclose(ok.anova_matvec(X, W, ell, v), expect, rtol=1e-14, atol=0)


def test_rows_subset_and_multi_rhs():
    X = _pts(120, 6, 8)
    W = consecutive_windows(6)
    rng = np.random.default_rng(9)
    V = rng.standard_normal((120, 4))
    full = ok.anova_matvec(X, W, 0.6, V)
    rows = np.array([0, 17, 63, 119])
    sub = ok.anova_matvec(X, W, 0.6, V, rows=rows)
    assert np.array_equal(sub, full[rows])
    assert np.array_equal(ok.anova_matvec(X, W, 0.6, V[:, 2]), full[:, 2])


def test_matches_pairwise_loop():
    # a second, independent statement of one window's kernel: a NumPy loop over pairs
    X = _pts(80, 3, 10)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(80)
    Kl = ok.window_kernel_matrix(X, [0, 1, 2], 0.45)
    assert np.allclose(ok.anova_matvec(X, np.array([[0, 1, 2]]), 0.45, v), Kl @ v,
                       rtol=1e-13, atol=1e-13)


def test_cross_matvec_by_brute_force():
    """Targets distinct from sources: against a NumPy double loop over both sets; with the targets
    equal to the sources it is the square matvec."""
    rng = np.random.default_rng(77)
    Xs = rng.uniform(-0.2, 0.2, size=(30, 4))
    Xt = rng.uniform(-0.2, 0.2, size=(17, 4))
    W = np.array([[0, 1, -1], [2, 3, -1], [1, -1, -1]])
    w = rng.standard_normal(30)
    ref = np.zeros(17)
    for j in range(17):
        for i in range(30):
            for win in W:
                f = [k for k in win if k >= 0]
                ref[j] += w[i] * np.exp(-np.sum((Xt[j, f] - Xs[i, f]) ** 2) / 0.7 ** 2)
    got = ok.anova_cross_matvec(Xs, Xt, W, 0.7, w)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.allclose(ok.anova_cross_matvec(Xs, Xs, W, 0.7, w), ok.anova_matvec(Xs, W, 0.7, w),
                       rtol=1e-14, atol=1e-14)
