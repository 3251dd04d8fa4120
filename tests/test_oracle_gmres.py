"""Pins of the GMRES oracle (Sec. 5): exact convergence, the residual it reports is the true
residual, the two-step convergence that the paper's preconditioner gives with the exact (1,1)
block, agreement with SciPy's GMRES, and the triangular apply against a dense solve."""
import numpy as np
import pytest

from oracle import gmres as og
from oracle import kernel as ok
from oracle import precond as op


def test_converges_to_the_solution_within_n_steps():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((25, 25)) + 2.0 * np.eye(25)
    b = rng.standard_normal(25)
    x, info = og.gmres(lambda v: A @ v, b, rtol=1e-13, max_iter=25)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
    assert info["iterations"] <= 25


def test_reported_residual_is_the_true_residual_and_never_grows():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((40, 40)) + 6.0 * np.eye(40)
    b = rng.standard_normal(40)
    D = np.diag(rng.uniform(0.5, 2.0, 40))                  # a right preconditioner P = D
    x, info = og.gmres(lambda v: A @ v, b, apply_Pinv=lambda r: np.linalg.solve(D, r), rtol=1e-6,
                       max_iter=40)
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-12 * h[0])
    assert abs(np.linalg.norm(b - A @ x) - info["resid"]) <= 1e-10 * np.linalg.norm(b)


def test_exact_block_gives_two_steps():
    """With A^ = A exactly, A P^{-1} has n unit eigenvalues and one more: two GMRES steps."""
    rng = np.random.default_rng(5)
    X = rng.uniform(-0.2, 0.2, size=(60, 3))
    K = ok.anova_kernel_matrix(X, np.array([[0, 1, 2]]), 0.5)
    y = np.where(rng.standard_normal(60) > 0, 1.0, -1.0)
    theta = rng.uniform(0.1, 2.0, 60)
    S = op.saddle_matrix(K, theta, y)
    A11 = S[:60, :60]
    b = rng.standard_normal(61)
    x, info = og.gmres(lambda v: S @ v, b,
                       apply_Pinv=lambda g: og.triangular_apply(lambda r: np.linalg.solve(A11, r), y, g),
                       rtol=1e-10, max_iter=20)
    assert info["iterations"] <= 2
    assert np.linalg.norm(S @ x - b) <= 1e-9 * np.linalg.norm(b)


def test_triangular_apply_is_the_inverse_of_P():
    rng = np.random.default_rng(6)
    n = 12
    Ah = rng.standard_normal((n, n)) + 4 * np.eye(n)
    y = np.where(rng.standard_normal(n) > 0, 1.0, -1.0)
    P = op.triangular_preconditioner(Ah, y)
    g = rng.standard_normal(n + 1)
    assert np.allclose(og.triangular_apply(lambda r: np.linalg.solve(Ah, r), y, g), np.linalg.solve(P, g),
                       rtol=1e-12, atol=1e-12)


def test_agrees_with_scipy_gmres():
    sla = pytest.importorskip("scipy.sparse.linalg")
    rng = np.random.default_rng(7)
    A = rng.standard_normal((30, 30)) + 5.0 * np.eye(30)
    b = rng.standard_normal(30)
    x, _ = og.gmres(lambda v: A @ v, b, rtol=1e-12, max_iter=30)
    xs, code = sla.gmres(A, b, rtol=1e-12, restart=30, maxiter=30)
    assert code == 0
    assert np.allclose(x, xs, rtol=1e-8, atol=1e-10)
