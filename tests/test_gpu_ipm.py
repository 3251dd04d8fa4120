"""The device interior point method (Algorithm 1) against the dense-KKT FP64 oracle.

Bar: the dual objective within 1e-6 relative of the oracle's optimum; the dual objective of both
iterates is evaluated by the oracle with the exact kernel matrix."""
import numpy as np
import pytest

from oracle import ipm as oi
from oracle import kernel as ok
from synth import config1, small_problem

from ._gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _solve(ab, X, y, W, C, tol, ell=1.0, rank=200, krylov_tol=1e-8):
    o = ab.svm_opts_default()
    o.ell = ell
    o.rank = rank
    o.krylov_tol = krylov_tol
    o.max_iter = 100
    return ab.svm_ipm_solve(X, y, C, tol, opts=o, windows=W)


def test_small_problem_matches_dense_oracle(env):
    torch, ab = env
    cfg = small_problem(200, 6, seed=7)
    X, y, W = cfg["X"], cfg["y"], cfg["windows"]
    C = 1.0
    alpha, b, st, status = _solve(ab, X, y, W, C, 1e-8, rank=50)
    assert status == ab.ANOVA_OK and st["converged"] == 1
    K = ok.anova_kernel_matrix(X, W, 1.0)
    ref = oi.ipm_dense(K, y, C, tol=1e-10, max_iter=200)
    d_gpu = oi.dual_objective(K, y, alpha)
    d_ref = oi.dual_objective(K, y, ref["alpha"])
    assert abs(d_gpu - d_ref) <= 1e-6 * abs(d_ref)
    assert np.all(alpha > 0) and np.all(alpha < C)
    assert abs(y @ alpha) <= 1e-6 * C * len(y)
    assert oi.duality_gap(K, y, alpha, b, C) <= 1e-6 * max(1.0, abs(d_ref))


def test_config1_dual_objective(env):
    """Workload 1: n = 2000, windows {0,1,2},{3,4,5}, sigma = 1, C = 1, gap 1e-6, MINRES 1e-8."""
    torch, ab = env
    cfg = config1()
    X, y, W, C = cfg["X"], cfg["y"], cfg["windows"], cfg["C"]
    alpha, b, st, status = _solve(ab, X, y, W, C, 1e-6, rank=200)
    assert status == ab.ANOVA_OK
    assert st["rel_gap"] <= 1e-6
    K = ok.anova_kernel_matrix(X, W, cfg["sigma"])
    ref = oi.ipm_dense(K, y, C, tol=1e-9, max_iter=200)
    d_gpu = oi.dual_objective(K, y, alpha)
    d_ref = oi.dual_objective(K, y, ref["alpha"])
    assert abs(d_gpu - d_ref) <= 1e-6 * abs(d_ref)
    # the solver's own FP64-plan objective agrees with the exact one
    assert abs(st["dual"] - d_gpu) <= 1e-8 * abs(d_gpu)
    assert oi.kkt_violation(K, y, alpha, b, C, eps_bound=1e-4) <= 5e-2


@pytest.mark.parametrize("C", [10.0, 100.0])
def test_large_C_workload3_like(env, C):
    """Workload-3-like data (Gaussian + binary features, tanh teacher, 5 % flips) at large C,
    where the barrier factor has to adapt to short steps (Sec. 2, sigma_it)."""
    torch, ab = env
    from synth import config3
    cfg = config3(n=1500)
    X, y, W = cfg["X"], cfg["y"], cfg["windows"]
    alpha, b, st, status = _solve(ab, X, y, W, C, 1e-6, rank=100, krylov_tol=1e-8)
    assert status == ab.ANOVA_OK, st
    K = ok.anova_kernel_matrix(X, W, 1.0)
    ref = oi.ipm_dense(K, y, C, tol=1e-9, max_iter=300)
    d_gpu = oi.dual_objective(K, y, alpha)
    d_ref = oi.dual_objective(K, y, ref["alpha"])
    assert abs(d_gpu - d_ref) <= 1e-6 * abs(d_ref)


@pytest.mark.parametrize("kind", ["random", "nystrom", "gmres", "per_window", "nystrom_random", "autotune"])
def test_other_preconditioners_reach_the_same_optimum(env, kind):
    """The optimum does not depend on the preconditioner or the Krylov method: randomly pivoted
    Cholesky, Nystrom (pivot set or orth(K G)), per-window stacked factors, and GMRES with the
    paper's block-triangular preconditioner (Sec. 5) reach the dense-KKT oracle's dual objective
    on workload 1 (only iteration counts differ); so do autotuned plans."""
    torch, ab = env
    cfg = config1()
    X, y, W, C = cfg["X"], cfg["y"], cfg["windows"], cfg["C"]
    o = ab.svm_opts_default()
    o.rank = 200
    o.krylov_tol = 1e-8
    o.max_iter = 100
    o.precond = {"random": ab.PCHOL_RANDOM, "nystrom": ab.NYSTROM, "gmres": ab.PCHOL_GREEDY,
                 "per_window": ab.PCHOL_PER_WINDOW, "nystrom_random": ab.NYSTROM_RANDOM,
                 "autotune": ab.PCHOL_GREEDY}[kind]
    o.autotune = 1 if kind == "autotune" else 0
    o.krylov = ab.SVM_KRYLOV_GMRES if kind == "gmres" else ab.SVM_KRYLOV_MINRES
    o.seed = 2023
    alpha, b, st, status = ab.svm_ipm_solve(X, y, C, 1e-6, opts=o, windows=W)
    assert status == ab.ANOVA_OK
    K = ok.anova_kernel_matrix(X, W, cfg["sigma"])
    ref = oi.ipm_dense(K, y, C, tol=1e-9, max_iter=200)
    d_ref = oi.dual_objective(K, y, ref["alpha"])
    assert abs(oi.dual_objective(K, y, alpha) - d_ref) <= 1e-6 * abs(d_ref)


def test_gmres_large_C(env):
    """GMRES with the block-triangular preconditioner on the harder C = 100 case."""
    torch, ab = env
    cfg = small_problem(400, 6, seed=11)
    X, y, W = cfg["X"], cfg["y"], cfg["windows"]
    o = ab.svm_opts_default()
    o.rank = 100
    o.max_iter = 150
    o.krylov = ab.SVM_KRYLOV_GMRES
    alpha, b, st, status = ab.svm_ipm_solve(X, y, 100.0, 1e-7, opts=o, windows=W)
    assert status == ab.ANOVA_OK
    K = ok.anova_kernel_matrix(X, W, 1.0)
    ref = oi.ipm_dense(K, y, 100.0, tol=1e-10, max_iter=400)
    d_ref = oi.dual_objective(K, y, ref["alpha"])
    assert abs(oi.dual_objective(K, y, alpha) - d_ref) <= 1e-6 * abs(d_ref)
