"""Pins of the dense IPM oracle (Algorithm 1, eq. (Newton)) against closed forms, brute-force
enumeration of the dual QP, the SVM optimality conditions and weak duality (Secs. 1-2)."""
import numpy as np
import pytest

from oracle import ipm as oi
from oracle import kernel as ok
from synth import minmax_scale, consecutive_windows, config1


def test_two_point_closed_form():
    X = np.array([[0.1, -0.05, 0.2], [-0.15, 0.05, 0.0]])
    W = np.array([[0, 1, 2]])
    K = ok.anova_kernel_matrix(X, W, 0.3)
    y = np.array([1.0, -1.0])
    for C in (0.5, 50.0):
        a_star = min(C, 2.0 / (K[0, 0] + K[1, 1] - 2 * K[0, 1]))
        res = oi.ipm_dense(K, y, C, tol=1e-12, max_iter=200)
        assert res["reason"] == "converged"
        assert np.allclose(res["alpha"], a_star, rtol=1e-8, atol=1e-9 * C)
        d_star = 2 * a_star - 0.5 * a_star ** 2 * (K[0, 0] + K[1, 1] - 2 * K[0, 1])
        assert oi.dual_objective(K, y, res["alpha"]) == pytest.approx(d_star, rel=1e-9)


@pytest.mark.parametrize("seed,C", [(1, 1.0), (2, 10.0), (3, 0.2)])
def test_matches_brute_force_enumeration(seed, C):
    rng = np.random.default_rng(seed)
    n = 7
    X = minmax_scale(rng.standard_normal((n, 4)))
    y = np.where(rng.standard_normal(n) >= 0, 1.0, -1.0)
    y[0], y[1] = 1.0, -1.0
    K = ok.anova_kernel_matrix(X, consecutive_windows(4), 0.25)
    best, _ = oi.brute_force_dual(K, y, C)
    res = oi.ipm_dense(K, y, C, tol=1e-12, max_iter=300)
    assert res["reason"] == "converged"
    assert oi.dual_objective(K, y, res["alpha"]) == pytest.approx(best, rel=1e-8, abs=1e-9)


def test_kkt_and_gap_at_solution_and_weak_duality_along_the_way():
    cfg = config1(n=300)
    K = ok.anova_kernel_matrix(cfg["X"], cfg["windows"], cfg["sigma"])
    y, C = cfg["y"], cfg["C"]
    gaps = []

    def rec(alpha, lam):
        gap = oi.duality_gap(K, y, alpha, -lam, C)
        slack = abs(lam) * abs(y @ alpha)
        gaps.append((gap, slack))

    res = oi.ipm_dense(K, y, C, tol=1e-9, max_iter=200, record=rec)
    assert res["reason"] == "converged"
    for gap, slack in gaps:
        assert gap >= -slack - 1e-10
    alpha, b = res["alpha"], res["b"]
    assert np.all(alpha > 0) and np.all(alpha < C)
    assert abs(y @ alpha) <= 1e-8 * C * len(y)
    assert oi.duality_gap(K, y, alpha, b, C) <= 1e-6 * max(1.0, abs(oi.dual_objective(K, y, alpha)))
    assert oi.kkt_violation(K, y, alpha, b, C, eps_bound=1e-6) <= 1e-3


def test_algorithm1_loop_test_stops_on_mu_and_infeasibilities():
    cfg = config1(n=120)
    K = ok.anova_kernel_matrix(cfg["X"], cfg["windows"], cfg["sigma"])
    # Table 1: tol_ip = 1e-1. (The relative xi_lambda plateaus near 1e-2 with a constant sigma = 0.6,
    # so the loop test cannot reach much smaller tolerances; the gap test is used for those.)
    res = oi.ipm_dense(K, cfg["y"], cfg["C"], tol=1e-1, stop="alg1", max_iter=50,
                       sigma_rule="constant")
    assert res["reason"] == "converged"
    assert res["mu"] <= 1e-1
    # mu is reduced by the constant factor 0.6 once per iteration from mu0 = 1
    assert res["mu"] == pytest.approx(0.6 ** res["iterations"], rel=1e-12)
    h = res["history"][-1]
    assert h["xi_alpha"] <= 1e-1 and h["xi_lambda"] <= 1e-1
    assert res["iterations"] >= 5      # 0.6^k <= 0.1 needs k >= 5


def test_newton_direction_solves_the_saddle_system():
    rng = np.random.default_rng(5)
    n = 12
    X = minmax_scale(rng.standard_normal((n, 3)))
    y = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    K = ok.anova_kernel_matrix(X, np.array([[0, 1, 2]]), 0.5)
    C, mu = 2.0, 0.3
    alpha = rng.uniform(0.1, 1.9, n)
    lam = 0.4
    Q = (y[:, None] * K) * y[None, :]
    r1, r2 = oi.newton_rhs(Q, y, alpha, lam, mu, C)
    # the optimality conditions of the barrier Lagrangian (Sec. 2) written out entry by entry
    for j in range(n):
        expect = 1 - sum(Q[j, i] * alpha[i] for i in range(n)) + lam * y[j] + mu / alpha[j] \
            - mu / (C - alpha[j])
        assert r1[j] == pytest.approx(expect, rel=1e-12, abs=1e-12)
    assert r2 == pytest.approx(sum(y * alpha), rel=1e-14)


def test_step_to_boundary():
    a = np.array([0.5, 0.5, 0.5])
    assert oi.step_to_boundary(a, np.array([-1.0, 0.0, 0.0]), 1.0) == pytest.approx(0.5)
    assert oi.step_to_boundary(a, np.array([0.0, 2.0, 0.0]), 1.0) == pytest.approx(0.25)
    assert oi.step_to_boundary(a, np.array([0.1, -0.1, 0.0]), 1.0) == 1.0


@pytest.mark.parametrize("C", [10.0, 100.0])
def test_adaptive_barrier_converges_for_large_C(C):
    """Sec. 2 allows a sigma_it that changes every iteration; with it the method reaches the
    optimum for large C, where the constant rule stalls at the boundary."""
    rng = np.random.default_rng(int(C))
    n = 8
    X = minmax_scale(rng.standard_normal((n, 3)))
    y = np.array([1.0, -1.0, 1.0, 1.0, -1.0, -1.0, 1.0, -1.0])
    K = ok.anova_kernel_matrix(X, consecutive_windows(3), 0.3)
    best, _ = oi.brute_force_dual(K, y, C)
    res = oi.ipm_dense(K, y, C, tol=1e-12, max_iter=300)
    assert res["reason"] == "converged"
    assert oi.dual_objective(K, y, res["alpha"]) == pytest.approx(best, rel=1e-8, abs=1e-9)


def test_adaptive_rule_equals_constant_rule_with_full_steps():
    # workload-1-like data at C = 1: every step is a full step after the first two, so both
    # rules reduce mu by 0.6 there and reach the same optimum
    cfg = config1(n=150)
    K = ok.anova_kernel_matrix(cfg["X"], cfg["windows"], cfg["sigma"])
    a = oi.ipm_dense(K, cfg["y"], 1.0, tol=1e-9, max_iter=200, sigma_rule="constant")
    b = oi.ipm_dense(K, cfg["y"], 1.0, tol=1e-9, max_iter=200)
    da = oi.dual_objective(K, cfg["y"], a["alpha"])
    db = oi.dual_objective(K, cfg["y"], b["alpha"])
    assert da == pytest.approx(db, rel=1e-7)
