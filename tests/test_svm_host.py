"""CPU-only checks of the solver ABI: Table 1 defaults (golden file) and argument validation."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ab():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_00538_gb300 as m
    return m


def test_defaults_follow_table1(ab):
    t = json.load(open(os.path.join(HERE, "golden", "table1_params.json")))
    o = ab.svm_opts_default()
    assert o.max_iter == t["iter_ip"]
    assert o.krylov_max == t["iter_krylov"]
    assert o.sigma_barrier == t["barrier_reduction_sigma"]
    assert o.gamma == t["step_factor_gamma"] == t["gamma0_algorithm1"]
    assert o.err_tol == t["cholesky_err_tol"]
    assert o.stop == ab.SVM_STOP_GAP
    assert (o.N, o.m, o.N_precise, o.m_precise) == (32, 4, 64, 6)
    assert o.m_refine == 4
    assert o.krylov == ab.SVM_KRYLOV_MINRES
    assert o.autotune == 0


@pytest.mark.parametrize("case", ["labels", "one_class", "C", "tol", "opts", "krylov", "autotune", "m_refine"])
def test_invalid_solver_arguments(ab, case):
    X = np.zeros((6, 3))
    y = np.array([1.0, -1.0, 1.0, -1.0, 1.0, -1.0])
    C, tol = 1.0, 1e-6
    o = ab.svm_opts_default()
    if case == "labels":
        y = y.copy()
        y[0] = 0.5
    if case == "one_class":
        y = np.ones(6)
    if case == "C":
        C = -1.0
    if case == "tol":
        tol = 0.0
    if case == "opts":
        o.sigma_barrier = 1.5
    if case == "krylov":
        o.krylov = 7
    if case == "autotune":
        o.autotune = 2
    if case == "m_refine":
        o.m_refine = 7
    with pytest.raises(ab.AnovaError) as ei:
        ab.svm_ipm_solve(X, y, C, tol, opts=o)
    assert ei.value.status == ab.ANOVA_ERR_INVALID_ARG


@pytest.mark.parametrize("case", ["slots0", "slots_big", "budget", "tol"])
def test_invalid_server_arguments(ab, case):
    slots, budget, tol = 2, 1 << 30, 1e-6
    if case == "slots0":
        slots = 0
    if case == "slots_big":
        slots = 1000
    if case == "budget":
        budget = 0
    if case == "tol":
        tol = -1.0
    with pytest.raises(ab.AnovaError) as ei:
        ab.SvmServer(tol, slots=slots, hbm_budget_bytes=budget)
    assert ei.value.status == ab.ANOVA_ERR_INVALID_ARG


def test_request_footprint(ab):
    """The admission estimate grows with n, the window count and the rank, and covers at least
    the FP64 + FP32 low-rank factor and the FP64 plan's grids."""
    o = ab.svm_opts_default()
    f = ab.svm_request_footprint
    assert f(0, 3, o) == 0 and f(100, 0, o) == 0
    assert f(10_000, 3, o) < f(20_000, 3, o) < f(20_000, 4, o)
    hi = ab.svm_opts_default()
    hi.rank = 400
    assert f(20_000, 3, o) < f(20_000, 3, hi)
    n, P, r = 50_000, 3, o.rank
    assert f(n, P, o) >= n * r * 12 + 8 * 4 * P * (2 * o.N_precise) ** 3
    # the refinement's own FP64 plan is counted when it differs from the precise plan
    one = ab.svm_opts_default()
    one.m_refine = 0
    assert f(n, P, one) < f(n, P, o)


def test_request_footprint_counts_transient_work(ab):
    """The randomised Nystrom factor holds K G and K Q (2 n r doubles) while it is built, and the
    autotuner holds a candidate FP64 plan beside the kept one: both raise the estimate."""
    o = ab.svm_opts_default()
    f = ab.svm_request_footprint
    n, P = 30_000, 3
    base = f(n, P, o)
    ny = ab.svm_opts_default()
    ny.precond = ab.NYSTROM_RANDOM
    assert f(n, P, ny) >= base + 2 * n * ny.rank * 8
    tu = ab.svm_opts_default()
    tu.autotune = 1
    assert f(n, P, tu) > base
