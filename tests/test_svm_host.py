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


@pytest.mark.parametrize("case", ["labels", "one_class", "C", "tol", "opts"])
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
    with pytest.raises(ab.AnovaError) as ei:
        ab.svm_ipm_solve(X, y, C, tol, opts=o)
    assert ei.value.status == ab.ANOVA_ERR_INVALID_ARG
