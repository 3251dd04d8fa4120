"""CPU-only checks of the solver ABI: Table 1 defaults (golden file) and argument validation."""
import ctypes
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


def test_admission_rule_cases(ab):
    """The workers' admission rule: the oldest request when it fits (or nothing runs), else the
    oldest younger request that fits, until the oldest has been passed four times."""
    f = ab.svm_server_admission
    assert f([], [], 0, 100, 0) == -1                       # empty queue
    assert f([60, 10], [0, 0], 30, 100, 1) == 0             # the oldest fits: FIFO
    assert f([70, 10], [0, 0], 30, 100, 1) == 0             # exactly at the budget still fits
    assert f([80, 10], [0, 0], 30, 100, 1) == 1             # backfill past the oldest
    assert f([80, 90, 20, 10], [0, 0, 0, 0], 30, 100, 2) == 2   # the oldest younger that fits, not the smallest
    assert f([80, 90, 75], [0, 0, 0], 30, 100, 1) == -1     # nothing fits
    assert f([500, 10], [0, 0], 0, 100, 0) == 0             # larger than the budget: runs alone when idle
    assert f([500, 10], [0, 0], 30, 100, 1) == 1
    assert f([80, 10], [3, 0], 30, 100, 1) == 1             # passed 3 times: one more backfill
    assert f([80, 10], [4, 0], 30, 100, 1) == -1            # passed 4 times: the rest waits for it
    assert f([80, 10], [4, 0], 30, 100, 0) == 0
    with pytest.raises(ValueError):
        f([1, 2], [0], 0, 10, 0)
    L = ab.lib()
    pick = ctypes.c_int(7)
    assert L.svm_server_admission(None, None, -1, 0, 10, 0, ctypes.byref(pick)) == ab.ANOVA_ERR_INVALID_ARG
    assert pick.value == -1
    assert L.svm_server_admission(None, None, 2, 0, 10, 0, ctypes.byref(pick)) == ab.ANOVA_ERR_INVALID_ARG
    assert L.svm_server_admission(None, None, 0, 0, 10, 0, None) == ab.ANOVA_ERR_INVALID_ARG


def test_admission_schedule_replay(ab):
    """A replayed schedule (one slot per request up to four, unit-time steps): every request
    starts, memory never exceeds the budget except for a request that runs alone, and no request
    is passed more than four times. Checked against a plain restatement of the rule."""
    rng = np.random.default_rng(2312)
    budget, slots = 100, 4

    def rule(fp, ps, reserved, running):
        if not fp:
            return -1
        if reserved + fp[0] <= budget or running == 0:
            return 0
        if ps[0] >= 4:
            return -1
        for k in range(1, len(fp)):
            if reserved + fp[k] <= budget:
                return k
        return -1

    backfills, capped = 0, 0
    for trial in range(20):
        reqs = [(int(rng.integers(5, 130)), int(rng.integers(1, 6))) for _ in range(40)]
        queue, running, t, started, max_passed = [], [], 0, 0, 0
        arrivals = sorted(int(a) for a in rng.integers(0, 60, size=len(reqs)))
        nxt = 0
        while started < len(reqs):
            while nxt < len(reqs) and arrivals[nxt] <= t:
                queue.append([reqs[nxt][0], reqs[nxt][1], 0])
                nxt += 1
            running = [r for r in running if r[1] > t]
            while len(running) < slots and queue:
                reserved = sum(r[0] for r in running)
                fp = [q[0] for q in queue]
                ps = [q[2] for q in queue]
                k = ab.svm_server_admission(fp, ps, reserved, budget, len(running))
                assert k == rule(fp, ps, reserved, len(running))
                if k < 0:
                    # the bound at work: a younger request would fit but the oldest was passed 4 times
                    if queue[0][2] >= 4 and any(reserved + q[0] <= budget for q in queue[1:]):
                        capped += 1
                    break
                if k > 0:
                    queue[0][2] += 1
                    backfills += 1
                q = queue.pop(k)
                max_passed = max(max_passed, q[2])
                running.append((q[0], t + q[1]))
                started += 1
                total = sum(r[0] for r in running)
                assert total <= budget or len(running) == 1
            t += 1
        assert max_passed <= 4
    assert backfills > 0 and capped > 0   # both branches of the rule were taken
