"""Serving loop: requests submitted to an svm_server give bitwise the result of svm_ipm_solve
alone, whatever the admission order, slot count or memory budget; the budget is respected."""
import numpy as np
import pytest

from synth import config4

from ._gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _opts(ab, ell=None):
    o = ab.svm_opts_default()
    o.rank = 60
    o.max_iter = 150
    if ell is not None:
        o.ell = ell
    return o


def _alone(ab, p, tol):
    return ab.svm_ipm_solve(p["X"], p["y"], p["C"], tol, opts=_opts(ab, p["sigma"]),
                            windows=p["windows"])


@pytest.mark.parametrize("slots,budget_kind", [(4, "large"), (3, "one_at_a_time")])
def test_server_equals_alone(slots, budget_kind):
    torch, ab = require_gpu()
    probs = config4(count=6, n_lo=300, n_hi=1500, seed=11)
    tol = 1e-7
    o = _opts(ab)
    foot = [ab.svm_request_footprint(p["X"].shape[0], len(p["windows"]), o) for p in probs]
    budget = (64 << 30) if budget_kind == "large" else max(foot)
    srv = ab.SvmServer(tol, opts=o, slots=slots, hbm_budget_bytes=budget)
    try:
        tickets = [srv.submit(p["X"], p["y"], p["C"], ell=p["sigma"], windows=p["windows"])
                   for p in probs]
        # wait in reverse order: completion order must not matter
        results = {t: srv.wait(t) for t in reversed(tickets)}
        st = srv.stats()
    finally:
        srv.destroy()
    assert st["submitted"] == st["completed"] == len(probs)
    assert st["running"] == 0 and st["queued"] == 0 and st["reserved_bytes"] == 0
    assert 0 < st["p50_latency_ms"] <= st["p99_latency_ms"]
    assert st["peak_reserved_bytes"] <= budget
    for p, t in zip(probs, tickets):
        alpha_s, b_s, stats_s, status_s = results[t]
        alpha, b, stats, status = _alone(ab, p, tol)
        assert status == status_s == ab.ANOVA_OK
        assert np.array_equal(alpha, alpha_s) and b == b_s
        assert stats["iterations"] == stats_s["iterations"]


def test_server_streaming_submission():
    """Requests that arrive while others run (submit, wait, submit again) are admitted as slots
    free up, and a request larger than the whole budget still runs (alone)."""
    torch, ab = require_gpu()
    probs = config4(count=4, n_lo=300, n_hi=900, seed=12)
    tol = 1e-7
    srv = ab.SvmServer(tol, opts=_opts(ab), slots=2, hbm_budget_bytes=1)
    try:
        t0 = srv.submit(probs[0]["X"], probs[0]["y"], probs[0]["C"], ell=probs[0]["sigma"],
                        windows=probs[0]["windows"])
        r0 = srv.wait(t0)
        rest = [srv.submit(p["X"], p["y"], p["C"], ell=p["sigma"], windows=p["windows"])
                for p in probs[1:]]
        srv.drain()
        rs = [r0] + [srv.wait(t) for t in rest]
        st = srv.stats()
    finally:
        srv.destroy()
    assert st["completed"] == 4
    for p, r in zip(probs, rs):
        alpha, b, _, status = _alone(ab, p, tol)
        assert r[3] == status == ab.ANOVA_OK
        assert np.array_equal(alpha, r[0]) and b == r[1]


def test_server_backfills_a_request_that_fits_past_one_that_does_not():
    """With A running and the budget too small for B beside it, C (younger, small) starts before B
    instead of waiting behind it (backfill); every result is still the one alone."""
    torch, ab = require_gpu()
    from synth import small_problem
    probs = [small_problem(1600, 9, 21), small_problem(1500, 9, 22), small_problem(300, 9, 23)]
    tol = 1e-7
    o = _opts(ab)
    foot = [ab.svm_request_footprint(p["X"].shape[0], len(p["windows"]), o) for p in probs]
    budget = foot[0] + foot[2]
    assert foot[0] + foot[1] > budget
    srv = ab.SvmServer(tol, opts=o, slots=2, hbm_budget_bytes=budget)
    try:
        tickets = [srv.submit(p["X"], p["y"], 1.0, windows=p["windows"]) for p in probs]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.destroy()
    assert st["completed"] == 3 and st["backfilled"] >= 1
    assert st["peak_reserved_bytes"] <= budget
    for p, r in zip(probs, results):
        alpha, b, _, status = ab.svm_ipm_solve(p["X"], p["y"], 1.0, tol, opts=o, windows=p["windows"])
        assert r[3] == status == ab.ANOVA_OK
        assert np.array_equal(alpha, r[0]) and b == r[1]
