"""Workload 3 through the device interior point method (Algorithm 1, Sec. 2) against the oracle.

Workload 3: n = 1e5, d = 12 (8 Gaussian + 4 binary features), four consecutive 3-D windows,
sigma = 1, C = 10, tanh teacher with 5 % flips, pivoted-Cholesky preconditioner of rank r = 200
(err_tol 0, so that the rank is the one the workload states), MINRES tolerance 1e-6, FP32
operator with FP64 refinement, stop at relative duality gap 1e-6.

Two checks:
* the stated 20,000-point subsample (rows subsample_rows(1e5, 20000, SEED_BASE + 300)): the dual
  objective of the device solution, evaluated by the oracle's direct FP64 sum, is within 1e-6
  relative of the optimum the oracle's dense Algorithm 1 reached (tests/golden/
  config3_sub20000_ipm.json, written by tests/golden/make_config3_ipm.py from oracle/ only);
* the full n = 1e5 problem: the oracle's direct FP64 matvec K (y .* alpha) at all 1e5 points
  gives the exact dual D and primal P of the device solution. Weak duality puts the optimum
  between them, so (P - D) / |P| <= 1e-6 proves D within 1e-6 of the optimum at full size
  without a dense solve."""
import json
import os

import numpy as np
import pytest

from oracle import ipm as oi
from oracle import kernel as ok
from synth import SEED_BASE, config3, subsample_rows

from ._gpu_util import require_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config3_sub20000_ipm.json")


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.fixture(scope="module")
def full():
    return config3()


def _opts(ab):
    o = ab.svm_opts_default()
    o.rank = 200
    o.err_tol = 0.0
    o.krylov_tol = 1e-6
    o.max_iter = 100
    o.ell = 1.0
    return o


def _exact_objectives(X, y, W, alpha, b, C):
    """D and P of (alpha, b) with f = K (y .* alpha) from the oracle's direct FP64 sum."""
    f = ok.anova_matvec(X, W, 1.0, y * alpha)
    D = float(alpha.sum() - 0.5 * (y * alpha) @ f)
    P = float(0.5 * (y * alpha) @ f + C * np.maximum(0.0, 1.0 - y * (f + b)).sum())
    return D, P


def test_config3_subsample_dual_objective_matches_oracle(env, full):
    torch, ab = env
    with open(GOLDEN) as fh:
        g = json.load(fh)
    idx = subsample_rows(g["n_full"], g["n_sub"], g["subsample_seed"])
    assert g["subsample_seed"] == SEED_BASE + 300
    X, y, W, C = full["X"][idx], full["y"][idx], full["windows"], full["C"]
    # the stored optimum belongs to exactly these rows and labels
    assert int(idx.sum()) == g["idx_sum"] and float(y.sum()) == g["y_sum"] and C == g["C"]
    assert g["reason"] == "converged" and g["rel_gap"] <= 1e-8
    alpha, b, st, status = ab.svm_ipm_solve(X, y, C, 1e-6, opts=_opts(ab), windows=W)
    assert status == ab.ANOVA_OK, st
    assert st["rank"] == 200
    D, P = _exact_objectives(X, y, W, alpha, b, C)
    assert abs(D - g["dual"]) <= 1e-6 * abs(g["dual"]), (D, g["dual"])
    assert np.all(alpha >= 0) and np.all(alpha <= C)
    assert abs(st["dual"] - D) <= 1e-8 * abs(D)


def test_config3_full_size_certified_by_exact_gap(env, full):
    torch, ab = env
    X, y, W, C = full["X"], full["y"], full["windows"], full["C"]
    assert X.shape == (100_000, 12)
    alpha, b, st, status = ab.svm_ipm_solve(X, y, C, 1e-6, opts=_opts(ab), windows=W)
    assert status == ab.ANOVA_OK, st
    assert st["rank"] == 200 and st["converged"] == 1
    assert np.all(alpha >= 0) and np.all(alpha <= C)
    D, P = _exact_objectives(X, y, W, alpha, b, C)
    # weak duality with an exact kernel: D(alpha) <= D* <= P(w(alpha), b) up to b y^T alpha
    slack = abs(b * float(y @ alpha))
    assert P - D >= -slack - 1e-9 * abs(P)
    assert (P - D) / max(1.0, abs(P)) <= 1.05e-6, (P, D)
    # the stopping rule's infeasibility: |y^T alpha| / max(1, |y^T alpha^0|), alpha^0 = 1/2 e
    assert abs(float(y @ alpha)) <= 1.01e-6 * max(1.0, 0.5 * abs(float(y.sum())))
    # the solver's own FP64-plan objectives agree with the exact ones
    assert abs(st["dual"] - D) <= 1e-8 * abs(D)
    assert abs(st["primal"] - P) <= 1e-7 * abs(P)
