"""Concurrent batched solves: every problem's result is bitwise the same alone and in the batch,
and matches the dense-KKT oracle's dual objective."""
import numpy as np
import pytest

from oracle import ipm as oi
from oracle import kernel as ok
from synth import config4

from ._gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_batch_equals_alone_and_oracle():
    torch, ab = require_gpu()
    probs = config4(count=6, n_lo=300, n_hi=1500)
    o = ab.svm_opts_default()
    o.rank = 60
    o.max_iter = 150
    tol = 1e-7
    batch = ab.svm_ipm_solve_batch(
        [dict(X=p["X"], y=p["y"], C=p["C"], ell=p["sigma"], windows=p["windows"]) for p in probs],
        tol, opts=o, concurrency=3)
    for p, (alpha_b, b_b, st_b, status_b) in zip(probs, batch):
        o1 = ab.svm_opts_default()
        o1.rank = 60
        o1.max_iter = 150
        o1.ell = p["sigma"]
        alpha, b, st, status = ab.svm_ipm_solve(p["X"], p["y"], p["C"], tol, opts=o1,
                                                windows=p["windows"])
        assert status == status_b == ab.ANOVA_OK
        assert np.array_equal(alpha, alpha_b) and b == b_b
        K = ok.anova_kernel_matrix(p["X"], p["windows"], p["sigma"])
        ref = oi.ipm_dense(K, p["y"], p["C"], tol=1e-10, max_iter=400)
        d = oi.dual_objective(K, p["y"], alpha)
        d_ref = oi.dual_objective(K, p["y"], ref["alpha"])
        assert abs(d - d_ref) <= 1e-6 * abs(d_ref), (p["C"], p["sigma"], d, d_ref)
