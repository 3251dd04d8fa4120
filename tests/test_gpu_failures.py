"""Failure detection without a GPU fault: every failure here is made by the host (a wait limit of
zero polls, a factor step given an indefinite matrix, an iteration cap), and each must come back
as the documented status while the context stays usable for the next call.

* ANOVA_ERR_TIMEOUT: the tensor-core interpolation's completion waits are bounded; with the limit
  lowered to zero polls the first wait gives up at once, the kernel sets the plan's flag, drains
  the products it started (with the full limit) and frees its tensor memory. anova_plan_check
  reports the flag; a fresh plan on the same device then gives the correct product.
* ANOVA_ERR_BREAKDOWN: the Woodbury core M = I + L^T Theta^-1 L (Sec. 5) is positive definite
  only for Theta > 0; a negative Theta makes it indefinite and its Cholesky factor breaks down.
* ANOVA_ERR_NOT_CONVERGED: Algorithm 1 (Sec. 2) stopped at max_iter = 1 returns the status with
  its last iterate."""
import numpy as np
import pytest

from oracle import kernel as ok
from synth import config1, matvec_vectors, minmax_scale

from ._gpu_util import from_dev, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def test_interpolation_wait_timeout_is_reported_and_the_context_survives(env):
    torch, ab = env
    rng = np.random.default_rng(71)
    X = minmax_scale(rng.standard_normal((6000, 6)))
    W = np.array([[0, 1, 2], [3, 4, 5]])
    v = rng.standard_normal(6000)
    flags = ab.ANOVA_FP32 | ab.ANOVA_INTERP_TENSOR
    plan = ab.anova_nfft_plan(X, W, 1.0, N=32, m=4, flags=flags)
    ab.anova_plan_set_wait_limit(plan, 0)
    dv = to_dev(torch, v, torch.float32)
    out = torch.empty_like(dv)
    ab.anova_matvec(plan, dv, out, 1)
    with pytest.raises(ab.AnovaError) as ei:
        ab.anova_plan_check(plan)
    assert ei.value.status == ab.ANOVA_ERR_TIMEOUT
    plan.destroy()
    # the device and the library still work: a fresh plan with the default limit is correct
    plan2 = ab.anova_nfft_plan(X, W, 1.0, N=32, m=4, flags=flags)
    out2 = torch.empty_like(dv)
    ab.anova_matvec(plan2, dv, out2, 1)
    ab.anova_plan_check(plan2)
    ref = ok.anova_matvec(X, W, 1.0, v)
    assert rel_l2(from_dev(out2), ref) <= 1e-4
    # restoring the default on a plan makes its calls valid again (a new plan's flag is clear)
    ab.anova_plan_set_wait_limit(plan2, -1)
    ab.anova_matvec(plan2, dv, out2, 1)
    ab.anova_plan_check(plan2)


def test_negative_theta_breaks_down_the_woodbury_core(env):
    torch, ab = env
    cfg = config1(n=1500)
    plan = ab.anova_nfft_plan(cfg["X"], cfg["windows"], 1.0, N=64, m=6, flags=ab.ANOVA_FP64)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_GREEDY, 40, 1e-5)
    y = torch.tensor(cfg["y"], dtype=torch.float64, device="cuda")
    theta = torch.full((1500,), -1e-3, dtype=torch.float64, device="cuda")
    with pytest.raises(ab.AnovaError) as ei:
        ab.lowrank_precond_set_theta(lr, theta, y)
    assert ei.value.status == ab.ANOVA_ERR_BREAKDOWN
    # a valid Theta on the same factor afterwards works and gives a finite apply
    theta.fill_(0.5)
    ab.lowrank_precond_set_theta(lr, theta, y)
    g = torch.ones(1501, dtype=torch.float64, device="cuda")
    x = torch.empty_like(g)
    ab.lowrank_precond_apply(lr, theta, y, g, x)
    torch.cuda.synchronize()
    assert torch.isfinite(x).all()


def test_iteration_cap_returns_not_converged_with_the_last_iterate(env):
    torch, ab = env
    cfg = config1(n=800)
    o = ab.svm_opts_default()
    o.max_iter = 1
    o.rank = 50
    alpha, b, st, status = ab.svm_ipm_solve(cfg["X"], cfg["y"], cfg["C"], 1e-6, opts=o, windows=cfg["windows"])
    assert status == ab.ANOVA_ERR_NOT_CONVERGED
    assert st["iterations"] == 1 and st["converged"] == 0
    assert np.all(np.isfinite(alpha)) and np.all(alpha > 0) and np.all(alpha < cfg["C"])
    # one Newton step moved the iterate away from the start alpha^0 = min(C/2, 1/2) e
    assert np.max(np.abs(alpha - 0.5)) > 0
