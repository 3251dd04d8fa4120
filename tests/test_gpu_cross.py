"""Targets distinct from sources (evaluating the decision function at new points, Sec. 6):
anova_cross_matvec against the oracle's direct cross sum, in FP32 (1e-4) and FP64 (1e-9), with
mixed window dimensions; with targets equal to the sources it is the square matvec; plans that
do not match are refused."""
import numpy as np
import pytest

from oracle import kernel as ok
from synth import minmax_scale, SEED_BASE

from ._gpu_util import require_gpu, rel_l2, to_dev, from_dev

pytestmark = pytest.mark.gpu

W = np.array([[0, 1, 2], [3, 4, -1], [5, -1, -1]])


def _points(n, seed):
    rng = np.random.default_rng(seed)
    # scale with the same fixed box as the sources so both sets share the coordinate system
    return np.clip(rng.standard_normal((n, 6)) * 0.06, -0.2, 0.2)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cross_matvec_matches_direct_sum(prec):
    torch, ab = require_gpu()
    Xs, Xt = _points(3000, SEED_BASE + 71), _points(1700, SEED_BASE + 72)
    w = np.random.default_rng(SEED_BASE + 73).standard_normal(3000)
    fl, dt, N, m, bar = ((ab.ANOVA_FP32, torch.float32, 32, 4, 1e-4) if prec == "fp32"
                         else (ab.ANOVA_FP64, torch.float64, 64, 6, 1e-9))
    src = ab.anova_nfft_plan(Xs, W, 0.8, N=N, m=m, flags=fl)
    tgt = ab.anova_nfft_plan(Xt, W, 0.8, N=N, m=m, flags=fl)
    f = torch.empty(1700, dtype=dt, device="cuda")
    ab.anova_cross_matvec(src, tgt, to_dev(torch, w, dt), f)
    torch.cuda.synchronize()
    assert rel_l2(from_dev(f), ok.anova_cross_matvec(Xs, Xt, W, 0.8, w)) <= bar


def test_cross_with_targets_equal_to_sources_is_the_matvec():
    torch, ab = require_gpu()
    X = _points(2500, SEED_BASE + 74)
    v = np.random.default_rng(SEED_BASE + 75).standard_normal(2500)
    a = ab.anova_nfft_plan(X, W, 0.8, N=32, m=4)
    b = ab.anova_nfft_plan(X, W, 0.8, N=32, m=4)
    vd = to_dev(torch, v, torch.float32)
    f = torch.empty_like(vd)
    kv = torch.empty_like(vd)
    ab.anova_cross_matvec(a, b, vd, f)
    ab.anova_matvec(a, vd, kv, 1)
    torch.cuda.synchronize()
    assert rel_l2(from_dev(f), from_dev(kv)) <= 2e-6


def test_mismatched_plans_are_refused():
    torch, ab = require_gpu()
    X = _points(200, SEED_BASE + 76)
    a = ab.anova_nfft_plan(X, W, 0.8, N=32, m=4)
    vd = torch.zeros(200, device="cuda")
    f = torch.empty(200, device="cuda")
    for other in (ab.anova_nfft_plan(X, W, 0.9, N=32, m=4), ab.anova_nfft_plan(X, W, 0.8, N=32, m=3),
                  ab.anova_nfft_plan(X, W[:2], 0.8, N=32, m=4)):
        with pytest.raises(ab.AnovaError) as ei:
            ab.anova_cross_matvec(a, other, vd, f)
        assert ei.value.status == ab.ANOVA_ERR_INVALID_ARG


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_kept_model_matches_cross_matvec_and_direct_sum(prec):
    """A model keeps the sources' convolved grids: evaluating it at two target sets equals the
    cross product (up to the order of sums) and the direct sum, after the source plan and the
    weights are gone."""
    torch, ab = require_gpu()
    Xs = _points(4000, SEED_BASE + 77)
    w = np.random.default_rng(SEED_BASE + 78).standard_normal(4000)
    fl, dt, N, m, bar = ((ab.ANOVA_FP32, torch.float32, 32, 4, 1e-4) if prec == "fp32"
                         else (ab.ANOVA_FP64, torch.float64, 64, 6, 1e-9))
    src = ab.anova_nfft_plan(Xs, W, 0.8, N=N, m=m, flags=fl)
    wd = to_dev(torch, w, dt)
    model = ab.anova_model_create(src, wd)
    targets = [_points(2100, SEED_BASE + 79), _points(900, SEED_BASE + 80)]
    crossed = []
    for Xt in targets:
        tgt = ab.anova_nfft_plan(Xt, W, 0.8, N=N, m=m, flags=fl)
        f = torch.empty(Xt.shape[0], dtype=dt, device="cuda")
        ab.anova_cross_matvec(src, tgt, wd, f)
        crossed.append(from_dev(f))
    src.destroy()
    del wd
    for Xt, fc in zip(targets, crossed):
        tgt = ab.anova_nfft_plan(Xt, W, 0.8, N=N, m=m, flags=fl)
        f = torch.empty(Xt.shape[0], dtype=dt, device="cuda")
        ab.anova_model_eval(model, tgt, f)
        torch.cuda.synchronize()
        ab.anova_plan_check(tgt)
        got = from_dev(f)
        assert rel_l2(got, fc) <= (2e-6 if prec == "fp32" else 1e-12)
        assert rel_l2(got, ok.anova_cross_matvec(Xs, Xt, W, 0.8, w)) <= bar
    model.destroy()


def test_kept_model_refuses_mismatched_plans():
    torch, ab = require_gpu()
    X = _points(300, SEED_BASE + 81)
    src = ab.anova_nfft_plan(X, W, 0.8, N=32, m=4)
    model = ab.anova_model_create(src, torch.ones(300, device="cuda"))
    f = torch.empty(300, device="cuda")
    for other in (ab.anova_nfft_plan(X, W, 0.9, N=32, m=4), ab.anova_nfft_plan(X, W, 0.8, N=32, m=3),
                  ab.anova_nfft_plan(X, W[:2], 0.8, N=32, m=4),
                  ab.anova_nfft_plan(X, W, 0.8, N=64, m=6, flags=ab.ANOVA_FP64)):
        with pytest.raises(ab.AnovaError) as ei:
            ab.anova_model_eval(model, other, f)
        assert ei.value.status == ab.ANOVA_ERR_INVALID_ARG
