"""The multi-GPU design of the matvec simulated on one GPU through the C ABI's stage calls:
the points are split into G shards with one plan each; every shard spreads its points onto the
full grid of each window (anova_spread_grid), the shard grids are summed (the all-reduce of the
design), the FFT and scaling run once (anova_conv_grid), and every shard interpolates its own
points (anova_interp_grid). The result must equal the single-plan matvec up to the rounding of
the summation order, and the direct sum within the plan's bar."""
import numpy as np
import pytest

from oracle import kernel as ok
from synth import config1, minmax_scale, SEED_BASE

from ._gpu_util import require_gpu, rel_l2, to_dev, from_dev

pytestmark = pytest.mark.gpu


def _sharded(torch, ab, X, W, sigma, v, bounds, flags, dt, N, m):
    plans = [ab.anova_nfft_plan(X[b0:b1], W, sigma, N=N, m=m, flags=flags)
             for b0, b1 in zip(bounds[:-1], bounds[1:])]
    vd = to_dev(torch, v, dt)
    n_os = 2 * N
    out = np.zeros(X.shape[0])
    for l, win in enumerate(np.asarray(W).reshape(-1, 3)):
        dw = int((win >= 0).sum())
        total = torch.zeros((n_os,) * dw, dtype=dt, device="cuda")
        for pl, b0, b1 in zip(plans, bounds[:-1], bounds[1:]):
            g = torch.empty((n_os,) * dw, dtype=dt, device="cuda")
            ab.anova_spread_grid(pl, l, vd[b0:b1].contiguous(), g)
            total += g                                  # the all-reduce
        conv = torch.empty_like(total)
        ab.anova_conv_grid(plans[0], l, total, conv)    # the same on every shard
        for pl, b0, b1 in zip(plans, bounds[:-1], bounds[1:]):
            f = torch.empty(b1 - b0, dtype=dt, device="cuda")
            ab.anova_interp_grid(pl, l, conv, f)
            torch.cuda.synchronize()
            out[b0:b1] += from_dev(f)
    return out


@pytest.mark.parametrize("bounds", [[0, 1000, 2000], [0, 1, 2000], [0, 500, 900, 2000]])
def test_sharded_fp32_equals_single_plan_and_direct_sum(bounds):
    torch, ab = require_gpu()
    cfg = config1()
    X, W, sigma = cfg["X"], cfg["windows"], cfg["sigma"]
    v = np.random.default_rng(SEED_BASE + 61).standard_normal(X.shape[0])
    got = _sharded(torch, ab, X, W, sigma, v, bounds, ab.ANOVA_FP32, torch.float32, 32, 4)
    plan = ab.anova_nfft_plan(X, W, sigma, N=32, m=4)
    vd = to_dev(torch, v, torch.float32)
    kv = torch.empty_like(vd)
    ab.anova_matvec(plan, vd, kv, 1)
    torch.cuda.synchronize()
    single = from_dev(kv)
    assert rel_l2(got, single) <= 2e-6
    assert rel_l2(got, ok.anova_matvec(X, W, sigma, v)) <= 1e-4


def test_sharded_fp64_mixed_windows():
    torch, ab = require_gpu()
    rng = np.random.default_rng(SEED_BASE + 62)
    X = minmax_scale(rng.standard_normal((1500, 6)))
    W = np.array([[0, 1, 2], [3, 4, -1], [5, -1, -1]])
    v = rng.standard_normal(1500)
    bounds = [0, 700, 1500]
    got = _sharded(torch, ab, X, W, 0.8, v, bounds, ab.ANOVA_FP64, torch.float64, 64, 6)
    assert rel_l2(got, ok.anova_matvec(X, W, 0.8, v)) <= 1e-9
