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


@pytest.mark.parametrize("flags_name,bounds_frac", [("fp32", (0, 0.5, 1.0)), ("fp32", (0, 0.07, 0.6, 1.0)),
                                                   ("fp64", (0, 0.3, 1.0))])
def test_split_matvec_over_shards_equals_one_plan(flags_name, bounds_frac):
    """anova_matvec_grids on every shard, the grids summed (the all-reduce of a multi-GPU run),
    anova_matvec_from_grids on every shard: the rows equal the one-plan matvec up to the order of
    sums, for several right-hand sides and mixed window dimensions, and the direct sum within the
    bar. One shard alone reproduces anova_matvec."""
    torch, ab = require_gpu()
    rng = np.random.default_rng(SEED_BASE + 77)
    n = 6000
    X = minmax_scale(rng.standard_normal((n, 8)))
    W = np.array([[0, 1, 2], [3, 4, -1], [5, 6, 7], [7, -1, -1]])
    fl, dt, N, m, bar = ((ab.ANOVA_FP32, torch.float32, 32, 4, 2e-6) if flags_name == "fp32"
                         else (ab.ANOVA_FP64, torch.float64, 64, 6, 1e-12))
    nrhs = 3
    V = rng.standard_normal((n, nrhs))
    bounds = [int(round(f * n)) for f in bounds_frac]
    plans = [ab.anova_nfft_plan(X[b0:b1], W, 0.8, N=N, m=m, flags=fl) for b0, b1 in zip(bounds[:-1], bounds[1:])]
    gt = ab.anova_plan_grid_size(plans[0])
    assert all(ab.anova_plan_grid_size(p) == gt for p in plans)
    total = torch.zeros((nrhs, gt), dtype=dt, device="cuda")
    for p, b0, b1 in zip(plans, bounds[:-1], bounds[1:]):
        g = torch.empty((nrhs, gt), dtype=dt, device="cuda")
        ab.anova_matvec_grids(p, to_dev(torch, V[b0:b1], dt), g, nrhs)
        total += g                                      # the all-reduce
    got = np.zeros((n, nrhs))
    for p, b0, b1 in zip(plans, bounds[:-1], bounds[1:]):
        kv = torch.empty((nrhs, b1 - b0), dtype=dt, device="cuda")
        ab.anova_matvec_from_grids(p, total, kv, nrhs)
        torch.cuda.synchronize()
        ab.anova_plan_check(p)
        got[b0:b1] = from_dev(kv)
    one = ab.anova_nfft_plan(X, W, 0.8, N=N, m=m, flags=fl)
    kv = torch.empty((nrhs, n), dtype=dt, device="cuda")
    ab.anova_matvec(one, to_dev(torch, V, dt), kv, nrhs)
    ref = from_dev(kv)
    for r in range(nrhs):
        assert rel_l2(got[:, r], ref[:, r]) <= bar
    direct = ok.anova_matvec(X, W, 0.8, V[:, 0])
    assert rel_l2(got[:, 0], direct) <= (1e-4 if flags_name == "fp32" else 1e-9)
    # one shard: grids then from_grids is the matvec itself
    g1 = torch.empty((nrhs, gt), dtype=dt, device="cuda")
    vd = to_dev(torch, V, dt)
    ab.anova_matvec_grids(one, vd, g1, nrhs)
    kv1 = torch.empty_like(kv)
    ab.anova_matvec_from_grids(one, g1, kv1, nrhs)
    torch.cuda.synchronize()
    for r in range(nrhs):
        assert rel_l2(from_dev(kv1)[:, r], ref[:, r]) <= bar
