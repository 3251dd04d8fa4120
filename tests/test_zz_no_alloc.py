"""anova_spread_grid_noalloc: the spread stage with its scratch in a static device array, for
callers that cannot allocate device memory during the call (a process whose device memory is
reserved up front by its own pool, or a loop whose per-call time budget excludes cudaMalloc).
It must give the grid of anova_spread_grid, call after call, and refuse windows whose scratch
would not fit. Collected last (file name) so a failure here does not hide the other tests."""
import numpy as np
import pytest

from synth import minmax_scale, consecutive_windows

from ._gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _compare(torch, ab, plan, l, v, n_os, dw, dt, tol):
    ref = torch.empty((n_os,) * dw, dtype=dt, device="cuda")
    ab.anova_spread_grid(plan, l, v, ref)
    torch.cuda.synchronize()
    r = ref.cpu().numpy().astype(np.float64)
    for _ in range(2):                      # two calls in a row share the static scratch
        out = torch.full((n_os,) * dw, 7.0, dtype=dt, device="cuda")
        ab.anova_spread_grid_noalloc(plan, l, v, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(o - r)) <= tol * np.max(np.abs(r))


def test_noalloc_spread_matches_spread_grid():
    torch, ab = require_gpu()
    rng = np.random.default_rng(41)
    X = minmax_scale(rng.standard_normal((20000, 8)))
    W = consecutive_windows(8)               # 3-D, 3-D and 2-D windows
    plan = ab.anova_nfft_plan(X, W, 0.9, N=32, m=4, flags=ab.ANOVA_FP32)
    for l, dw in ((0, 3), (2, 2), (1, 3)):
        v = torch.tensor(rng.standard_normal(20000), dtype=torch.float32, device="cuda")
        _compare(torch, ab, plan, l, v, 64, dw, torch.float32, 2e-6)
    plan64 = ab.anova_nfft_plan(X[:3000], W, 0.9, N=16, m=4, flags=ab.ANOVA_FP64)
    v = torch.tensor(rng.standard_normal(3000), dtype=torch.float64, device="cuda")
    _compare(torch, ab, plan64, 0, v, 32, 3, torch.float64, 1e-13)


def test_noalloc_spread_rejects_windows_beyond_its_scratch():
    torch, ab = require_gpu()
    rng = np.random.default_rng(42)
    X = rng.uniform(-0.2, 0.2, size=(50000, 3))   # ~16k occupied bins at N = 64, FP64
    plan = ab.anova_nfft_plan(X, [[0, 1, 2]], 1.0, N=64, m=6, flags=ab.ANOVA_FP64)
    v = torch.zeros(50000, dtype=torch.float64, device="cuda")
    grid = torch.zeros((128, 128, 128), dtype=torch.float64, device="cuda")
    with pytest.raises(ab.AnovaError) as ei:
        ab.anova_spread_grid_noalloc(plan, 0, v, grid)
    assert ei.value.status == ab.ANOVA_ERR_INVALID_ARG
    assert "scratch" in str(ei.value)
