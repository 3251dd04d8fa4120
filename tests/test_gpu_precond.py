"""Parity of the device low-rank preconditioners (Secs. 4-5) with the FP64 oracle."""
import numpy as np
import pytest

from oracle import kernel as ok
from oracle import precond as op
from synth import minmax_scale, consecutive_windows

from ._gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _setup(ab, n=300, d=6, ell=0.5, seed=1, binary=False):
    rng = np.random.default_rng(seed)
    if binary:
        X = minmax_scale(rng.integers(0, 2, size=(n, d)).astype(float))
    else:
        X = minmax_scale(rng.standard_normal((n, d)))
    W = consecutive_windows(d)
    plan = ab.anova_nfft_plan(X, W, ell, N=64, m=6, flags=ab.ANOVA_FP64)
    K = ok.anova_kernel_matrix(X, W, ell)
    return X, W, plan, K, rng


def _factor(torch, ab, lr, n):
    rank, piv = ab.lowrank_info(lr)
    L = torch.empty((rank, n), dtype=torch.float64, device="cuda")
    ab.lowrank_factor(lr, L)
    return L.cpu().numpy().T, piv


def test_pivoted_cholesky_matches_algorithm2(env):
    torch, ab = env
    X, W, plan, K, _ = _setup(ab)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_GREEDY, 25, 0.0)
    L, piv = _factor(torch, ab, lr, 300)
    Lo, pivo = op.pivoted_cholesky(K, 25)
    assert L.shape == (300, 25)
    assert np.array_equal(piv, pivo)
    assert np.allclose(L, Lo, rtol=0, atol=1e-10)


def test_pivoted_cholesky_full_rank_and_err_tol(env):
    torch, ab = env
    X, W, plan, K, _ = _setup(ab, n=80, ell=0.05)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_GREEDY, 80, 0.0)
    L, _ = _factor(torch, ab, lr, 80)
    assert np.allclose(L @ L.T, K, rtol=0, atol=1e-10 * np.max(K))
    X2, W2, plan2, K2, _ = _setup(ab, n=200, d=3, ell=2.0)
    lr2 = ab.lowrank_precond_build(plan2, ab.PCHOL_GREEDY, 200, 1e-5)
    L2, _ = _factor(torch, ab, lr2, 200)
    assert L2.shape[1] < 40
    assert np.max(np.diag(K2 - L2 @ L2.T)) <= 1e-5 * np.max(np.diag(K2)) + 1e-13


def test_rank_of_duplicate_heavy_window(env):
    torch, ab = env
    X, W, plan, K, _ = _setup(ab, n=400, d=3, ell=0.3, binary=True)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_GREEDY, 50, 1e-10)
    L, _ = _factor(torch, ab, lr, 400)
    assert L.shape[1] == 8
    assert np.allclose(L @ L.T, K, atol=1e-9)


def test_nystrom_on_pivot_set(env):
    torch, ab = env
    X, W, plan, K, _ = _setup(ab, n=250, seed=3)
    lr = ab.lowrank_precond_build(plan, ab.NYSTROM, 20, 0.0)
    Z, piv = _factor(torch, ab, lr, 250)
    Zo = op.nystrom_columns(K, piv)
    assert np.allclose(Z @ Z.T, Zo @ Zo.T, rtol=0, atol=1e-8 * np.max(K))
    assert np.allclose((Z @ Z.T)[:, piv], K[:, piv], atol=1e-8)


def test_woodbury_block_preconditioner(env):
    torch, ab = env
    X, W, plan, K, rng = _setup(ab, n=500, seed=4)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_GREEDY, 30, 0.0)
    L, _ = _factor(torch, ab, lr, 500)
    L32 = L.astype(np.float32).astype(np.float64)   # the apply uses the FP32 panel
    y = np.where(rng.standard_normal(500) >= 0, 1.0, -1.0)
    theta = np.exp(rng.uniform(-4, 4, 500))
    g = rng.standard_normal(501)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    th, yy, gg = dev(theta), dev(y), dev(g)
    x = torch.empty(501, dtype=torch.float64, device="cuda")
    ab.lowrank_precond_set_theta(lr, th, yy)
    ab.lowrank_precond_apply(lr, th, yy, gg, x)
    torch.cuda.synchronize()
    s = y @ op.woodbury_apply(L32, theta, y, y)
    ref = op.blockdiag_apply(L32, theta, y, g, s)
    got = x.cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-8, atol=1e-10 * np.max(np.abs(ref)))
    # and against the dense inverse of A^ with the same factor
    dense = np.linalg.solve(op.dense_Ahat(L32, theta, y), g[:500])
    assert np.allclose(got[:500], dense, rtol=1e-7, atol=1e-9 * np.max(np.abs(dense)))


@pytest.mark.parametrize("seed", [0, 12345, 2 ** 63 + 7])
def test_randomly_pivoted_cholesky_matches_oracle(env, seed):
    """Same SplitMix64 draws on both sides: identical pivots and the same factor."""
    torch, ab = env
    X, W, plan, K, _ = _setup(ab, n=400, seed=3)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_RANDOM, 30, 0.0, seed=seed)
    L, piv = _factor(torch, ab, lr, 400)
    Lo, pivo = op.rp_cholesky(K, 30, seed=seed)
    assert np.array_equal(piv, pivo)
    assert np.allclose(L, Lo, rtol=0, atol=1e-10)


def test_randomly_pivoted_cholesky_err_tol_stop(env):
    torch, ab = env
    X, W, plan, K, _ = _setup(ab, n=200, d=3, ell=2.0)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_RANDOM, 200, 1e-5, seed=99)
    L, piv = _factor(torch, ab, lr, 200)
    Lo, pivo = op.rp_cholesky(K, 200, seed=99, err_tol=1e-5)
    assert np.array_equal(piv, pivo)
    assert np.max(np.diag(K - L @ L.T)) <= 1e-5 * np.max(np.diag(K)) + 1e-13


def test_per_window_stacked_factors_match_oracle(env):
    """Per-window stacked factors: each window's block equals Algorithm 2 on that window's kernel,
    blocks in the plan's window order (stable, decreasing dimension)."""
    torch, ab = env
    rng = np.random.default_rng(17)
    n = 300
    X = minmax_scale(rng.standard_normal((n, 6)))
    W = np.array([[0, -1, -1], [1, 2, 3], [4, 5, -1]], dtype=np.int32)
    # ell and rank keep every pivot choice clear of rounding (the 1-D window's residual is still
    # ~1e-5 at its last pivot, with the runner-up ~1e-9 below it)
    plan = ab.anova_nfft_plan(X, W, 0.2, N=64, m=6, flags=ab.ANOVA_FP64)
    internal = sorted(range(3), key=lambda l: -int(np.sum(W[l] >= 0)))
    Ks = [ok.window_kernel_matrix(X, W[l], 0.2) for l in internal]
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_PER_WINDOW, 24, 0.0)
    L, piv = _factor(torch, ab, lr, n)
    Lo, pivo = op.per_window_cholesky(Ks, 8)
    assert L.shape == Lo.shape
    assert np.array_equal(piv, pivo)
    assert np.allclose(L, Lo, rtol=0, atol=1e-10)


def test_per_window_full_rank_and_early_stop(env):
    """A one-feature window on binary data has rank 2: its block stops there and the next window's
    block starts right after it; with enough rank per window L L^T is the summed kernel."""
    torch, ab = env
    rng = np.random.default_rng(5)
    n = 120
    X = minmax_scale(np.column_stack([rng.integers(0, 2, n), rng.standard_normal((n, 2))]).astype(float))
    W = np.array([[0, -1, -1], [1, 2, -1]], dtype=np.int32)
    plan = ab.anova_nfft_plan(X, W, 0.3, N=64, m=6, flags=ab.ANOVA_FP64)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_PER_WINDOW, 240, 1e-12)
    L, piv = _factor(torch, ab, lr, n)
    K = ok.anova_kernel_matrix(X, W, 0.3)
    K1, K0 = (ok.window_kernel_matrix(X, W[l], 0.3) for l in (1, 0))   # plan order: 2-D window first
    assert L.shape[1] < 240
    assert np.allclose(L[:, -2:] @ L[:, -2:].T, K0, atol=1e-12)
    assert np.allclose(L[:, :-2] @ L[:, :-2].T, K1, atol=1e-9)
    assert np.allclose(L @ L.T, K, atol=1e-9)
    assert piv[-2] == 0 and X[piv[-1], 0] != X[0, 0]


def test_randomised_nystrom_matches_oracle(env):
    """Q = orth(K G) with the same Box-Muller/SplitMix64 G on both sides; K G and K Q by the FP64
    plan. Z Z^T depends only on range(Q), so it is compared with the oracle's (Householder QR)."""
    torch, ab = env
    X, W, plan, K, _ = _setup(ab, n=400, seed=6)
    lr = ab.lowrank_precond_build(plan, ab.NYSTROM_RANDOM, 20, 0.0, seed=77)
    Z, piv = _factor(torch, ab, lr, 400)
    assert Z.shape == (400, 20) and np.all(piv == -1)
    Zo = op.nystrom_random(K, 20, seed=77)
    assert np.allclose(Z @ Z.T, Zo @ Zo.T, rtol=0, atol=1e-7 * np.max(K))
    # a different seed gives a different (but equally valid) approximation
    lr2 = ab.lowrank_precond_build(plan, ab.NYSTROM_RANDOM, 20, 0.0, seed=78)
    Z2, _ = _factor(torch, ab, lr2, 400)
    assert not np.allclose(Z2 @ Z2.T, Z @ Z.T, rtol=0, atol=1e-7 * np.max(K))
    assert np.min(np.linalg.eigvalsh(K - Z @ Z.T)) > -1e-6 * np.max(K)


def test_randomised_nystrom_full_rank_and_fp32_plan(env):
    torch, ab = env
    X, W, plan, K, _ = _setup(ab, n=80, ell=0.05)
    lr = ab.lowrank_precond_build(plan, ab.NYSTROM_RANDOM, 80, 0.0, seed=3)
    Z, _ = _factor(torch, ab, lr, 80)
    assert Z.shape[1] == 80
    assert np.allclose(Z @ Z.T, K, rtol=0, atol=1e-7 * np.max(K))
    p32 = ab.anova_nfft_plan(X, W, 0.05, N=32, m=4, flags=ab.ANOVA_FP32)
    with pytest.raises(ab.AnovaError):
        ab.lowrank_precond_build(p32, ab.NYSTROM_RANDOM, 10, 0.0, seed=3)


@pytest.mark.parametrize("rank", [240, 300])
def test_woodbury_at_large_rank(env, rank):
    """The core factor in packed shared memory (rank 240, the largest that fits) and in global
    memory (rank 300), with its triangular inverse, against the dense oracle."""
    torch, ab = env
    n = 700
    X, W, plan, K, rng = _setup(ab, n=n, ell=0.05, seed=9)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_GREEDY, rank, 0.0)
    L, _ = _factor(torch, ab, lr, n)
    assert L.shape[1] == rank
    L32 = L.astype(np.float32).astype(np.float64)
    y = np.where(rng.standard_normal(n) >= 0, 1.0, -1.0)
    theta = np.exp(rng.uniform(-3, 3, n))
    g = rng.standard_normal(n + 1)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    th, yy, gg = dev(theta), dev(y), dev(g)
    x = torch.empty(n + 1, dtype=torch.float64, device="cuda")
    ab.lowrank_precond_set_theta(lr, th, yy)
    ab.lowrank_precond_apply(lr, th, yy, gg, x)
    torch.cuda.synchronize()
    s = y @ op.woodbury_apply(L32, theta, y, y)
    ref = op.blockdiag_apply(L32, theta, y, g, s)
    got = x.cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-8, atol=1e-10 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n, rank", [(20000, 200), (6000, 100), (3000, 57), (700, 256)])
def test_woodbury_core_on_tensor_cores_is_fp64_accurate(env, n, rank):
    """M = I + L^T Theta^-1 L (Sec. 5) from exact bf16 slices on the tensor cores agrees with the
    FP64 evaluation of the same sum (host, from the FP32 panel the library uses) to 1e-13 of its
    norm, with Theta^-1 spread over 1e-2 .. 1e8 as late interior point steps produce it; so does the
    FP64-pipe path. Both Cholesky factors then succeed and the applies agree."""
    torch, ab = env
    from synth import config3
    cfg = config3(n=n)
    plan = ab.anova_nfft_plan(cfg["X"], cfg["windows"], 1.0, N=64, m=6, flags=ab.ANOVA_FP64)
    lr = ab.lowrank_precond_build(plan, ab.PCHOL_GREEDY, rank, 0.0)
    L, _ = _factor(torch, ab, lr, n)
    r = L.shape[1]
    assert r == rank
    L32 = L.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(rank)
    itheta = 10.0 ** rng.uniform(-2, 8, n)
    theta = 1.0 / itheta
    ref = np.eye(r) + L32.T @ (itheta[:, None] * L32)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    th, yy = dev(theta), dev(cfg["y"])
    got = {}
    for path in (ab.LOWRANK_CORE_SIMT, ab.LOWRANK_CORE_TENSOR):
        ab.lowrank_set_core_path(lr, path)
        for rep in range(2):                  # the second call reuses the slice workspace
            ab.lowrank_precond_set_theta(lr, th, yy)
            M = torch.empty((r, r), dtype=torch.float64, device="cuda")
            assert ab.lowrank_core(lr, M) == path
            got[(path, rep)] = M.cpu().numpy()
    nrm = np.linalg.norm(ref)
    for key, M in got.items():
        assert np.linalg.norm(M - ref) <= 1e-13 * nrm, (key, np.linalg.norm(M - ref) / nrm)
        assert np.array_equal(M, M.T)
    # deterministic: the tensor-core path gives the same bits call after call
    assert np.array_equal(got[(ab.LOWRANK_CORE_TENSOR, 0)], got[(ab.LOWRANK_CORE_TENSOR, 1)])
    # the default path picks the tensor cores at this rank
    ab.lowrank_set_core_path(lr, ab.LOWRANK_CORE_AUTO)
    ab.lowrank_precond_set_theta(lr, th, yy)
    assert ab.lowrank_core(lr) == ab.LOWRANK_CORE_TENSOR
